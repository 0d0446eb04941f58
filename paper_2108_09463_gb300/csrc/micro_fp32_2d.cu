// Host side of the resident 2D FP32 kernel (micro_fp32_2d.cuh): which compiled
// instance and cluster size serve each box, the work items (packs of small boxes,
// single boxes for clusters), the launch shapes and the launches.
#include <algorithm>
#include <string>
#include <vector>

#include "micro_fp32_3d_col.cuh"

#include <map>
#include <utility>

namespace hmm {

size_t res2d_slot_bytes(int nmax) { return (res2d_arena_doubles(nmax) * 8 + 255) & ~(size_t)255; }
size_t res3d_slot_bytes(int nmax) { return (res3d_arena_doubles(nmax) * 8 + 255) & ~(size_t)255; }

namespace {

const std::vector<ResVariant>& variants(int dim) {
  static const std::vector<ResVariant> all2 = [] {
    std::vector<ResVariant> v;
    int (*getters[])(const ResVariant**) = {res2d_variants_pack, res2d_variants_cluster_a,
                                            res2d_variants_cluster_b, res2d_variants_any, res2d_variants_rk4,
                                            res2d_variants_tr2};
    for (auto g : getters) {
      const ResVariant* t = nullptr;
      const int n = g(&t);
      v.insert(v.end(), t, t + n);
    }
    return v;
  }();
  static const std::vector<ResVariant> all3 = [] {
    const ResVariant* t = nullptr;
    const int n = res3d_variants(&t);
    return std::vector<ResVariant>(t, t + n);
  }();
  return dim == 3 ? all3 : all2;
}

// 3D: the z-column kernel when it may run and holds the box (slabs of 3 to kCol3S
// planes, at most kCol3MaxTerms separable terms), else the first z-slab canvas that
// holds the box (its cluster size is fixed), if its slabs fit.
bool choose3(int N, int R, int interp_k, int n_terms, size_t budget, bool allow_col3, int* vi, int* cs_out) {
  const auto& V = variants(3);
  const int Ni = N - 2 * R;
  for (int i = 0; i < (int)V.size(); ++i) {
    const ResVariant& v = V[i];
    if (v.TZ >= 0 || !allow_col3 || v.R != R || N > v.NC || n_terms > kCol3MaxTerms) continue;
    const int cs = (Ni + kCol3S - 1) / kCol3S;   // the fewest CTAs; res2d_prepare may take more
    if (cs > 16) continue;
    int LD = 0, hw = 0;
    col3_layout(N, &LD, &hw);
    const int NT = (16 * hw + 31) / 32 * 32;
    // small boxes leave a column CTA with few warps: those run on the z-slab kernel
    if (NT > kCol3MaxThreads || NT < 256) continue;
    const Col3Offsets o = col3_offsets(N, LD, NT);
    if ((size_t)o.total + kResHeaderFloats > budget) continue;
    // the set-up tables and the plane-wise interpolation buffer overlay the stage-state planes
    if ((setup_smem_doubles(3, N, interp_k, n_terms) + (size_t)3 * (2 * interp_k + 1) * N) * 2 >
        (size_t)3 * kCol3S * N * LD)
      continue;
    *vi = i;
    *cs_out = cs;
    return true;
  }
  for (int i = 0; i < (int)V.size(); ++i) {
    const ResVariant& v = V[i];
    if (v.TZ < 0 || v.R != R || v.NC < N || v.cs > Ni) continue;
    const int Sa = (Ni + v.cs - 1) / v.cs;
    if (Sa > v.SAC) continue;
    const Res3Dims d = res3_dims(v.NC, R, v.SAC);
    if ((size_t)res3_offsets(d).total + kResHeaderFloats > budget) continue;
    if ((res3_tiles(Sa, Ni, d.CPp, v.TZ) + 31) / 32 * 32 > kResThreads) continue;
    if (setup_smem_doubles(3, N, interp_k, n_terms) * 2 > (size_t)3 * d.Sc * d.PV) continue;
    *vi = i;
    *cs_out = v.cs;
    return true;
  }
  return false;
}

ResDims geom(const ResVariant& v, int N, int Sa) {
  ResDims d = v.NC > 0 ? res_dims(v.NC, v.R, v.SAC) : res_dims(N, v.R, Sa);
  d.rk4 = v.stepper;
  d.TR = v.tr > 0 ? v.tr : kResTR;
  return d;
}

int tile_rows(const ResVariant& v) { return v.tr > 0 ? v.tr : kResTR; }

// A slab of Sa rows of a box of N nodes under geometry d fits one CTA: shared
// memory (with the header), threads, and the set-up tables inside the vB region.
bool slab_fits(const ResDims& d, int N, int Sa, int interp_k, int n_terms, size_t budget_floats) {
  return (size_t)res_offsets(d).total + kResHeaderFloats <= budget_floats &&
         (res_tiles(Sa, d.CPp, d.TR) + 31) / 32 * 32 <= kResThreads && res_setup_fits(d, N, interp_k, n_terms);
}

bool cluster_ok(int cs, int Sa, int Ni, int R) {
  return cs == 1 || ((cs - 1) * Sa < Ni && Sa >= R);   // every rank has rows; halos from one neighbour
}

// The instance and cluster size for a box: the first canvas (table order: growing
// canvases) that holds it, else the box-stride instance with the smallest cluster.
bool choose(int N, int R, int interp_k, int n_terms, size_t budget, int* vi, int* cs_out, int stepper, int tr) {
  if (tr <= 0) tr = kResTR;
  const auto& V = variants(2);
  const int Ni = N - 2 * R;
  int canvases = 0;
  for (int i = 0; i < (int)V.size() && canvases < 3; ++i) {
    const ResVariant& v = V[i];
    if (v.stepper != stepper || tile_rows(v) != tr || v.R != R || v.NC == 0 || v.NC < N) continue;
    const int Sa = (Ni + v.cs - 1) / v.cs;
    if (Sa > v.SAC || !cluster_ok(v.cs, Sa, Ni, R)) continue;
    if (!slab_fits(geom(v, N, Sa), N, Sa, interp_k, n_terms, budget)) continue;
    *vi = i;
    *cs_out = v.cs;
    return true;
  }
  for (int i = 0; i < (int)V.size(); ++i) {
    const ResVariant& v = V[i];
    if (v.stepper != stepper || tile_rows(v) != kResTR || v.R != R || v.NC != 0) continue;
    if (tr != kResTR) continue;   // the box-stride instances have 4-row tiles
    for (int cs = 1; cs <= kResMaxCluster; ++cs) {
      const int Sa = (Ni + cs - 1) / cs;
      if (!cluster_ok(cs, Sa, Ni, R)) continue;
      if (!slab_fits(geom(v, N, Sa), N, Sa, interp_k, n_terms, budget)) continue;
      *vi = i;
      *cs_out = cs;
      return true;
    }
  }
  return false;
}

}  // namespace

std::vector<std::pair<int, int>> res2d_candidates(int N, int R, int interp_k, int n_terms, size_t smem_bytes,
                                                  int stepper, int tr) {
  // the (instance, cluster size) pairs worth timing for a 2D box of N nodes: the
  // heuristic's own choice first, the three smallest canvases that hold the box (a
  // larger canvas only adds idle threads and shared memory) and the box-stride
  // instance with the two smallest cluster sizes that fit
  const size_t budget = smem_bytes / sizeof(float);
  const auto& V = variants(2);
  const int Ni = N - 2 * R;
  std::vector<std::pair<int, int>> out;
  int vi = -1, cs = 0;
  if (choose(N, R, interp_k, n_terms, budget, &vi, &cs, stepper, tr)) out.emplace_back(vi, cs);
  // the three smallest canvases of 4-row tiles and the two smallest of 2-row tiles
  for (int trc : {kResTR, 2}) {
    if (tr > 0 && trc != tr) continue;
    int canvases = 0;
    for (int i = 0; i < (int)V.size() && canvases < (trc == kResTR ? 3 : 2); ++i) {
      const ResVariant& v = V[i];
      if (v.stepper != stepper || tile_rows(v) != trc || v.R != R || v.NC == 0 || v.NC < N) continue;
      const int Sa = (Ni + v.cs - 1) / v.cs;
      if (Sa > v.SAC || !cluster_ok(v.cs, Sa, Ni, R)) continue;
      if (!slab_fits(geom(v, N, Sa), N, Sa, interp_k, n_terms, budget)) continue;
      ++canvases;
      if (std::find(out.begin(), out.end(), std::make_pair(i, v.cs)) == out.end()) out.emplace_back(i, v.cs);
    }
  }
  for (int i = 0; i < (int)V.size(); ++i) {
    const ResVariant& v = V[i];
    if (v.stepper != stepper || tile_rows(v) != kResTR || v.R != R || v.NC != 0) continue;
    if (tr > 0 && tr != kResTR) continue;
    int found = 0;
    for (int c = 1; c <= kResMaxCluster && found < 2; ++c) {
      const int Sa = (Ni + c - 1) / c;
      if (!cluster_ok(c, Sa, Ni, R) || !slab_fits(geom(v, N, Sa), N, Sa, interp_k, n_terms, budget)) continue;
      ++found;
      if (std::find(out.begin(), out.end(), std::make_pair(i, c)) == out.end()) out.emplace_back(i, c);
    }
  }
  return out;
}

int res2d_variant_canvas(int vi) { return variants(2)[vi].NC; }
int res2d_variant_rows(int vi) { return tile_rows(variants(2)[vi]); }

bool res3d_plan_uses_col3(const Res2dPlan& plan) {
  if (plan.dim != 3) return false;
  for (const Res2dGroup& g : plan.groups)
    if (variants(3)[g.variant].TZ < 0) return true;
  return false;
}

bool res2d_make_plan(int dim, const BoxDesc* boxes, int n, int R, int interp_k, int n_terms, size_t smem_bytes,
                     Res2dPlan* plan, std::string* why, const std::map<int, std::pair<int, int>>* pick,
                     bool allow_col3, int stepper, int tr) {
  const size_t budget = smem_bytes / sizeof(float);
  const auto& V = variants(2);
  plan->items.clear();
  plan->groups.clear();
  plan->smem = smem_bytes;
  plan->dim = dim;
  // the instance and cluster size of a box of N nodes: the tuned pick when there is one
  auto choose_for = [&](int N, int* vi, int* cs) {
    if (pick) {
      const auto it = pick->find(N);
      if (it != pick->end()) {
        *vi = it->second.first;
        *cs = it->second.second;
        return true;
      }
    }
    return choose(N, R, interp_k, n_terms, budget, vi, cs, stepper, tr);
  };
  int i = 0;
  while (i < n) {
    int vi = -1, cs = 0;
    if (dim == 3) {
      const int N = boxes[i].N;
      if (!choose3(N, R, interp_k, n_terms, budget, allow_col3, &vi, &cs)) {
        *why = "no 3D resident instance holds a box of N = " + std::to_string(N) + " with this stencil";
        return false;
      }
      const bool col3 = variants(3)[vi].TZ < 0;
      int LD = 0, hw = 0;
      if (col3) col3_layout(N, &LD, &hw);
      const int threads = col3 ? (16 * hw + 31) / 32 * 32 : kResThreads;
      // one group per instance and cluster size (the z-column kernel: per box size)
      if (plan->groups.empty() || plan->groups.back().variant != vi || plan->groups.back().cs != cs ||
          (col3 && plan->groups.back().N != N))
        plan->groups.push_back(Res2dGroup{cs, vi, (int)plan->items.size(), 0, 0, threads, LD, col3 ? N : 0});
      plan->items.push_back(make_int2(i, 1));
      plan->groups.back().n_items++;
      ++i;
      continue;
    }
    if (!choose_for(boxes[i].N, &vi, &cs)) {
      *why = "a box of N = " + std::to_string(boxes[i].N) + " fits no cluster of at most " +
             std::to_string(kResMaxCluster) + " CTAs";
      return false;
    }
    int k = 1;
    if (cs == 1) {
      // pack consecutive boxes (sorted by size) served by the same instance
      size_t floats = kResHeaderFloats;
      int warps = 0;
      k = 0;
      while (i + k < n && k < kResMaxPack) {
        const int N = boxes[i + k].N, Ni = N - 2 * R;
        int vj = -1, csj = 0;
        if (!choose_for(N, &vj, &csj) || vj != vi || csj != 1) break;
        const ResDims dq = geom(V[vi], N, Ni);
        const size_t f = res_offsets(dq).total;
        const int w = (res_tiles(Ni, dq.CPp, dq.TR) + 31) / 32;
        if (k > 0 && (floats + f > budget || (warps + w) * 32 > kResThreads)) break;
        floats += f;
        warps += w;
        ++k;
      }
    }
    if (plan->groups.empty() || plan->groups.back().variant != vi || plan->groups.back().cs != cs)
      plan->groups.push_back(Res2dGroup{cs, vi, (int)plan->items.size(), 0, 0, kResThreads, 0, 0});
    plan->items.push_back(make_int2(i, k));
    plan->groups.back().n_items++;
    i += k;
  }
  return true;
}

static cudaLaunchConfig_t launch_config(const Res2dGroup& g, int grid, size_t smem, cudaStream_t st,
                                        cudaLaunchAttribute* at) {
  cudaLaunchConfig_t cfg = {};
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = g.cs;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(g.threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = at;
  cfg.numAttrs = g.cs > 1 ? 1 : 0;
  return cfg;
}

cudaError_t res2d_prepare(int radius, Res2dPlan* plan, int num_sms) {
  (void)radius;
  const auto& V = variants(plan->dim);
  for (Res2dGroup& g : plan->groups) {
    const void* fn = reinterpret_cast<const void*>(V[g.variant].fn);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)plan->smem);
    if (e != cudaSuccess) return e;
    if (V[g.variant].TZ < 0) {
      // z-column kernel: the cluster size that finishes boxes fastest, the clusters the
      // GPU holds at once (whole clusters per GPC) over the planes of the largest slab
      const int Ni = g.N - 2 * V[g.variant].R;
      e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      if (e != cudaSuccess) return e;
      double best = -1.0;
      int best_cs = 0, best_cl = 0;
      for (int cs = 1; cs <= 16 && cs <= Ni; ++cs) {
        const int smax = (Ni + cs - 1) / cs;
        if (smax > kCol3S) continue;
        Res2dGroup t = g;
        t.cs = cs;
        cudaLaunchAttribute at[1];
        cudaLaunchConfig_t cfg = launch_config(t, cs * num_sms, plan->smem, 0, at);
        int clusters = 0;
        if (cs == 1) {
          e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&clusters, fn, g.threads, plan->smem);
          clusters *= num_sms;
        } else {
          e = cudaOccupancyMaxActiveClusters(&clusters, fn, &cfg);
        }
        if (e != cudaSuccess) {
          cudaGetLastError();
          continue;
        }
        const double score = (double)std::min(clusters, g.n_items) / smax;
        if (clusters > 0 && score > best) {
          best = score;
          best_cs = cs;
          best_cl = clusters;
        }
      }
      if (best_cs == 0) return cudaErrorInvalidConfiguration;
      g.cs = best_cs;
      g.grid = std::min(g.n_items, best_cl) * best_cs;
      continue;
    }
    if (g.cs > 8) {   // clusters beyond the portable size of 8
      e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      if (e != cudaSuccess) return e;
    }
    if (g.cs == 1) {
      int per_sm = 0;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, g.threads, plan->smem);
      if (e != cudaSuccess) return e;
      if (per_sm < 1) return cudaErrorInvalidConfiguration;
      g.grid = std::min(g.n_items, per_sm * num_sms);
    } else {
      cudaLaunchAttribute at[1];
      cudaLaunchConfig_t cfg = launch_config(g, g.cs * num_sms, plan->smem, 0, at);
      int clusters = 0;
      e = cudaOccupancyMaxActiveClusters(&clusters, fn, &cfg);
      if (e != cudaSuccess) return e;
      if (clusters < 1) return cudaErrorInvalidConfiguration;
      g.grid = std::min(g.n_items, clusters) * g.cs;
    }
  }
  return cudaSuccess;
}

int res2d_max_grid(const Res2dPlan& plan) {
  int g = 0;
  for (const Res2dGroup& x : plan.groups) g = std::max(g, x.grid);
  return g;
}

cudaError_t res2d_launch(const MicroArgs& a, int radius, const Res2dPlan& plan, const int2* d_items,
                         int* d_queues, cudaStream_t st) {
  (void)radius;
  const auto& V = variants(plan.dim);
  for (size_t gi = 0; gi < plan.groups.size(); ++gi) {
    const Res2dGroup& g = plan.groups[gi];
    const ResLaunch L{d_items + g.first_item, g.n_items, d_queues + gi, g.cs, g.aux};
    cudaLaunchAttribute at[1];
    cudaLaunchConfig_t cfg = launch_config(g, g.grid, plan.smem, st, at);
    const cudaError_t e = cudaLaunchKernelEx(&cfg, V[g.variant].fn, a, L);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

}  // namespace hmm

// Batched FP32 micro kernel for 3D boxes on chip, z-column form.
//
// Same mathematics, perturbation form, compensated state, stage carry and
// increment-form average as the 2D resident kernel (micro_fp32_2d.cuh) and the
// z-slab 3D kernel (micro_fp32_3d.cuh), whose FP64 set-up this kernel repeats.
// What differs is how the time loop maps onto the SM:
//
//  * A box is split by z-planes over a cluster of cs CTAs, at most kCol3S interior
//    planes per CTA (the host picks cs from the clusters that fit the GPU at once:
//    9 CTAs of about 3 planes for 32^3). Each thread owns one interior row y and a
//    pair of adjacent columns (x, x+1), and walks its z-column through the whole
//    slab: a rolling window over planes -3 .. S+2 of the slab with all three
//    components interleaved, so that every z-face flux is computed once; the
//    planes beyond the slab are read from the neighbouring CTAs' shared memory
//    (distributed shared memory) and ring planes are zero.
//  * Only v^n and the stage state live in row-major planes (the stencil reads
//    neighbours); m_init, H(m_init) and H(W) are private to the thread that owns
//    the node and are stored in thread order (one float2 per thread and plane), as
//    is the carried rounding error of the state (bf16); the rounding carry of the
//    stage state lives from stage 1 to stage 2 in registers.
//  * The material coefficient is evaluated in the loop from the per-box FP32
//    tables of its separable factors (at most kCol3MaxTerms terms): per thread and
//    term, the products of the factors along the thread's fixed row and columns are
//    kept in registers, so a face coefficient costs one fma per term.
//  * Bank conflicts: the planes have a row stride LD (floats) and thread t owns
//    the tile (y, j) (j: column pair) that makes (LD/2 * y + j) mod 16 distinct
//    within every half-warp (the 16 lanes of one 64-bit shared-memory wavefront).
//    Half-warp g takes, for each residue r, the g-th tile of residue r (rows in
//    increasing order); LD is chosen on the host to make the largest residue class
//    (the number of half-warps) smallest.
#pragma once
#include <type_traits>

#include "micro_fp32_3d.cuh"

namespace hmm {

constexpr int kCol3S = 3;            // interior planes per CTA at most
constexpr int kCol3MaxTerms = 1;     // separable coefficient terms evaluated in the loop
constexpr int kCol3MaxThreads = 352; // threads per CTA at most (the launch bound)

// Row stride LD (floats) of the planes of a box of N nodes per axis and the number
// of half-warps it needs: column j is stored at offset j + 1, and the x direction
// reads up to offset N + 1, so LD >= N + 2.
__host__ __device__ inline void col3_layout(int N, int* LD_out, int* halfwarps_out) {
  const int Ni = N - 6, P = (Ni + 1) / 2;
  int best = 1 << 30, bestLD = 0;
  for (int LD = (N + 3) & ~1; LD <= N + 34; LD += 2) {
    const int L = LD / 2;
    int cnt[16] = {0};
    for (int y = 0; y < Ni; ++y)
      for (int j = 0; j < P; ++j) cnt[(L * y + j) & 15]++;
    int m = 0;
    for (int r = 0; r < 16; ++r) m = cnt[r] > m ? cnt[r] : m;
    if (m < best) {
      best = m;
      bestLD = LD;
    }
  }
  *LD_out = bestLD;
  *halfwarps_out = best;
}

// Threads of a CTA for boxes of N nodes (whole warps).
__host__ __device__ inline int col3_threads(int N) {
  int LD = 0, hw = 0;
  col3_layout(N, &LD, &hw);
  return (16 * hw + 31) / 32 * 32;
}

// Float offsets (after the header) of one CTA's arrays; NT threads, planes of N rows x LD.
struct Col3Offsets {
  int vA, vB, mi, hi, hw, lo, ctab, total;
};

__host__ __device__ inline Col3Offsets col3_offsets(int N, int LD, int NT) {
  Col3Offsets o;
  const int PV = N * LD;
  int x = 0;
  o.vA = x; x += 3 * kCol3S * PV;
  o.vB = x; x += 3 * kCol3S * PV;
  o.mi = x; x += 3 * kCol3S * NT * 2;
  o.hi = x; x += 3 * kCol3S * NT * 2;
  o.hw = x; x += kCol3S * NT * 2;
  o.lo = x; x += 3 * kCol3S * NT;   // bf16 pairs
  o.ctab = x; x += kCol3MaxTerms * 3 * (2 * N - 1);
  o.total = (x + 3) & ~3;
  return o;
}

// Tile of thread t: row y and column pair j, or false if the thread has none.
__device__ __forceinline__ bool col3_tile(int t, int Ni, int L, int* y_out, int* j_out) {
  const int P = (Ni + 1) / 2, r = t & 15, g = t >> 4;
  int cnt = 0;
  for (int y = 0; y < Ni; ++y) {
    const int j = (r - L * y) & 15;
    if (j < P) {
      if (cnt == g) {
        *y_out = y;
        *j_out = j;
        return true;
      }
      ++cnt;
    }
  }
  return false;
}

// The thread that owns tile (y, j) (the inverse of col3_tile).
__device__ __forceinline__ int col3_owner(int y, int j, int Ni, int L) {
  const int P = (Ni + 1) / 2, r = (L * y + j) & 15;
  int g = 0;
  for (int yy = 0; yy < y; ++yy) g += ((r - L * yy) & 15) < P ? 1 : 0;
  return 16 * g + r;
}

// ld.shared::cluster of a float2 at a shared::cluster byte address.
__device__ __forceinline__ float2 col3_remote(unsigned addr) { return ld_cluster2(addr); }

template <int R>
__global__ void __launch_bounds__(kCol3MaxThreads, 1)
micro_fp32_3d_col_kernel(MicroArgs a, ResLaunch L) {
  static_assert(R == 3, "the z-column kernel implements the order-4 stencil");
  constexpr int D = 3;
  extern __shared__ __align__(16) float fsm[];
  __shared__ int s_item;
  double* red = reinterpret_cast<double*>(fsm);
  double* csum = red + kResRedDoubles;
  PackBox* pk = reinterpret_cast<PackBox*>(csum + kResCsumDoubles);
  float* kahA = reinterpret_cast<float*>(pk + kResMaxPack);
  unsigned* rtab = reinterpret_cast<unsigned*>(pk + 1);   // [2][6]: planes -3..-1, S..S+2 of vA, vB
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int cs = L.cs;
  const unsigned rank = cs > 1 ? cg::this_cluster().block_rank() : 0u;
  float* kah = kahA + 6 * warp;
  const int LD = L.aux, Lh = LD / 2;
  const size_t cap = (size_t)a.nmax * a.nmax * a.nmax;
  double* mi64 = reinterpret_cast<double*>(a.arena + (size_t)blockIdx.x * a.slot_bytes);
  double* af64 = mi64 + 3 * cap;
  const float am = (float)a.alpha_micro;
  const float2 alpha2 = f2(am, am);
  const float c0f = (float)a.c0;
  const float2 c02 = f2(c0f, c0f);
  const int nterm = a.n_terms;
  double wsum = 0.0;
  for (int n = 0; n <= a.msteps; ++n) wsum += a.w64[n];

  for (;;) {
    // ---- Next box (the cluster's rank 0 takes it and tells the others).
    if (cs == 1) {
      __syncthreads();
      if (tid == 0) s_item = atomicAdd(L.queue, 1);
      __syncthreads();
    } else {
      cg::cluster_group cl = cg::this_cluster();
      cl.sync();   // every CTA is done with the previous box (its shared memory is free)
      if (rank == 0 && tid == 0) {
        const int it = atomicAdd(L.queue, 1);
        for (int q = 0; q < cs; ++q) *cl.map_shared_rank(&s_item, q) = it;
      }
      cl.sync();
    }
    const int item = s_item;
    if (item >= L.n_items) break;
    const int bi = L.items[item].x;
    const BoxDesc bd = a.boxes[bi];
    const int N = bd.N, Ni = N - 2 * R, nh = 2 * N - 1;
    const int r0 = res3_r0((int)rank, Ni, cs);
    const int S = res3_r0((int)rank + 1, Ni, cs) - r0;   // this CTA's planes (<= kCol3S)
    const int PV = N * LD;
    const Col3Offsets of = col3_offsets(N, LD, nt);
    float* base = fsm + kResHeaderFloats;
    float* vA = base + of.vA;
    float* vB = base + of.vB;
    float* miS = base + of.mi;
    float* hiS = base + of.hi;
    float* hwS = base + of.hw;
    __nv_bfloat162* loS = reinterpret_cast<__nv_bfloat162*>(base + of.lo);
    float* ctab = base + of.ctab;
    if (tid < 6 * (kCol3MaxThreads / 32)) kahA[tid] = 0.f;

    int ty = 0, tj = 0;
    const bool active = col3_tile(tid, Ni, Lh, &ty, &tj);
    const int xb0 = R + 2 * tj;                 // box column of the tile's first node
    const bool col2 = xb0 + 1 < N - R;          // odd Ni: the last pair's second column is ring

    // ---- FP64 set-up (m_init, a^eps, H(m_init), H(W)) of this CTA's planes, through the arenas.
    // Each CTA computes m_init on its own planes (the first and last CTA also on the ring
    // planes) into its arena; after a cluster barrier the face fluxes read m_init from the
    // arenas of the CTAs that own the planes (the CTAs of a cluster are consecutive blocks).
    SetupSmem smr = carve_setup(reinterpret_cast<double*>(vB), D, N, a.interp_k, a.n_terms);
    smr.red = red;
    box_setup_tables<D>(a, bd, smr);
    // the coefficient's factor tables in FP32 for the time loop
    for (int e = tid; e < kCol3MaxTerms * 3 * nh; e += nt) {
      const int t = e / (3 * nh);
      ctab[e] = t < nterm ? (float)smr.ctab[e] : 0.f;
    }
    {
      const int plo = rank == 0 ? 0 : r0 + R;
      const int phi = (int)rank == cs - 1 ? N : r0 + R + S;   // box planes [plo, phi)
      // Plane by plane: the neighbourhood contracted along the last axis (smr.part) is
      // contracted along the first axis at this plane's Lagrange weights into Q (in the
      // set-up region after its tables), then each node takes the middle axis: 5 FP64 fmas
      // per component and node instead of 30.
      const int w = 2 * a.interp_k + 1;
      double* Q = reinterpret_cast<double*>(vB) + setup_smem_doubles(D, N, a.interp_k, a.n_terms);   // [3][w][N]
      for (int zb = plo; zb < phi; ++zb) {
        const double* l0 = smr.lag + (size_t)zb * w;
        for (int e = tid; e < 3 * w * N; e += nt) {
          const int c = e / (w * N), r = e - c * w * N, a1 = r / N, jl = r - a1 * N;
          const double* pc = smr.part + (size_t)c * w * w * N;
          double acc = 0.0;
          for (int a0 = 0; a0 < w; ++a0) acc += l0[a0] * pc[((size_t)a0 * w + a1) * N + jl];
          Q[e] = acc;
        }
        __syncthreads();
        for (int e = tid; e < N * N; e += nt) {
          const int j1 = e / N, jl = e - j1 * N;
          const double* l1 = smr.lag + ((size_t)N + j1) * w;
          double P[3];
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            double acc = 0.0;
            for (int a1 = 0; a1 < w; ++a1) acc += l1[a1] * Q[((size_t)c * w + a1) * N + jl];
            P[c] = acc;
          }
          const double x = P[0] * P[0] + P[1] * P[1] + P[2] * P[2];
          // 1/sqrt(x): an FP32 estimate refined by two Newton steps in FP64
          double y = (double)rsqrtf((float)x);
          y = y * fma(-0.5 * x * y, y, 1.5);
          y = y * fma(-0.5 * x * y, y, 1.5);
          const size_t idx = (size_t)zb * N * N + e;
#pragma unroll
          for (int c = 0; c < 3; ++c) mi64[c * cap + idx] = P[c] * y;
        }
        __syncthreads();
      }
    }
    if (cs > 1) cg::this_cluster().sync(); else __syncthreads();
    {
      const size_t slot = a.slot_bytes;
      char* arena0 = a.arena + (size_t)(blockIdx.x - rank) * slot;   // rank 0's arena
      // m_init of component c at box node (zb, yb, xb), from the arena of the plane's owner
      auto mi_at = [&](int c, int zb, size_t o) {
        const int q = zb < R ? 0 : (zb >= N - R ? cs - 1 : res3_owner(zb - R, Ni, cs));
        return reinterpret_cast<const double*>(arena0 + (size_t)q * slot)[c * cap + o];
      };
      const double cs64 = 1.0 / ((24.0 * bd.dx) * (24.0 * bd.dx));
      const double* W1d = a.W64 + bd.wofs;
      double* fl3 = af64 + 3 * cap;   // [axis][4][cap] face fluxes of m_init (3) and W (4th)
      const int zo = r0 + R;           // first own plane (box coordinates)
      const int nn = Ni * Ni;
      const int zf0 = zo - 2, nzf = S + 3;   // z-faces the own nodes use: left planes zo-2 .. zo+S
      const int g0 = R - 2, ng = Ni + 3;
      const size_t sz = (size_t)N * N;
      auto bidx = [&](int zb, int yb, int xb) { return ((size_t)zb * N + yb) * N + xb; };
      auto fdiff = [](const double* u, size_t o, size_t st_) {
        return (u[o - st_] - u[o + 2 * st_]) + 27.0 * (u[o + st_] - u[o]);
      };
      const int fax = bd.fax;
      int bad = 0;
      for (int e = tid; e < nzf * nn + S * ng * Ni + S * Ni * ng; e += nt) {
        int k, zb, yb, xb;
        if (e < nzf * nn) {
          k = 0;
          zb = zf0 + e / nn;
          yb = R + (e % nn) / Ni;
          xb = R + (e % nn) % Ni;
        } else if (e < nzf * nn + S * ng * Ni) {
          const int r = e - nzf * nn;
          k = 1;
          zb = zo + r / (ng * Ni);
          yb = g0 + (r % (ng * Ni)) / Ni;
          xb = R + (r % (ng * Ni)) % Ni;
        } else {
          const int r = e - nzf * nn - S * ng * Ni;
          k = 2;
          zb = zo + r / (Ni * ng);
          yb = R + (r % (Ni * ng)) / ng;
          xb = g0 + (r % (Ni * ng)) % ng;
        }
        const size_t o = bidx(zb, yb, xb);
        const size_t st_ = k == 0 ? sz : (k == 1 ? (size_t)N : 1);
        const double af = face_value<D>(a, bd, smr, N, (int)o, k);   // the face between node o and o + e_k
        bad |= !(af > 0.0);
        double* F = fl3 + (size_t)k * 4 * cap;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          // nodes o - e_k, o, o + e_k, o + 2 e_k (along z they may belong to other CTAs)
          const double um = mi_at(c, k == 0 ? zb - 1 : zb, o - st_), u0 = mi_at(c, zb, o);
          const double u1 = mi_at(c, k == 0 ? zb + 1 : zb, o + st_), u2 = mi_at(c, k == 0 ? zb + 2 : zb, o + 2 * st_);
          F[c * cap + o] = af * ((um - u2) + 27.0 * (u1 - u0));
        }
        const double* W1f = W1d + N;
        double wd;
        if (fax < 0)
          wd = k == 0 ? W1d[yb] * W1d[xb] * fdiff(W1d, zb, 1)
                      : (k == 1 ? W1d[zb] * W1d[xb] * fdiff(W1d, yb, 1) : W1d[zb] * W1d[yb] * fdiff(W1d, xb, 1));
        else if (k != fax)
          wd = 0.0;
        else
          wd = k == 0 ? W1f[zb] * W1d[yb] * W1d[xb] : (k == 1 ? W1d[zb] * W1f[yb] * W1d[xb] : W1d[zb] * W1d[yb] * W1f[xb]);
        F[3 * cap + o] = af * wd;
      }
      if (bad) atomicOr(a.err, kErrCoefNonPositive);
      __syncthreads();
      auto fcomb = [](const double* F, size_t o, size_t st_) {
        return (F[o - 2 * st_] - F[o + st_]) + 27.0 * (F[o] - F[o - st_]);
      };
      const double cf = 1.0 / (24.0 * bd.dx);
      double s0 = 0.0, s1 = 0.0, s2 = 0.0;
      // each thread its own nodes: planes 0..S-1 of the slab, row ty, columns xb0, xb0 + 1
      // (a ring column of an odd interior gets zeros)
      if (active) {
        for (int kz = 0; kz < S; ++kz) {
          for (int h = 0; h < 2; ++h) {
            const int io = (kz * nt + tid) * 2 + h;
            if (h == 1 && !col2) {
#pragma unroll
              for (int c = 0; c < 3; ++c) {
                miS[c * kCol3S * nt * 2 + io] = 0.f;
                hiS[c * kCol3S * nt * 2 + io] = 0.f;
              }
              hwS[io] = 0.f;
              continue;
            }
            const int zb = zo + kz, yb = R + ty, xb = xb0 + h;
            const size_t idx = bidx(zb, yb, xb);
            double H[4];
#pragma unroll
            for (int c = 0; c < 4; ++c)
              H[c] = (fcomb(fl3 + c * cap, idx, sz) + fcomb(fl3 + (4 + c) * cap, idx, (size_t)N) +
                      fcomb(fl3 + (8 + c) * cap, idx, 1)) * (c < 3 || fax < 0 ? cs64 : -cf);
            const double W = fax < 0 ? W1d[zb] * W1d[yb] * W1d[xb] : 0.0;
            s0 += W * H[0];
            s1 += W * H[1];
            s2 += W * H[2];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              miS[c * kCol3S * nt * 2 + io] = (float)mi64[c * cap + idx];
              hiS[c * kCol3S * nt * 2 + io] = (float)H[c];
            }
            hwS[io] = (float)H[3];
          }
        }
      }
      if (fax >= 0) {
        // the flux of m_init over the faces along fax this CTA owns (as in the z-slab kernel)
        const double* W1f = W1d + N;
        const int na = fax == 0 ? S + (r0 == 0 ? 1 : 0) : N - 2 * R + 1;
        const int f0a = fax == 0 ? r0 + R - (r0 == 0 ? 1 : 0) : R - 1;
        const int nb_ = fax == 0 ? nn : S * Ni;
        const double* Fk = fl3 + (size_t)fax * 4 * cap;
        for (int e = tid; e < na * nb_; e += nt) {
          const int f = f0a + e / nb_, u = e % nb_;
          int zb, yb, xb;
          if (fax == 0) { zb = f; yb = R + u / Ni; xb = R + u % Ni; }
          else if (fax == 1) { zb = zo + u / Ni; yb = f; xb = R + u % Ni; }
          else { zb = zo + u / Ni; yb = R + u % Ni; xb = f; }
          const size_t o = bidx(zb, yb, xb);
          const double WF = (fax == 0 ? W1f[zb] : W1d[zb]) * (fax == 1 ? W1f[yb] : W1d[yb]) *
                            (fax == 2 ? W1f[xb] : W1d[xb]);
          s0 += WF * Fk[o] * cf;
          s1 += WF * Fk[cap + o] * cf;
          s2 += WF * Fk[2 * cap + o] * cf;
        }
      }
      block_sum3(s0, s1, s2, red);
      if (tid == 0) {
        pk[0].s0[0] = s0 * wsum;
        pk[0].s0[1] = s1 * wsum;
        pk[0].s0[2] = s2 * wsum;
      }
    }
    // every CTA of the cluster is done reading the arenas: drop this one's from L2, and
    // clear the state planes (the set-up tables overlaid vB) and the state's carries
    if (cs > 1) cg::this_cluster().sync(); else __syncthreads();
    l2_discard(mi64, res3d_arena_doubles(a.nmax) * sizeof(double), tid, nt);
    for (int e = tid; e < of.mi; e += nt) base[e] = 0.f;
    for (int e = of.lo + tid; e < of.ctab; e += nt) base[e] = 0.f;
    __syncthreads();
    // shared::cluster addresses of the planes beyond the slab (-3..-1 and S..S+2; the
    // same layout in every CTA) in vA and vB, or kRes3Ring for ring planes
    if (tid < 12) {
      const int which = tid / 6, e = tid % 6;
      const int zg = r0 + (e < 3 ? e - 3 : S + e - 3);   // interior plane index in the box
      unsigned ad = kRes3Ring;
      if (zg >= 0 && zg < Ni) {
        const int q = res3_owner(zg, Ni, cs);
        ad = cluster_addr((which ? vB : vA) + (zg - res3_r0(q, Ni, cs)) * PV, (unsigned)q);
      }
      rtab[tid] = ad;
    }
    __syncthreads();
    if (cs > 1) cluster_arrive();   // neighbours read this CTA's planes from stage 1 on

    // ---- Per-thread constants: the coefficient's factor products along the tile's row and columns.
    const int yb = R + ty;
    auto tabv = [&](int t, int ax, int j2) { return ctab[(t * 3 + ax) * nh + j2]; };
    float2 Cyx[kCol3MaxTerms], Gy[kCol3MaxTerms][4];
    float Gx[kCol3MaxTerms][5];
#pragma unroll
    for (int t = 0; t < kCol3MaxTerms; ++t) {
      const float amp = t < nterm ? (float)a.terms[t].amp : 0.f;
      const float gy = tabv(t, 1, 2 * yb);
      const float gx0 = tabv(t, 2, 2 * xb0), gx1 = tabv(t, 2, min(2 * xb0 + 2, nh - 1));
      Cyx[t] = f2(amp * gy * gx0, amp * gy * gx1);
#pragma unroll
      for (int f = 0; f < 4; ++f) {   // y-faces with left rows yb-2 .. yb+1
        const float gyh = tabv(t, 1, 2 * (yb - 2 + f) + 1);
        Gy[t][f] = f2(amp * gyh * gx0, amp * gyh * gx1);
      }
#pragma unroll
      for (int f = 0; f < 5; ++f)     // x-faces with left columns xb0-2 .. xb0+2
        Gx[t][f] = amp * gy * tabv(t, 2, min(2 * (xb0 - 2 + f) + 1, nh - 1));
    }

    const int rowoff = (yb)*LD + xb0 + 1;   // the tile in a plane of vA/vB (column j at offset j + 1)
    const int cstrV = kCol3S * PV, cstrI = kCol3S * nt * 2;
    const float dtf = (float)bd.dt;
    const float csf = (float)(1.0 / ((24.0 * bd.dx) * (24.0 * bd.dx)));
    const float2 cs2 = f2(csf, csf);
    const float2 dt2 = f2(dtf, dtf), hdt2 = f2(0.5f * dtf, 0.5f * dtf);
    const float2 half2 = f2(0.5f, 0.5f);
    const float2 k27 = f2(27.f, 27.f);
    const int zo = r0 + R;
    __nv_bfloat162 eB[3][kCol3S];   // loS (the state's carry) was zeroed with the planes
#pragma unroll
    for (int k = 0; k < kCol3S; ++k)
#pragma unroll
      for (int c = 0; c < 3; ++c) eB[c][k] = __float2bfloat162_rn(0.f);

    for (int n = 0; n < a.msteps; ++n) {
      const float om = a.om32[n + 1];
#pragma unroll 1
      for (int stage = 0; stage < 2; ++stage) {
        const float* src = stage == 0 ? vA : vB;
        const unsigned* rt = rtab + 6 * stage;
        // The tile's own values of the stage's state and the addresses of the planes beyond
        // the slab need no barrier (this thread stored the former, the latter are fixed per
        // box), so they are loaded before it and arrive while it completes.
        float2 vk[kCol3S][3];
        unsigned rtl[6];
        if (active) {
#pragma unroll
          for (int k = 0; k < kCol3S; ++k)
            if (k < S) {
#pragma unroll
              for (int c = 0; c < 3; ++c) vk[k][c] = lds2(src + c * cstrV + k * PV + rowoff);
            }
#pragma unroll
          for (int e = 0; e < 6; ++e) rtl[e] = rt[e];
        }
        if (cs > 1) cluster_wait(); else __syncthreads();
        float2 part2[3] = {f2(0.f, 0.f), f2(0.f, 0.f), f2(0.f, 0.f)};
        // y and x directions of the stencil at slab plane k (local planes only), v0 the
        // tile's own values there: into Hs
        auto yx_pass = [&](int k, const float2* v0s, float2* Hs) {
          const float* Pk = src + k * PV + rowoff;
          float2 ay[4] = {c02, c02, c02, c02};
          float ax[5] = {c0f, c0f, c0f, c0f, c0f};
#pragma unroll
          for (int t = 0; t < kCol3MaxTerms; ++t) {
            const float gz = tabv(t, 0, 2 * (zo + k));
#pragma unroll
            for (int q = 0; q < 4; ++q) ay[q] = fma2(f2(gz, gz), Gy[t][q], ay[q]);
#pragma unroll
            for (int q = 0; q < 5; ++q) ax[q] = fmaf(gz, Gx[t][q], ax[q]);
          }
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const float* P = Pk + c * cstrV;
            const float2 v0 = v0s[c];
            // y direction: rows y-3 .. y+3 of plane k, faces y-2|y-1 .. y+1|y+2
            const float2 vm3 = lds2(P - 3 * LD), vm2 = lds2(P - 2 * LD), vm1 = lds2(P - LD);
            const float2 vp1 = lds2(P + LD), vp2 = lds2(P + 2 * LD), vp3 = lds2(P + 3 * LD);
            const float2 Ya = mul2(ay[0], fma2(k27, sub2(vm1, vm2), sub2(vm3, v0)));
            const float2 Yb = mul2(ay[1], fma2(k27, sub2(v0, vm1), sub2(vm2, vp1)));
            const float2 Yc = mul2(ay[2], fma2(k27, sub2(vp1, v0), sub2(vm1, vp2)));
            const float2 Yd = mul2(ay[3], fma2(k27, sub2(vp2, vp1), sub2(v0, vp3)));
            const float2 h = fma2(k27, sub2(Yc, Yb), sub2(Ya, Yd));
            // x direction: columns x-3 .. x+4 of the row, faces x-2|x-1 .. x+2|x+3
            // (a 64-bit load for the one column past R1 keeps the access conflict-free)
            const float2 L1 = lds2(P - 2), R1 = lds2(P + 2), L2 = lds2(P - 4);
            const float r2x = lds2(P + 4).x;
            const float2 g01 = fma2(k27, sub2(shift2(L1, v0), L1), sub2(shift2(L2, L1), v0));
            const float2 g23 = fma2(k27, sub2(shift2(v0, R1), v0), sub2(shift2(L1, v0), R1));
            const float g4 = (v0.y - r2x) + 27.f * (R1.y - R1.x);
            const float2 F01 = mul2(f2(ax[0], ax[1]), g01), F23 = mul2(f2(ax[2], ax[3]), g23);
            const float F4 = ax[4] * g4;
            Hs[c] = add2(h, fma2(k27, sub2(F23, shift2(F01, F23)), sub2(F01, f2(F23.y, F4))));
          }
        };
        // One stage on a slab of SS planes (a compile-time count, so that every plane
        // value lives in registers): the loads of the six planes beyond the slab go out
        // first, the y and x directions of all own planes (independent of them) follow,
        // then the z direction walks planes -3 .. SS+2 and each finished plane is updated.
        auto stage_body = [&](auto ssc) {
          constexpr int SS = decltype(ssc)::value;
          float2 rem[6][3];
#pragma unroll
          for (int e = 0; e < 6; ++e) {
            const unsigned b = rtl[e];
            if (b == kRes3Ring) {
#pragma unroll
              for (int c = 0; c < 3; ++c) rem[e][c] = f2(0.f, 0.f);
            } else {
#pragma unroll
              for (int c = 0; c < 3; ++c) rem[e][c] = col3_remote(b + 4u * (unsigned)(c * cstrV + rowoff));
            }
          }
          float2 Hk[SS][3];
#pragma unroll
          for (int k = 0; k < SS; ++k) yx_pass(k, vk[k], Hk[k]);
          auto val = [&](int z, int c) -> float2 { return z < 0 ? rem[z + 3][c] : (z < SS ? vk[z][c] : rem[z - SS + 3][c]); };
          float2 Fa[3], Fb[3], Fc[3];
#pragma unroll
          for (int f = -2; f <= SS; ++f) {
            // z-face between slab planes f and f + 1
            float2 az = c02;
#pragma unroll
            for (int t = 0; t < kCol3MaxTerms; ++t) {
              const float g = tabv(t, 0, 2 * (zo + f) + 1);
              az = fma2(f2(g, g), Cyx[t], az);
            }
            float2 F[3];
#pragma unroll
            for (int c = 0; c < 3; ++c)
              F[c] = mul2(az, fma2(k27, sub2(val(f + 1, c), val(f, c)), sub2(val(f - 1, c), val(f + 2, c))));
            if (f >= 1) {
              const int k = f - 1;   // plane k is complete in z
              float2 Hs[3], p0[3];
#pragma unroll
              for (int c = 0; c < 3; ++c) {
                Hs[c] = add2(Hk[k][c], fma2(k27, sub2(Fc[c], Fb[c]), sub2(Fa[c], F[c])));
                p0[c] = vk[k][c];
              }
              const int io = (k * nt + tid) * 2;
              if (stage == 0) {
                // Stage 1: k1 = f(m_init + v, H(m_init) + H(v)); vB = v + dt k1.
                float2 v[3], m[3], H[3], fr[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                  v[c] = p0[c];
                  m[c] = add2(lds2(miS + c * cstrI + io), v[c]);
                  H[c] = fma2(Hs[c], cs2, lds2(hiS + c * cstrI + io));
                }
                ll_rhs2(m, H, alpha2, fr);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                  float2 vb = fma2(dt2, fr[c], v[c]);
                  eB[c][k] = __float22bfloat162_rn(fma2(hdt2, fr[c], mul2(half2, sub2(v[c], vb))));
                  if (!col2) vb.y = 0.f;
                  *reinterpret_cast<float2*>(vB + c * cstrV + k * PV + rowoff) = vb;
                }
              } else {
                // Stage 2: k2 = f(m_init + vB); v += dt/2 (k1 + k2) + projection, compensated.
                float2 mi[3], m[3], H[3], k2[3], vh[3], dd[3], vt[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                  mi[c] = lds2(miS + c * cstrI + io);
                  m[c] = add2(mi[c], p0[c]);
                  H[c] = fma2(Hs[c], cs2, lds2(hiS + c * cstrI + io));
                }
                ll_rhs2(m, H, alpha2, k2);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                  vh[c] = lds2(vA + c * cstrV + k * PV + rowoff);
                  dd[c] = fma2(hdt2, k2[c], fma2(half2, sub2(p0[c], vh[c]), __bfloat1622float2(eB[c][k])));
                  vt[c] = add2(vh[c], dd[c]);
                }
                const float2 hw = lds2(hwS + io);
                float2 sdot = mul2(mi[0], vt[0]);
                sdot = fma2(mi[1], vt[1], sdot);
                sdot = fma2(mi[2], vt[2], sdot);
                float2 sq = mul2(vt[0], vt[0]);
                sq = fma2(vt[1], vt[1], sq);
                sq = fma2(vt[2], vt[2], sq);
                const float2 s = fma2(f2(2.f, 2.f), sdot, sq);
                const float rr0 = rsqrtf(1.f + s.x), rr1 = rsqrtf(1.f + s.y);
                const float2 cf = f2(__fdividef(-s.x * rr0 * rr0, 1.f + rr0), __fdividef(-s.y * rr1 * rr1, 1.f + rr1));
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                  __nv_bfloat162* lo = loS + (c * kCol3S + k) * nt + tid;
                  const float2 inc = add2(fma2(cf, add2(mi[c], vt[c]), dd[c]), __bfloat1622float2(*lo));
                  float2 nv = add2(vh[c], inc);
                  *lo = __float22bfloat162_rn(sub2(inc, sub2(nv, vh[c])));
                  if (!col2) nv.y = 0.f;
                  *reinterpret_cast<float2*>(vA + c * cstrV + k * PV + rowoff) = nv;
                  part2[c] = fma2(hw, sub2(nv, vh[c]), part2[c]);
                }
              }
          }
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              Fa[c] = Fb[c];
              Fb[c] = Fc[c];
              Fc[c] = F[c];
            }
          }
        };
        if (active) {
          if (S == 3) stage_body(std::integral_constant<int, 3>{});
          else if (S == 2) stage_body(std::integral_constant<int, 2>{});
          else stage_body(std::integral_constant<int, 1>{});
        }
        // arrive first: the warp's Kahan sum touches only its own shared-memory slots
        if (cs > 1) cluster_arrive();
        if (stage == 1 && om != 0.f) {
          float part[3] = {part2[0].x + part2[0].y, part2[1].x + part2[1].y, part2[2].x + part2[2].y};
          warp_kahan_add(kah, lane, om, part);
        }
      }
    }
    if (cs > 1) cluster_wait();   // pairs the last arrive

    // ---- H_avg: s0 plus the warps' Kahan sums; the slabs are added in rank order on rank 0.
    __syncthreads();
    if (tid == 0) {
      double acc[3] = {pk[0].s0[0], pk[0].s0[1], pk[0].s0[2]};
      for (int w = 0; w < nt / 32; ++w)
#pragma unroll
        for (int c = 0; c < 3; ++c) acc[c] += (double)kahA[6 * w + c] - (double)kahA[6 * w + 3 + c];
      if (cs == 1) {
        double* out = bd.fax >= 0 ? a.Fout + (size_t)bd.fax * 3 * a.P : a.Havg;
        out[bd.p] = acc[0];
        out[a.P + bd.p] = acc[1];
        out[2 * a.P + bd.p] = acc[2];
        if (!(isfinite(acc[0]) && isfinite(acc[1]) && isfinite(acc[2]))) atomicOr(a.err, kErrNonFinite);
      } else {
        double* dst = cg::this_cluster().map_shared_rank(csum, 0u) + 4 * rank;
        dst[0] = acc[0];
        dst[1] = acc[1];
        dst[2] = acc[2];
      }
    }
    if (cs > 1) {
      cg::this_cluster().sync();
      if (rank == 0 && tid == 0) {
        double acc[3] = {0.0, 0.0, 0.0};
        for (int r = 0; r < cs; ++r)
#pragma unroll
          for (int c = 0; c < 3; ++c) acc[c] += csum[4 * r + c];
        double* out = bd.fax >= 0 ? a.Fout + (size_t)bd.fax * 3 * a.P : a.Havg;
        out[bd.p] = acc[0];
        out[a.P + bd.p] = acc[1];
        out[2 * a.P + bd.p] = acc[2];
        if (!(isfinite(acc[0]) && isfinite(acc[1]) && isfinite(acc[2]))) atomicOr(a.err, kErrNonFinite);
      }
    }
  }
}

}  // namespace hmm

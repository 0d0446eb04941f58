// Batched FP32 micro kernel for 3D boxes held on chip, each box split by z-planes
// over a thread-block cluster.
//
// The mathematics, the perturbation form, the compensated state, the stage carry
// and the average over state increments are those of the 2D resident kernel
// (micro_fp32_2d.cuh, whose helpers this file uses). The 3D box does not fit one
// SM: a cluster of cs CTAs shares it, CTA q holding the interior z-planes
// [r0(q), r0(q+1)), r0(q) = floor(q Ni / cs). Each CTA keeps only its own planes in
// shared memory; the stencil reads the r planes beyond its slab from the
// neighbouring CTAs' shared memory (distributed shared memory) and takes ring
// planes as zero. Two cluster barriers per step order these reads: every CTA
// finishes stage 1 (which reads v^n everywhere) before any writes v^{n+1}, and
// finishes stage 2 (which reads the stage state) before any overwrites it.
//
// Thread tiles: TZ planes x 2 adjacent x-columns at one interior row y; the z
// direction walks a rolling window over planes and face fluxes, the y direction
// reads rows y-r..y+r of the same plane, the x direction is the 2D kernel's
// column stencil. Tiles are numbered (plane group, y, column pair) with the column
// pairs padded to CPp as in 2D (every row a half-warp or a warp, or bank-congruent
// strides), so shared-memory wavefronts stay conflict-free.
#pragma once
#include "micro_fp32_2d.cuh"

namespace hmm {

// Dimensions of one CTA's slab of a 3D box of N nodes per axis, Sc planes of capacity.
struct Res3Dims {
  int N, Ni, Sc;
  int LD;    // row stride of vA/vB (column j at offset j + 1)
  int LDI;   // row stride of the interior arrays
  int LDY;   // row stride of the x-face array
  int CPp;   // tiles per row
  int PV, PI, PY, PFY;   // plane strides: vA/vB, interior arrays, x-faces, y-faces
};

__host__ __device__ inline Res3Dims res3_dims(int N, int R, int Sc) {
  Res3Dims d;
  d.N = N;
  d.Ni = N - 2 * R;
  d.Sc = Sc;
  d.CPp = res_cp_pad(d.Ni);
  // the x-direction reads columns up to j0 + 4: N + 2 for odd Ni, N - 1 for even Ni
  d.LD = res_stride((d.Ni & 1) ? N + 4 : N + 2, d.CPp);
  d.LDI = res_stride(d.Ni, d.CPp);
  d.LDY = res_stride(d.Ni + (R == 3 ? 4 : 2), d.CPp);
  d.PV = N * d.LD;
  d.PI = d.Ni * d.LDI;
  d.PY = d.Ni * d.LDY;
  d.PFY = (d.Ni + (R == 3 ? 3 : 1)) * d.LDI;
  return d;
}

template <int R, int NC, int SAC>
__host__ __device__ inline Res3Dims res3_geom(int N, int Sa) {
  return NC > 0 ? res3_dims(NC, R, SAC) : res3_dims(N, R, Sa);
}

struct Res3Offsets {
  int vA, vB, mi, hi, hw, fx, fy, fz, total;
};

__host__ __device__ inline Res3Offsets res3_offsets(const Res3Dims& d) {
  Res3Offsets o;
  const int nfz = d.Sc + (d.N - d.Ni == 6 ? 3 : 1);
  int x = 0;
  o.vA = x; x += 3 * d.Sc * d.PV;
  o.vB = x; x += 3 * d.Sc * d.PV;
  o.mi = x; x += 3 * d.Sc * d.PI;
  o.hi = x; x += 3 * d.Sc * d.PI;
  o.hw = x; x += d.Sc * d.PI;
  o.fx = x; x += d.Sc * d.PY;
  o.fy = x; x += d.Sc * d.PFY;
  o.fz = x; x += nfz * d.PI;
  o.total = (x + 3) & ~3;
  return o;
}

// Tiles (threads) of a slab of S planes of a box with Ni interior nodes per axis,
// TZ planes per tile.
__host__ __device__ inline int res3_tiles(int S, int Ni, int CPp, int TZ) {
  return ((S + TZ - 1) / TZ) * Ni * CPp;
}

// First interior plane of rank q's slab.
__host__ __device__ inline int res3_r0(int q, int Ni, int cs) { return (q * Ni) / cs; }
// The rank whose slab holds interior plane z.
__host__ __device__ inline int res3_owner(int z, int Ni, int cs) { return ((z + 1) * cs - 1) / Ni; }

// per CTA: m_init (3), face coefficients (3), face fluxes of m_init and W per axis (3 x 4)
__host__ __device__ inline size_t res3d_arena_doubles(int nmax) { return (size_t)18 * nmax * nmax * nmax; }

// y direction of the stencil for one plane and one component: rows y-r..y+r of the
// plane (P points at the tile's row, column j0), faces between rows from fyp (the
// face between interior rows g-2 and g-1 at row g of the array, row stride LDI).
template <int R>
__device__ __forceinline__ float2 ypass(const float* __restrict__ P, int LD, const float* __restrict__ fyp, int LDI) {
  const float2 k27 = f2(27.f, 27.f);
  if (R == 3) {
    const float2 vm3 = lds2(P - 3 * LD), vm2 = lds2(P - 2 * LD), vm1 = lds2(P - LD), v0 = lds2(P);
    const float2 vp1 = lds2(P + LD), vp2 = lds2(P + 2 * LD), vp3 = lds2(P + 3 * LD);
    // faces y-2|y-1, y-1|y, y|y+1, y+1|y+2 (rows y, y+1, y+2, y+3 of the face array)
    const float2 Fa = mul2(lds2(fyp), fma2(k27, sub2(vm1, vm2), sub2(vm3, v0)));
    const float2 Fb = mul2(lds2(fyp + LDI), fma2(k27, sub2(v0, vm1), sub2(vm2, vp1)));
    const float2 Fc = mul2(lds2(fyp + 2 * LDI), fma2(k27, sub2(vp1, v0), sub2(vm1, vp2)));
    const float2 Fd = mul2(lds2(fyp + 3 * LDI), fma2(k27, sub2(vp2, vp1), sub2(v0, vp3)));
    return fma2(k27, sub2(Fc, Fb), sub2(Fa, Fd));
  } else {
    const float2 vm1 = lds2(P - LD), v0 = lds2(P), vp1 = lds2(P + LD);
    const float2 Fa = mul2(lds2(fyp), sub2(v0, vm1));
    const float2 Fb = mul2(lds2(fyp + LDI), sub2(vp1, v0));
    return sub2(Fb, Fa);
  }
}

// x direction for one row and one component (the 2D kernel's column stencil):
// row points at column j0, ay at the row's x-faces from column pair jj0.
template <int R>
__device__ __forceinline__ float2 xpass(const float* __restrict__ row, const float* __restrict__ ay) {
  const float2 k27 = f2(27.f, 27.f);
  const float2 C = lds2(row), L1 = lds2(row - 2), R1 = lds2(row + 2);
  if (R == 3) {
    const float2 L2 = lds2(row - 4);
    const float r2x = row[4];
    const float2 a01 = lds2(ay), a23 = lds2(ay + 2);
    const float a4 = ay[4];
    const float2 g01 = fma2(k27, sub2(shift2(L1, C), L1), sub2(shift2(L2, L1), C));
    const float2 g23 = fma2(k27, sub2(shift2(C, R1), C), sub2(shift2(L1, C), R1));
    const float g4 = (C.y - r2x) + 27.f * (R1.y - R1.x);
    const float2 F01 = mul2(a01, g01), F23 = mul2(a23, g23);
    const float F4 = a4 * g4;
    return fma2(k27, sub2(F23, shift2(F01, F23)), sub2(F01, f2(F23.y, F4)));
  } else {
    const float2 a01 = lds2(ay);
    const float a2 = ay[2];
    const float2 g01 = sub2(C, shift2(L1, C));
    const float g2 = R1.x - C.y;
    const float2 F01 = mul2(a01, g01);
    const float F2 = a2 * g2;
    return sub2(f2(F01.y, F2), F01);
  }
}

// The shared::cluster address of a location in the shared memory of CTA q of the cluster.
__device__ __forceinline__ unsigned cluster_addr(const void* p, unsigned q) {
  unsigned r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"((unsigned)__cvta_generic_to_shared(p)), "r"(q));
  return r;
}

__device__ __forceinline__ float2 ld_cluster2(unsigned addr) {
  float2 v;
  asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr));
  return v;
}

constexpr unsigned kRes3Ring = 0xffffffffu;   // table entry of a ring plane (zero)

// Split cluster barrier: arrive (release: this thread's shared-memory writes become
// visible to the cluster) and wait (acquire). Executed by every thread of every CTA.
__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }

// z direction for one component over the tile's TZ planes, added to H: a rolling window over the
// planes zl = z0-r .. z0+TZ+r-1 of the slab (local planes from this CTA's shared
// memory; planes of the neighbouring slabs through the table rtab, indexed by zl + r,
// of their shared::cluster addresses (component 0, row 0); ring planes zero) and over
// the face fluxes (fzp: the tile's column in the z-face array, plane stride PI).
template <int R, int TZ>
__device__ __forceinline__ void zpass(const float* __restrict__ Vc, int coff, int PV, int rowoff, int z0, int S,
                                      const unsigned* __restrict__ rtab, const float* __restrict__ fzp, int nfz, int PI,
                                      float2* H) {
  auto ld = [&](int k) -> float2 {
    const int zl = z0 - R + k;
    if (zl >= 0 && zl < S) return lds2(Vc + zl * PV + rowoff);
    const unsigned b = rtab[zl + R];
    if (b == kRes3Ring) return f2(0.f, 0.f);
    return ld_cluster2(b + 4u * (unsigned)(coff + rowoff));
  };
  auto fz = [&](int f) { return lds2(fzp + min(z0 + f, nfz - 1) * PI); };
  const float2 k27 = f2(27.f, 27.f);
  if (R == 3) {
    float2 p0 = ld(0), p1 = ld(1), p2 = ld(2);
    float2 Fa = f2(0.f, 0.f), Fb = Fa, Fc = Fa;
#pragma unroll
    for (int f = 0; f < TZ + 3; ++f) {
      const float2 p3 = ld(f + 3);
      const float2 F = mul2(fz(f), fma2(k27, sub2(p2, p1), sub2(p0, p3)));
      if (f >= 3) H[f - 3] = add2(H[f - 3], fma2(k27, sub2(Fc, Fb), sub2(Fa, F)));
      Fa = Fb;
      Fb = Fc;
      Fc = F;
      p0 = p1;
      p1 = p2;
      p2 = p3;
    }
  } else {
    float2 p0 = ld(0), Fa = f2(0.f, 0.f);
#pragma unroll
    for (int f = 0; f < TZ + 1; ++f) {
      const float2 p1 = ld(f + 1);
      const float2 F = mul2(fz(f), sub2(p1, p0));
      if (f >= 1) H[f - 1] = add2(H[f - 1], sub2(F, Fa));
      Fa = F;
      p0 = p1;
    }
  }
}

template <int R, int TZ, int NC, int SAC>
__global__ void __launch_bounds__(kResThreads)
micro_fp32_3d_kernel(MicroArgs a, ResLaunch L) {
  constexpr int D = 3;
  extern __shared__ __align__(16) float fsm[];
  __shared__ int s_item;
  double* red = reinterpret_cast<double*>(fsm);
  double* csum = red + kResRedDoubles;
  PackBox* pk = reinterpret_cast<PackBox*>(csum + kResCsumDoubles);
  float* kahA = reinterpret_cast<float*>(pk + kResMaxPack);
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int cs = L.cs;
  const unsigned rank = cs > 1 ? cg::this_cluster().block_rank() : 0u;
  float* kah = kahA + 6 * warp;
  const size_t cap = (size_t)a.nmax * a.nmax * a.nmax;
  double* mi64 = reinterpret_cast<double*>(a.arena + (size_t)blockIdx.x * a.slot_bytes);
  double* af64 = mi64 + 3 * cap;
  const float am = (float)a.alpha_micro;
  const float2 alpha2 = f2(am, am);
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
    const int N = bd.N, Ni = N - 2 * R;
    const int r0 = res3_r0((int)rank, Ni, cs);
    const int S = res3_r0((int)rank + 1, Ni, cs) - r0;      // this CTA's planes
    const int Sa = (Ni + cs - 1) / cs;                        // the largest slab
    const Res3Dims d = res3_geom<R, NC, SAC>(N, Sa);
    const Res3Offsets of = res3_offsets(d);
    const int base = kResHeaderFloats;
    float* vA = fsm + base + of.vA;
    float* vB = fsm + base + of.vB;
    if (tid < 6 * (kResThreads / 32)) kahA[tid] = 0.f;
    if (tid == 0) {
      pk[0].box = bi;
      pk[0].r0 = r0;
      pk[0].S = S;
      pk[0].Sa = Sa;
      pk[0].base = base;
    }

    // ---- FP64 set-up of this CTA's planes and their halo: m_init (Section 4.1), a^eps.
    {
      SetupSmem smr = carve_setup(reinterpret_cast<double*>(vB), D, N, a.interp_k, a.n_terms);
      smr.red = red;
      box_setup_tables<D>(a, bd, smr);
      const int plo = r0, phi = min(N, r0 + S + 2 * R);   // box planes
      int bad = 0;
      for (int idx = plo * N * N + tid; idx < phi * N * N; idx += nt) {
        double P[3];
        interp_P<D>(a, smr, N, idx, P);
        const double inv = 1.0 / sqrt(P[0] * P[0] + P[1] * P[1] + P[2] * P[2]);
#pragma unroll
        for (int c = 0; c < 3; ++c) mi64[c * cap + idx] = P[c] * inv;
        int j[3];
        node_coords<D>(idx, N, j);
#pragma unroll
        for (int k = 0; k < D; ++k) {
          double v = 0.0;
          if (j[k] < N - 1) {
            v = face_value<D>(a, bd, smr, N, idx, k);
            bad |= !(v > 0.0);
          }
          af64[k * cap + idx] = v;
        }
      }
      if (bad) atomicOr(a.err, kErrCoefNonPositive);
    }
    __syncthreads();   // the set-up tables (overlaying vB) are no longer needed
    for (int e = tid; e < of.total; e += nt) fsm[base + e] = 0.f;
    __syncthreads();
    {
      const int f0 = R == 3 ? R - 2 : R - 1;
      const int nfy = Ni + (R == 3 ? 3 : 1);
      const int nfz = S + (R == 3 ? 3 : 1);
      float* miS = fsm + base + of.mi;
      float* hiS = fsm + base + of.hi;
      float* hwS = fsm + base + of.hw;
      float* fxS = fsm + base + of.fx;
      float* fyS = fsm + base + of.fy;
      float* fzS = fsm + base + of.fz;
      auto bidx = [&](int zb, int yb, int xb) { return ((size_t)zb * N + yb) * N + xb; };
      const int nn = Ni * Ni;
      for (int e = tid; e < 3 * S * nn; e += nt) {
        const int c = e / (S * nn), r = e - c * S * nn;
        const int z = r / nn, yx = r - z * nn, y = yx / Ni, x = yx - y * Ni;
        miS[(c * d.Sc + z) * d.PI + y * d.LDI + x] = (float)mi64[c * cap + bidx(r0 + z + R, y + R, x + R)];
      }
      for (int e = tid; e < S * Ni * nfy; e += nt) {   // x-faces: between columns g+f0, g+f0+1
        const int z = e / (Ni * nfy), r = e - z * Ni * nfy, y = r / nfy, g = r - y * nfy;
        fxS[z * d.PY + y * d.LDY + g] = (float)af64[2 * cap + bidx(r0 + z + R, y + R, g + f0)];
      }
      for (int e = tid; e < S * nfy * Ni; e += nt) {   // y-faces: between rows g+f0, g+f0+1
        const int z = e / (nfy * Ni), r = e - z * nfy * Ni, g = r / Ni, x = r - g * Ni;
        fyS[z * d.PFY + g * d.LDI + x] = (float)af64[cap + bidx(r0 + z + R, g + f0, x + R)];
      }
      for (int e = tid; e < nfz * nn; e += nt) {       // z-faces: between planes r0+f+f0, +1
        const int f = e / nn, yx = e - f * nn, y = yx / Ni, x = yx - y * Ni;
        fzS[f * d.PI + y * d.LDI + x] = (float)af64[bidx(r0 + f + f0, y + R, x + R)];
      }
      const double cs64 = R == 3 ? 1.0 / ((24.0 * bd.dx) * (24.0 * bd.dx)) : 1.0 / (bd.dx * bd.dx);
      const double* W1d = a.W64 + bd.wofs;
      // H(m_init) and H(W) in FP64, face fluxes first (each face once): components 0-2
      // of m_init and, as a fourth, W = W(z) W(y) W(x), whose face differences factor
      // into 1D differences of the weight table. Per axis k the fluxes at the faces
      // between nodes j and j + e_k that the slab's interior nodes use.
      double* fl3 = af64 + 3 * cap;   // [axis][4][cap]
      const int fl = R == 3 ? 2 : 1, fh = R == 3 ? 1 : 0;   // a node uses faces j-fl .. j+fh
      const int zf0 = r0 + R - fl, nzf = S + fl + fh;       // z-face planes
      const int g0 = R - fl, ng = Ni + fl + fh;              // y- and x-face rows/columns
      const int zo = r0 + R;                                 // first own plane (box coordinates)
      auto fdiff = [](const double* u, size_t o, size_t st_) {
        return R == 3 ? (u[o - st_] - u[o + 2 * st_]) + 27.0 * (u[o + st_] - u[o]) : u[o + st_] - u[o];
      };
      const size_t sz = (size_t)N * N;
      for (int e = tid; e < nzf * nn + S * ng * Ni + S * Ni * ng; e += nt) {
        int k, zb, yb, xb;
        if (e < nzf * nn) {                          // z-faces
          k = 0;
          zb = zf0 + e / nn;
          yb = R + (e % nn) / Ni;
          xb = R + (e % nn) % Ni;
        } else if (e < nzf * nn + S * ng * Ni) {     // y-faces
          const int r = e - nzf * nn;
          k = 1;
          zb = zo + r / (ng * Ni);
          yb = g0 + (r % (ng * Ni)) / Ni;
          xb = R + (r % (ng * Ni)) % Ni;
        } else {                                     // x-faces
          const int r = e - nzf * nn - S * ng * Ni;
          k = 2;
          zb = zo + r / (Ni * ng);
          yb = R + (r % (Ni * ng)) / ng;
          xb = g0 + (r % (Ni * ng)) % ng;
        }
        const size_t o = bidx(zb, yb, xb);
        const size_t st_ = k == 0 ? sz : (k == 1 ? (size_t)N : 1);
        const double af = af64[k * cap + o];
        double* F = fl3 + (size_t)k * 4 * cap;
#pragma unroll
        for (int c = 0; c < 3; ++c) F[c * cap + o] = af * fdiff(mi64 + c * cap, o, st_);
        // flux model (bd.fax = axis): the fourth component holds W_f a_f on the faces
        // along that axis (face weights after the node weights in the table), so that
        // -fcomb of it is the node weight of the flux average (summation by parts)
        const double* W1f = W1d + N;
        double wd;
        if (bd.fax < 0)
          wd = k == 0 ? W1d[yb] * W1d[xb] * fdiff(W1d, zb, 1)
                      : (k == 1 ? W1d[zb] * W1d[xb] * fdiff(W1d, yb, 1) : W1d[zb] * W1d[yb] * fdiff(W1d, xb, 1));
        else if (k != bd.fax)
          wd = 0.0;
        else
          wd = k == 0 ? W1f[zb] * W1d[yb] * W1d[xb] : (k == 1 ? W1d[zb] * W1f[yb] * W1d[xb] : W1d[zb] * W1d[yb] * W1f[xb]);
        F[3 * cap + o] = af * wd;
      }
      __syncthreads();
      auto fcomb = [](const double* F, size_t o, size_t st_) {
        return R == 3 ? (F[o - 2 * st_] - F[o + st_]) + 27.0 * (F[o] - F[o - st_]) : F[o] - F[o - st_];
      };
      double s0 = 0.0, s1 = 0.0, s2 = 0.0;
      const int fax = bd.fax;
      const double cf = R == 3 ? 1.0 / (24.0 * bd.dx) : 1.0 / bd.dx;
      for (int e = tid; e < S * nn; e += nt) {
        const int z = e / nn, yx = e - z * nn, y = yx / Ni, x = yx - y * Ni;
        const size_t idx = bidx(r0 + z + R, y + R, x + R);
        double H[4];
#pragma unroll
        for (int c = 0; c < 4; ++c)
          H[c] = (fcomb(fl3 + c * cap, idx, sz) + fcomb(fl3 + (4 + c) * cap, idx, (size_t)N) +
                  fcomb(fl3 + (8 + c) * cap, idx, 1)) * (c < 3 || fax < 0 ? cs64 : -cf);
        const double W = fax < 0 ? W1d[r0 + z + R] * W1d[y + R] * W1d[x + R] : 0.0;
        s0 += W * H[0];
        s1 += W * H[1];
        s2 += W * H[2];
        const int io = z * d.PI + y * d.LDI + x;
#pragma unroll
        for (int c = 0; c < 3; ++c) hiS[c * d.Sc * d.PI + io] = (float)H[c];
        hwS[io] = (float)H[3];
      }
      if (fax >= 0) {
        // the flux of m_init over the faces along fax this CTA owns: along z the face
        // planes [r0 + R, r0 + R + S) (and R - 1 in the first slab), along y or x the
        // faces R-1 .. N-R-1 of the own planes; the other axes' interior nodes
        const double* W1f = W1d + N;
        const int na = fax == 0 ? S + (r0 == 0 ? 1 : 0) : N - 2 * R + 1;
        const int f0a = fax == 0 ? r0 + R - (r0 == 0 ? 1 : 0) : R - 1;
        const int nb_ = fax == 0 ? nn : S * Ni;      // (y, x) or (z, other)
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
      __syncthreads();
      l2_discard(mi64, res3d_arena_doubles(a.nmax) * sizeof(double), tid, nt);
      __syncthreads();
    }
    // Addresses of the planes beyond this slab (in the neighbouring CTAs' shared
    // memory; the same layout everywhere) for vA (first half) and vB (second half).
    // Entries cover every plane a tile window touches: zl = -r .. ceil(Sa/TZ) TZ + r - 1.
    unsigned* rtab = reinterpret_cast<unsigned*>(pk + 1);
    const int ntab = (Sa + TZ - 1) / TZ * TZ + 2 * R;
    static_assert((kResMaxPack - 1) * sizeof(PackBox) >= 2 * (SAC + TZ + 2 * R) * sizeof(unsigned),
                  "the plane address table must fit the spare pack-table entries");
    if (tid < 2 * ntab) {
      const int which = tid / ntab, zl = tid - which * ntab - R, zg = r0 + zl;
      unsigned e = kRes3Ring;
      if (zg >= 0 && zg < Ni && (zl < 0 || zl >= S)) {
        const int q = res3_owner(zg, Ni, cs);
        e = cluster_addr((which ? vB : vA) + (zg - res3_r0(q, Ni, cs)) * d.PV, (unsigned)q);
      }
      rtab[tid] = e;
    }
    __syncthreads();
    // The neighbouring CTAs read this CTA's planes from stage 1 on (after their wait).
    if (cs > 1) cluster_arrive();

    // ---- This thread's tile: planes z0 .. z0+TZ-1 of the slab, row y, columns jj0, jj0+1.
    const int LD = d.LD, LDI = d.LDI, LDY = d.LDY, PV = d.PV, PI = d.PI, PY = d.PY, PFY = d.PFY;
    const int cstrV = d.Sc * PV, cstrI = d.Sc * PI;
    const int nfz = S + (R == 3 ? 3 : 1);
    const int t = tid;
    const int pg = t / (Ni * d.CPp), rem = t - pg * Ni * d.CPp;
    const int y = rem / d.CPp, jj0 = 2 * (rem - y * d.CPp);
    const int z0 = pg * TZ;
    const bool active = t < res3_tiles(S, Ni, d.CPp, TZ) && jj0 < Ni;
    const int j0 = R + jj0;
    const bool col2 = jj0 + 1 < Ni;
    const int rowoff = (y + R) * LD + j0 + 1;         // the tile's row and column in a plane of vA/vB
    const int io = y * LDI + jj0;                      // in a plane of the interior arrays
    const float* miS = fsm + base + of.mi;
    const float* hiS = fsm + base + of.hi;
    const float* hwS = fsm + base + of.hw;
    const float* fxS = fsm + base + of.fx + y * LDY + jj0;
    const float* fyS = fsm + base + of.fy + y * LDI + jj0;
    const float* fzS = fsm + base + of.fz + io;
    const float dtf = (float)bd.dt;
    const float csf = (float)(R == 3 ? 1.0 / ((24.0 * bd.dx) * (24.0 * bd.dx)) : 1.0 / (bd.dx * bd.dx));
    const float2 cs2 = f2(csf, csf);
    const float2 dt2 = f2(dtf, dtf), hdt2 = f2(0.5f * dtf, 0.5f * dtf);
    const float2 half2 = f2(0.5f, 0.5f);
    __nv_bfloat162 eB[3][TZ], vlo[3][TZ];
#pragma unroll
    for (int k = 0; k < TZ; ++k)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        vlo[c][k] = __float2bfloat162_rn(0.f);
        eB[c][k] = __float2bfloat162_rn(0.f);
      }

    for (int n = 0; n < a.msteps; ++n) {
      const float om = a.om32[n + 1];
      // Stage 1: k1 = f(m_init + v, H(m_init) + H(v)); vB = v + dt k1. The y and x
      // directions read only this CTA's planes; the z direction waits for the cluster.
      float2 Hs[3][TZ];
      if (active) {
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int k = 0; k < TZ; ++k) {
            const int zl = min(z0 + k, S - 1);
            const float* P = vA + c * cstrV + zl * PV + rowoff;
            Hs[c][k] = add2(ypass<R>(P, LD, fyS + zl * PFY, LDI), xpass<R>(P, fxS + zl * PY));
          }
      }
      if (cs > 1) cluster_wait();
      if (active) {
#pragma unroll
        for (int c = 0; c < 3; ++c)
          zpass<R, TZ>(vA + c * cstrV, c * cstrV, PV, rowoff, z0, S, rtab, fzS, nfz, PI, Hs[c]);
#pragma unroll
        for (int k = 0; k < TZ; ++k) {
          const int zl = z0 + k;
          if (zl >= S) continue;
          const int ro = zl * PI + io;
          const int vo = zl * PV + rowoff;
          float2 v[3], m[3], H[3], f[3];
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            v[c] = lds2(vA + c * cstrV + vo);
            m[c] = add2(lds2(miS + c * cstrI + ro), v[c]);
            H[c] = fma2(Hs[c][k], cs2, lds2(hiS + c * cstrI + ro));
          }
          ll_rhs2(m, H, alpha2, f);
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            float2 vb = fma2(dt2, f[c], v[c]);
            eB[c][k] = __float22bfloat162_rn(fma2(hdt2, f[c], mul2(half2, sub2(v[c], vb))));
            if (!col2) vb.y = 0.f;
            *reinterpret_cast<float2*>(vB + c * cstrV + vo) = vb;
          }
        }
      }
      __syncthreads();
      if (cs > 1) cluster_arrive();
      // Stage 2: k2 = f(m_init + vB); v += dt/2 (k1 + k2) + projection, compensated.
      float2 part2[3] = {f2(0.f, 0.f), f2(0.f, 0.f), f2(0.f, 0.f)};
      if (active) {
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int k = 0; k < TZ; ++k) {
            const int zl = min(z0 + k, S - 1);
            const float* P = vB + c * cstrV + zl * PV + rowoff;
            Hs[c][k] = add2(ypass<R>(P, LD, fyS + zl * PFY, LDI), xpass<R>(P, fxS + zl * PY));
          }
      }
      if (cs > 1) cluster_wait();
      if (active) {
#pragma unroll
        for (int c = 0; c < 3; ++c)
          zpass<R, TZ>(vB + c * cstrV, c * cstrV, PV, rowoff, z0, S, rtab + ntab, fzS, nfz, PI, Hs[c]);
#pragma unroll
        for (int k = 0; k < TZ; ++k) {
          const int zl = z0 + k;
          if (zl >= S) continue;
          const int ro = zl * PI + io;
          const int vo = zl * PV + rowoff;
          float2 mi[3], m[3], H[3], k2[3], vh[3], dd[3], vt[3], vbo[3];
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            mi[c] = lds2(miS + c * cstrI + ro);
            vbo[c] = lds2(vB + c * cstrV + vo);
            m[c] = add2(mi[c], vbo[c]);
            H[c] = fma2(Hs[c][k], cs2, lds2(hiS + c * cstrI + ro));
          }
          ll_rhs2(m, H, alpha2, k2);
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            vh[c] = lds2(vA + c * cstrV + vo);
            dd[c] = fma2(hdt2, k2[c], fma2(half2, sub2(vbo[c], vh[c]), __bfloat1622float2(eB[c][k])));
            vt[c] = add2(vh[c], dd[c]);
          }
          const float2 hw = lds2(hwS + ro);
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
            const float2 inc = add2(fma2(cf, add2(mi[c], vt[c]), dd[c]), __bfloat1622float2(vlo[c][k]));
            float2 nh = add2(vh[c], inc);
            vlo[c][k] = __float22bfloat162_rn(sub2(inc, sub2(nh, vh[c])));
            if (!col2) nh.y = 0.f;
            *reinterpret_cast<float2*>(vA + c * cstrV + vo) = nh;
            part2[c] = fma2(hw, sub2(nh, vh[c]), part2[c]);
          }
        }
      }
      if (om != 0.f) {
        float part[3] = {part2[0].x + part2[0].y, part2[1].x + part2[1].y, part2[2].x + part2[2].y};
        warp_kahan_add(kah, lane, om, part);
      }
      __syncthreads();
      if (cs > 1) cluster_arrive();
    }
    if (cs > 1) cluster_wait();   // pairs the last arrive

    // ---- H_avg: s0 plus the warps' Kahan sums; the slabs are added in rank order on rank 0.
    __syncthreads();
    if (tid == 0) {
      double acc[3] = {pk[0].s0[0], pk[0].s0[1], pk[0].s0[2]};
      for (int w = 0; w < kResThreads / 32; ++w)
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

int res3d_variants(const ResVariant** v);

}  // namespace hmm

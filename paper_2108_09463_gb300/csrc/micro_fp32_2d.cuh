// Batched FP32 micro kernel for 2D boxes held on chip: one box per CTA, several
// small boxes per CTA, or one large box split by rows over a thread-block cluster.
//
// Same mathematics and perturbation form as micro_fp32.cu (see there): v = m -
// m_init stepped by HeunP (Section 3.1) under H(m) = H(m_init) + H(v), the
// Dirichlet ring v = 0 (Section 4.2), the average of eq. upscaling evaluated as
// (sum_n w_n) sum_xi W H(m_init) + sum_n w_n sum_xi H(W)(xi) v^n(xi), by the
// symmetry of the discrete operator on fields that vanish on the ring.
//
// Because v^0 = 0, the time sum is taken over the increments of the stored state:
// sum_n w_n S(v^n) = sum_n Omega_{n+1} S(v^{n+1} - v^n), S(u) = sum_xi H(W) u and
// Omega_j = sum_{n >= j} w_n. The kernel K0^{p,q} makes the w_n large and of both
// signs (sum |w_n| is about 24 for p = 3, q = 7), so FP32 rounding in S(v^n) would
// be amplified; the increments are small, and so are the rounding errors of
// S(v^{n+1} - v^n).
//
// Work items. The host sorts the boxes by size and cuts the list into items: a
// pack of up to kResMaxPack boxes that fit one CTA together, or a single box that
// a cluster of cs CTAs shares. Items of one cluster size form one persistent
// launch; CTAs (clusters) pull items from an atomic counter.
//
// Layout of one box (or of one CTA's slab of S interior rows of a box) in shared
// memory, FP32: v^n (vA) and the stage state v^n + dt k1 (vB) on the slab's rows
// plus r halo rows on each side (ring rows are zero, halo rows inside the box are
// written by the neighbouring CTAs of the cluster through distributed shared
// memory after each stage); m_init, H(m_init), H(W) and the face coefficients of
// both axes on the slab's interior rows. Each thread owns a tile of TR rows x 2
// adjacent columns of one box; tiles are numbered row-major within the box and
// each box's tiles start at a warp boundary, so a warp never mixes boxes. The two
// columns are processed together with packed FP32x2 instructions. Per-node
// registers, both in bf16 because each only carries a rounding error forward: the
// rounding error e_B of the stored stage state v_B = fl(v + dt k1) (stage 2
// recovers dt k1 = (v_B - v) + e_B exactly, v_B - v being exact by Sterbenz's
// lemma) and the carried rounding error of v itself (v_lo). The weighted sum of
// H(W) (v^{n+1} - v^n) is reduced per warp and accumulated (Kahan, with the exact
// rounding error of each product by Omega) in shared memory. The FP64 set-up
// (m_init, a^eps, H(m_init), H(W)) goes through the CTA's global arena once per
// box and covers only the rows the CTA needs.
#pragma once
#include <cooperative_groups.h>
#include <cuda_bf16.h>

#include <algorithm>

#include "micro_common.cuh"
#include "stencil.cuh"

namespace hmm {

namespace cg = cooperative_groups;

constexpr int kResTR = 4;            // rows per thread tile
constexpr int kResThreads = 512;     // threads per CTA (16 warps, 128 registers each)
constexpr int kResMaxPack = 8;       // boxes per work item
constexpr int kResMaxCluster = 8;    // CTAs per cluster (portable limit)

// Thread tiles of a box (TR rows x 2 columns) are numbered row-major, CPp tiles
// per row group: the column pairs (Ni + 1)/2 padded to 16 (two row groups per warp,
// one per half-warp), to 32 (one per warp) or to a multiple of 4. In the last case
// row groups share half-warps, and every row stride is chosen congruent to CPp/2
// mod 8 floats: then TR * stride = 2 CPp mod 32 and tile t reads its float2 at bank
// 2t + const mod 32, so the 16 lanes of a half-warp (one 64-bit wavefront) never
// share a bank.
__host__ __device__ inline int res_cp_pad(int Ni) {
  const int CP = (Ni + 1) / 2;
  if (CP <= 16) return 16;
  if (CP > 28 && CP <= 32) return 32;
  return (CP + 3) & ~3;
}

// The smallest even stride >= minimum that keeps the tiles' accesses conflict-free.
__host__ __device__ inline int res_stride(int minimum, int CPp) {
  if (CPp == 16 || CPp == 32) return (minimum + 1) & ~1;
  const int r = (CPp / 2) & 7;
  int s = minimum;
  while ((s & 7) != r) ++s;
  return s;
}

// Dimensions of one slab: interior rows [r0, r0 + S) of a box of N nodes per axis.
struct ResDims {
  int N, Ni, S;
  int rows;   // rows of vA/vB: S + 2r (halo or ring rows on both sides)
  int LD;     // row stride of vA/vB (column j at offset j + 1; columns up to N + 2 readable)
  int LDI;    // row stride of the interior arrays (>= Ni)
  int nf;     // face rows of the x-face array, S + 3 (order 4) or S + 1 (order 2)
  int LDY;    // row stride of the y-face array (>= Ni + 4 or Ni + 2)
  int CPp;    // tiles per row group
  int rk4;    // 1: the RK4P instance (a third state array and the stage accumulator)
  int TR;     // rows per thread tile of the instance
};

__host__ __device__ inline ResDims res_dims(int N, int R, int S) {
  ResDims d;
  d.N = N;
  d.Ni = N - 2 * R;
  d.S = S;
  d.rows = S + 2 * R;
  d.CPp = res_cp_pad(d.Ni);
  d.LD = res_stride(N + 4, d.CPp);
  d.LDI = res_stride(d.Ni, d.CPp);
  d.nf = S + (R == 3 ? 3 : 1);
  d.LDY = res_stride(d.Ni + (R == 3 ? 4 : 2), d.CPp);
  d.rk4 = 0;
  d.TR = kResTR;
  return d;
}

// Strides and allocation of a slab: from the box itself (NC = 0), or from a fixed
// canvas of NC nodes per axis and SAC slab rows that holds any box with N <= NC
// (the strides are then compile-time constants, which keeps the address arithmetic
// of the time loop out of the registers).
template <int R, int NC, int SAC, int ST = 0, int TRr = kResTR>
__host__ __device__ inline ResDims res_geom(int N, int Sa) {
  ResDims d = NC > 0 ? res_dims(NC, R, SAC) : res_dims(N, R, Sa);
  d.rk4 = ST;
  d.TR = TRr;
  return d;
}

// Float offsets of the arrays of one slab, relative to the slab's base. The RK4P
// instance adds a second stage-state array vC and, in thread order, the per-node
// accumulator of k1 + 2 k2 + 2 k3 (3 components x TR rows x 2 columns per tile).
//
// The stencil reads the state arrays and the face coefficients without clamping its
// rows: the tiles of a ragged last tile row read up to TR - 1 rows past the slab, whose
// values only reach the rows it discards. So those arrays come first (vA, vB, vC, afx,
// afy), each followed by arrays that absorb the overrun, and the slab is padded where
// the rest of it is shorter than the overrun of the array before.
struct ResOffsets {
  int vA, vB, mi, hi, hw, afx, afy, vC, acc, total;
};

__host__ __device__ inline ResOffsets res_offsets(const ResDims& d) {
  ResOffsets o;
  int x = 0, need = 0;
  const int over = ((d.S + d.TR - 1) / d.TR) * d.TR - d.S + 1;   // rows past the end, + column overshoot
  auto place = [&](int* off, int size, int stride) {
    *off = x;
    x += size;
    if (stride > 0) need = need > x + over * stride + 8 ? need : x + over * stride + 8;
  };
  o.vC = 0;
  o.acc = 0;
  place(&o.vA, 3 * d.rows * d.LD, d.LD);
  place(&o.vB, 3 * d.rows * d.LD, d.LD);
  if (d.rk4) place(&o.vC, 3 * d.rows * d.LD, d.LD);
  place(&o.afx, d.nf * d.LDI, d.LDI);
  place(&o.afy, d.S * d.LDY, d.LDY);
  place(&o.mi, 3 * d.S * d.LDI, 0);
  place(&o.hi, 3 * d.S * d.LDI, 0);
  place(&o.hw, d.S * d.LDI, 0);
  if (d.rk4) place(&o.acc, 3 * d.TR * 2 * (((d.S + d.TR - 1) / d.TR) * d.CPp), 0);
  x = x > need ? x : need;
  o.total = (x + 3) & ~3;   // 16-byte aligned bases
  return o;
}

// One box of the current work item (shared memory, written by thread 0).
struct PackBox {
  double s0[3];   // sum_n w_n sum_xi W H(m_init) over this CTA's rows (FP64)
  int box;        // index into the sorted box table
  int r0, S, Sa;  // first interior row, rows of this CTA, rows allocated (equal on all ranks)
  int base;       // float offset of the slab's arrays
  int warp0, nwarps;
  int pad;
};

// CTA-wide header at the start of the dynamic shared memory (floats).
constexpr int kResRedDoubles = 96;
constexpr int kResCsumDoubles = 4 * kResMaxCluster;
constexpr int kResHeaderFloats =
    ((2 * (kResRedDoubles + kResCsumDoubles) + (int)(kResMaxPack * sizeof(PackBox) / 4) + 6 * (kResThreads / 32)) + 3) & ~3;

// Tiles (threads) of a slab of S rows with CPp tiles per row group.
__host__ __device__ inline int res_tiles(int S, int CPp, int TR = kResTR) { return ((S + TR - 1) / TR) * CPp; }

// Whether a box of Ni interior nodes per row, laid out CPp tiles per row group, can
// take its right-hand y faces from the next two lanes: the row group fills a half or
// a whole warp, and the two lanes after its last interior tile are in it.
__host__ __device__ inline bool res_yshfl_ok(int Ni, int CPp) {
  return (CPp == 16 || CPp == 32) && (Ni + 1) / 2 <= CPp - 2;
}

// Set-up tables (FP64) overlay the slab's vB region while the slab is being set up.
__host__ __device__ inline bool res_setup_fits(const ResDims& d, int N, int interp_k, int n_terms) {
  return setup_smem_doubles(2, N, interp_k, n_terms) * 2 <= (size_t)3 * d.rows * d.LD;
}

// per CTA: m_init (3), face coefficients (2), x- and y-face fluxes of m_init and W (4 + 4)
__host__ __device__ inline size_t res2d_arena_doubles(int nmax) { return (size_t)13 * nmax * nmax; }

// Drops the whole 128-byte lines of [p, p + bytes) from L2 without writing them
// back (discard.global.L2): the CTA's set-up arena is dead once the box's
// shared-memory tables are built, and the next box's set-up rewrites it. Call
// between two barriers: the first ends every read of the range, the second
// orders the discards before any later write to it.
__device__ __forceinline__ void l2_discard(const void* p, size_t bytes, int tid, int nt) {
  const unsigned long long b = ((unsigned long long)p + 127ull) & ~127ull;
  const unsigned long long e = ((unsigned long long)p + bytes) & ~127ull;
  for (unsigned long long q = b + 128ull * (unsigned long long)tid; q < e; q += 128ull * (unsigned long long)nt)
    asm volatile("discard.global.L2 [%0], 128;" ::"l"(q) : "memory");
}


// One persistent launch: its work items, its queue counter and its cluster size.
struct ResLaunch {
  const int2* items;
  int n_items;
  int* queue;
  int cs;
  int aux;   // z-column 3D kernel: the row stride of its planes (0 otherwise)
};

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, f2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 shift2(float2 a, float2 b) { return f2(a.y, b.x); }  // (a.y, b.x)
__device__ __forceinline__ float2 lds2(const float* p) { return *reinterpret_cast<const float2*>(p); }

// Stencil of one component at the thread's TR x 2 tile. V: the component plane of
// vA or vB (row stride LD, column j at offset j + 1). Result H (without the
// 1/dx^2 or 1/(24 dx)^2 factor) per row.
//
// yshfl (warp-uniform): every lane of the warp runs this, a row group of tiles lies in
// consecutive lanes with at least two lanes of slack after its last interior tile
// (res_yshfl_ok), and each lane computes only the y-face fluxes on the left of its two
// nodes; the faces on the right are the next lanes' left faces, taken by shuffles.
// Otherwise each lane computes all the y faces it needs (2.5 per node).
template <int R, int TR>
__device__ __forceinline__ void tile_stencil(const float* __restrict__ V, int LD, int i0, int j0,
                                             const float* __restrict__ afx, int LDI, int jj0,
                                             const float* __restrict__ afy, int LDY, int ii0, bool yshfl,
                                             float2* H) {
  // x direction (rows): a rolling window over the rows and over the face fluxes.
  // Each node combines its four fluxes as (F_t - F_{t+3}) + 27 (F_{t+2} - F_{t+1}):
  // the two differences of neighbouring fluxes cancel with little rounding.
  // (rows are not clamped: the slab layout absorbs the ragged tile row's overrun)
  auto ld = [&](int k) { return lds2(V + (i0 - R + k) * LD + j0 + 1); };
  auto axf = [&](int f) { return lds2(afx + (ii0 + f) * LDI + jj0); };
  const float2 k27 = f2(27.f, 27.f);
  float2 Cc[TR];   // centre values of the tile rows (reused by the y direction)
  if (R == 3) {
    float2 p0 = ld(0), p1 = ld(1), p2 = ld(2);
    float2 Fa = f2(0.f, 0.f), Fb = Fa, Fc = Fa;   // F_{f-3}, F_{f-2}, F_{f-1}
#pragma unroll
    for (int f = 0; f < TR + 3; ++f) {
      const float2 p3 = ld(f + 3);
      if (f < TR) Cc[f] = p3;
      const float2 F = mul2(axf(f), fma2(k27, sub2(p2, p1), sub2(p0, p3)));
      if (f >= 3) H[f - 3] = fma2(k27, sub2(Fc, Fb), sub2(Fa, F));
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
    for (int f = 0; f < TR + 1; ++f) {
      const float2 p1 = ld(f + 1);
      if (f < TR) Cc[f] = p1;
      const float2 F = mul2(axf(f), sub2(p1, p0));
      if (f >= 1) H[f - 1] = sub2(F, Fa);   // H[t] = F_{t+1} - F_t
      Fa = F;
      p0 = p1;
    }
  }
  // y direction (columns), faces between columns, row by row
  if (yshfl) {
    constexpr unsigned kAll = 0xffffffffu;
#pragma unroll
    for (int t = 0; t < TR; ++t) {
      const float* row = V + (i0 + t) * LD + j0 + 1;
      const float2 C = Cc[t];
      const float2 a01 = lds2(afy + (ii0 + t) * LDY + jj0);
      if (R == 3) {
        // this lane's faces j0-2, j0-1; faces j0, j0+1 from lane + 1 and j0+2 from lane + 2
        const float2 L1 = lds2(row - 2);
        const float l2 = row[-3];
        const float2 F01 = mul2(a01, fma2(k27, sub2(shift2(L1, C), L1), sub2(f2(l2, L1.x), C)));
        const float2 F23 = f2(__shfl_down_sync(kAll, F01.x, 1), __shfl_down_sync(kAll, F01.y, 1));
        const float F4 = __shfl_down_sync(kAll, F01.x, 2);
        const float2 hy = fma2(k27, sub2(F23, shift2(F01, F23)), sub2(F01, f2(F23.y, F4)));
        H[t] = add2(H[t], hy);
      } else {
        // this lane's faces j0-1|j0 and j0|j0+1; face j0+1|j0+2 from lane + 1
        const float l1 = row[-1];
        const float2 F01 = mul2(a01, sub2(C, f2(l1, C.x)));
        const float F2 = __shfl_down_sync(kAll, F01.x, 1);
        H[t] = add2(H[t], sub2(f2(F01.y, F2), F01));
      }
    }
    return;
  }
#pragma unroll
  for (int t = 0; t < TR; ++t) {
    const float* row = V + (i0 + t) * LD + j0 + 1;
    const float2 C = Cc[t];
    const float2 L1 = lds2(row - 2);
    const float2 R1 = lds2(row + 2);
    const float* ay = afy + (ii0 + t) * LDY + jj0;
    if (R == 3) {
      const float2 L2 = lds2(row - 4);
      const float r2x = row[4];
      const float2 a01 = lds2(ay), a23 = lds2(ay + 2);
      const float a4 = ay[4];
      // faces b = j0-2, j0-1 | j0, j0+1 | j0+2
      const float2 g01 = fma2(k27, sub2(shift2(L1, C), L1), sub2(shift2(L2, L1), C));
      const float2 g23 = fma2(k27, sub2(shift2(C, R1), C), sub2(shift2(L1, C), R1));
      const float g4 = (C.y - r2x) + 27.f * (R1.y - R1.x);
      const float2 F01 = mul2(a01, g01), F23 = mul2(a23, g23);
      const float F4 = a4 * g4;
      const float2 hy = fma2(k27, sub2(F23, shift2(F01, F23)), sub2(F01, f2(F23.y, F4)));
      H[t] = add2(H[t], hy);
    } else {
      const float2 a01 = lds2(ay);
      const float a2 = ay[2];
      const float2 g01 = sub2(C, shift2(L1, C));
      const float g2 = R1.x - C.y;
      const float2 F01 = mul2(a01, g01);
      const float F2 = a2 * g2;
      H[t] = add2(H[t], sub2(f2(F01.y, F2), F01));
    }
  }
}

// f = -m x H - alpha m x (m x H) for two nodes at once.
__device__ __forceinline__ void ll_rhs2(const float2* m, const float2* H, float2 alpha, float2* f) {
  // f = q + alpha m x q with q = H x m = -m x H (so m x q = -m x (m x H)); the cross
  // products as one product and one fma each, the sign in the negated m.
  const float2 n0 = f2(-m[0].x, -m[0].y), n1 = f2(-m[1].x, -m[1].y), n2 = f2(-m[2].x, -m[2].y);
  const float2 q0 = fma2(H[1], m[2], mul2(H[2], n1));
  const float2 q1 = fma2(H[2], m[0], mul2(H[0], n2));
  const float2 q2 = fma2(H[0], m[1], mul2(H[1], n0));
  const float2 d0 = fma2(m[1], q2, mul2(n2, q1));
  const float2 d1 = fma2(m[2], q0, mul2(n0, q2));
  const float2 d2 = fma2(m[0], q1, mul2(n1, q0));
  f[0] = fma2(alpha, d0, q0);
  f[1] = fma2(alpha, d1, q1);
  f[2] = fma2(alpha, d2, q2);
}

// Add w * (warp sum of part[0..2]) to the warp's Kahan accumulators in shared
// memory (sum kah[c], compensation kah[3 + c]; the total is kah[c] - kah[3 + c]).
// The product's rounding error e = w x - fl(w x) is exact (one fma) and goes into
// the compensation. Explicit _rn intrinsics keep the compiler from contracting.
__device__ __forceinline__ void warp_kahan_add(float* kah, int lane, float w, float* part) {
#pragma unroll
  for (int c = 0; c < 3; ++c) part[c] = warp_sum(part[c]);
  if (lane == 0) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float p = __fmul_rn(w, part[c]);
      const float e = __fmaf_rn(w, part[c], -p);
      const float s = kah[c], cmp = kah[3 + c];
      const float y = __fsub_rn(p, cmp);
      const float t = __fadd_rn(s, y);
      kah[3 + c] = __fsub_rn(__fsub_rn(__fsub_rn(t, s), y), e);
      kah[c] = t;
    }
  }
}
// Copy the first and last r rows of this CTA's slab of vA (which = 0), vB
// (which = 1) or vC (which = 2, RK4P), all three components, into the halo rows of the neighbouring
// slabs of the cluster (distributed shared memory). Item geometry from pk[0].
template <int R, int NC, int SAC, int ST = 0, int TR = kResTR>
__device__ __forceinline__ void push_halo(const MicroArgs& a, float* fsm, const PackBox* pk, int which, unsigned rank,
                                          int cs) {
  cg::cluster_group cl = cg::this_cluster();
  const PackBox& p = pk[0];
  const ResDims d = res_geom<R, NC, SAC, ST, TR>(a.boxes[p.box].N, p.Sa);
  const ResOffsets of = res_offsets(d);
  float* V = fsm + p.base + (which == 0 ? of.vA : (which == 1 ? of.vB : of.vC));
  const int cstr = d.rows * d.LD, w2 = d.LD / 2, per = 3 * R * w2, S = p.S, Sa = p.Sa;
  for (int e = threadIdx.x; e < 2 * per; e += blockDim.x) {
    const int side = e / per;   // 0: to rank - 1 (its bottom halo), 1: to rank + 1 (its top halo)
    if (side == 0 ? rank == 0 : (int)rank == cs - 1) continue;
    int r = e - side * per;
    const int c = r / (R * w2);
    r -= c * R * w2;
    const int k = r / w2, x = r - k * w2;
    const int lr = side == 0 ? R + k : S + k;      // slab rows 0..r-1 or S-r..S-1 (local rows)
    const int dr = side == 0 ? lr + Sa : lr - Sa;  // the same box rows in the neighbour's slab
    const float2 val = *reinterpret_cast<const float2*>(V + c * cstr + lr * d.LD + 2 * x);
    float* dst = cl.map_shared_rank(V + c * cstr + dr * d.LD + 2 * x, side == 0 ? rank - 1 : rank + 1);
    *reinterpret_cast<float2*>(dst) = val;
  }
}

template <int R, int TR, int NC, int SAC, int ST = 0>
__global__ void __launch_bounds__(kResThreads)
micro_fp32_2d_kernel(MicroArgs a, ResLaunch L) {
  constexpr int D = 2;
  extern __shared__ __align__(16) float fsm[];
  __shared__ int s_item;
  double* red = reinterpret_cast<double*>(fsm);
  double* csum = red + kResRedDoubles;                              // [rank][4] slab partial sums (rank 0)
  PackBox* pk = reinterpret_cast<PackBox*>(csum + kResCsumDoubles);
  float* kahA = reinterpret_cast<float*>(pk + kResMaxPack);          // [warp][6] Kahan sums
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int cs = L.cs;
  const unsigned rank = cs > 1 ? cg::this_cluster().block_rank() : 0u;
  float* kah = kahA + 6 * warp;
  const size_t cap = (size_t)a.nmax * a.nmax;
  double* mi64 = reinterpret_cast<double*>(a.arena + (size_t)blockIdx.x * a.slot_bytes);
  double* af64 = mi64 + 3 * cap;
  const float am = (float)a.alpha_micro;
  const float2 alpha2 = f2(am, am);
  double wsum = 0.0;
  for (int n = 0; n <= a.msteps; ++n) wsum += a.w64[n];

  for (;;) {
    // ---- Next work item (the cluster's rank 0 takes it and tells the others).
    if (cs == 1) {
      __syncthreads();
      if (tid == 0) s_item = atomicAdd(L.queue, 1);
      __syncthreads();
    } else {
      cg::cluster_group cl = cg::this_cluster();
      cl.sync();   // every CTA is done with the previous item (its shared memory is free)
      if (rank == 0 && tid == 0) {
        const int it = atomicAdd(L.queue, 1);
        for (int q = 0; q < cs; ++q) *cl.map_shared_rank(&s_item, q) = it;
      }
      cl.sync();
    }
    const int item = s_item;
    if (item >= L.n_items) break;
    const int2 itd = L.items[item];   // (first box, box count)
    const int npack = itd.y;
    if (tid == 0) {
      int o = kResHeaderFloats, w0 = 0;
      for (int q = 0; q < npack; ++q) {
        const int Ni = a.boxes[itd.x + q].N - 2 * R;
        const int Sa = cs == 1 ? Ni : (Ni + cs - 1) / cs;
        const int r0 = (int)rank * Sa;
        const int S = max(0, min(Sa, Ni - r0));
        PackBox& p = pk[q];
        p.box = itd.x + q;
        p.r0 = r0;
        p.S = S;
        p.Sa = Sa;
        p.base = o;
        p.warp0 = w0;
        const ResDims dq = res_geom<R, NC, SAC, ST, TR>(Ni + 2 * R, Sa);
        p.nwarps = (res_tiles(S, dq.CPp, TR) + 31) / 32;
        w0 += p.nwarps;
        o += res_offsets(dq).total;
      }
    }
    if (tid < 6 * (kResThreads / 32)) kahA[tid] = 0.f;
    __syncthreads();

    // ---- Set-up of each box of the item (all threads, one box after the other).
    for (int q = 0; q < npack; ++q) {
      const PackBox p = pk[q];
      const BoxDesc bd = a.boxes[p.box];
      const int N = bd.N;
      const ResDims d = res_geom<R, NC, SAC, ST, TR>(N, p.Sa);
      const ResOffsets of = res_offsets(d);
      float* base = fsm + p.base;
      float* vA = base + of.vA;
      float* vB = base + of.vB;
      SetupSmem smr = carve_setup(reinterpret_cast<double*>(vB), D, N, a.interp_k, a.n_terms);
      smr.red = red;
      box_setup_tables<D>(a, bd, smr);
      const Strides<D> st(N);
      // FP64 m_init (Section 4.1) and a^eps at the faces, box rows [r0, r0 + S + 2r).
      const int rlo = p.r0, rhi = min(N, p.r0 + p.S + 2 * R);
      int bad = 0;
      for (int idx = rlo * N + tid; idx < rhi * N; idx += nt) {
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
      __syncthreads();   // the set-up tables (overlaying vB) are no longer needed
      for (int e = tid; e < of.total; e += nt) base[e] = 0.f;   // padding included
      __syncthreads();
      const int Ni = N - 2 * R, S = p.S, r0 = p.r0;
      const int f0 = R == 3 ? R - 2 : R - 1;     // first face row/column the stencil uses
      const int nfy = Ni + (R == 3 ? 3 : 1);     // y-face columns
      float* miS = base + of.mi;
      float* hiS = base + of.hi;
      float* hwS = base + of.hw;
      float* afx = base + of.afx;
      float* afy = base + of.afy;
      for (int e = tid; e < 3 * S * Ni; e += nt) {
        const int c = e / (S * Ni), r = e - c * S * Ni;
        const int ii = r / Ni, jj = r - ii * Ni;
        miS[(c * d.S + ii) * d.LDI + jj] = (float)mi64[c * cap + (r0 + ii + R) * N + (jj + R)];
      }
      for (int e = tid; e < (S + (R == 3 ? 3 : 1)) * Ni; e += nt) {
        const int f = e / Ni, jj = e - f * Ni;
        afx[f * d.LDI + jj] = (float)af64[(r0 + f + f0) * N + (jj + R)];   // between rows r0+f+f0 and +1
      }
      for (int e = tid; e < S * nfy; e += nt) {
        const int ii = e / nfy, g = e - ii * nfy;
        afy[ii * d.LDY + g] = (float)af64[cap + (r0 + ii + R) * N + (g + f0)];   // between columns g+f0, +1
      }
      const double cs64 = R == 3 ? 1.0 / ((24.0 * bd.dx) * (24.0 * bd.dx)) : 1.0 / (bd.dx * bd.dx);
      const double* W1d = a.W64 + bd.wofs;
      // H(m_init) and H(W) in FP64, face fluxes first (each face once): components 0-2
      // of m_init and, as a fourth, the weight W = W(x) W(y), whose face differences
      // factor into 1D differences of the weight table. x-faces (between rows f and
      // f+1, f in [xf0, xf1)) at the interior columns; y-faces (between columns g and
      // g+1, g in [yg0, yg1)) at the slab's rows.
      double* flx = af64 + 2 * cap;   // [4][cap] x-face fluxes at (f, j)
      double* fly = flx + 4 * cap;    // [4][cap] y-face fluxes at (i, g)
      const int fl = R == 3 ? 2 : 1, fh = R == 3 ? 1 : 0;   // a node uses faces i-fl .. i+fh
      const int xf0 = r0 + R - fl, xf1 = r0 + S + R + fh, nxf = xf1 - xf0;
      const int yg0 = R - fl, yg1 = N - R + fh, nyg = yg1 - yg0;
      auto fdiff = [](const double* u, int o, int st_) {   // the face difference at face o
        return R == 3 ? (u[o - st_] - u[o + 2 * st_]) + 27.0 * (u[o + st_] - u[o]) : u[o + st_] - u[o];
      };
      // Flux model (bd.fax = k): the box averages a_f D_k m over the faces along k
      // instead of H. By summation by parts its state part is sum_xi G(xi) v(xi)
      // with G = -fcomb(WA) / (24 dx) (order 2: / dx), WA_f = W_f a_f the face
      // weight times the coefficient: the fourth flux component then holds WA on
      // the axis k faces (zero on the other axis), and G takes H(W)'s place in the
      // time loop's average. W_f: face weights along k (after the node weights in
      // the table) times node weights along the other axis.
      const int fax = bd.fax;
      const double* W1f = W1d + N;
      for (int e = tid; e < nxf * Ni; e += nt) {
        const int f = xf0 + e / Ni, j = R + e % Ni;
        const int o = f * N + j;
        const double af = af64[o];
#pragma unroll
        for (int c = 0; c < 3; ++c) flx[c * cap + o] = af * fdiff(mi64 + c * cap, o, N);
        flx[3 * cap + o] = fax < 0 ? af * W1d[j] * fdiff(W1d, f, 1) : (fax == 0 ? af * W1f[f] * W1d[j] : 0.0);
      }
      for (int e = tid; e < S * nyg; e += nt) {
        const int i = r0 + R + e / nyg, g = yg0 + e % nyg;
        const int o = i * N + g;
        const double af = af64[cap + o];
#pragma unroll
        for (int c = 0; c < 3; ++c) fly[c * cap + o] = af * fdiff(mi64 + c * cap, o, 1);
        fly[3 * cap + o] = fax < 0 ? af * W1d[i] * fdiff(W1d, g, 1) : (fax == 1 ? af * W1d[i] * W1f[g] : 0.0);
      }
      __syncthreads();
      auto fcomb = [](const double* F, int o, int st_) {   // node combination of the fluxes
        return R == 3 ? (F[o - 2 * st_] - F[o + st_]) + 27.0 * (F[o] - F[o - st_]) : F[o] - F[o - st_];
      };
      double s0 = 0.0, s1 = 0.0, s2 = 0.0;
      const double cf = R == 3 ? 1.0 / (24.0 * bd.dx) : 1.0 / bd.dx;
      for (int e = tid; e < S * Ni; e += nt) {
        const int ii = e / Ni, jj = e - ii * Ni;
        const int idx = (r0 + ii + R) * N + (jj + R);
        double H[4];
#pragma unroll
        for (int c = 0; c < 3; ++c) H[c] = (fcomb(flx + c * cap, idx, N) + fcomb(fly + c * cap, idx, 1)) * cs64;
        const double c3 = fcomb(flx + 3 * cap, idx, N) + fcomb(fly + 3 * cap, idx, 1);
        H[3] = fax < 0 ? c3 * cs64 : -c3 * cf;
        if (fax < 0) {
          const double W = W1d[r0 + ii + R] * W1d[jj + R];
          s0 += W * H[0];
          s1 += W * H[1];
          s2 += W * H[2];
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) hiS[(c * d.S + ii) * d.LDI + jj] = (float)H[c];
        hwS[ii * d.LDI + jj] = (float)H[3];
      }
      if (fax >= 0) {
        // the flux of m_init over the faces along k this CTA owns: along the slab's
        // axis the faces f in [r0 + R, r0 + R + S) (and f = R - 1 in the first slab),
        // along the other axis the faces R-1 .. N-R-1 of the slab's rows
        const int fa = fax == 0 ? r0 + R - (r0 == 0 ? 1 : 0) : R - 1;
        const int fb = fax == 0 ? r0 + R + S : N - R;
        const int nfa = fb - fa, nother = fax == 0 ? Ni : S;
        for (int e = tid; e < nfa * nother; e += nt) {
          const int f = fa + e / nother, u = e % nother;
          const int o = fax == 0 ? f * N + (R + u) : (r0 + R + u) * N + f;
          const double WF = fax == 0 ? W1f[f] * W1d[R + u] : W1d[r0 + R + u] * W1f[f];
          const double* Fl = fax == 0 ? flx : fly;
          s0 += WF * Fl[o] * cf;
          s1 += WF * Fl[cap + o] * cf;
          s2 += WF * Fl[2 * cap + o] * cf;
        }
      }
      block_sum3(s0, s1, s2, red);
      if (tid == 0) {
        pk[q].s0[0] = s0 * wsum;
        pk[q].s0[1] = s1 * wsum;
        pk[q].s0[2] = s2 * wsum;
      }
      __syncthreads();
      l2_discard(mi64, res2d_arena_doubles(a.nmax) * sizeof(double), tid, nt);
      __syncthreads();
    }
    // Neighbouring CTAs write halo rows into this CTA's slabs from stage 1 on: the
    // whole cluster finishes its set-up (which clears those rows) first.
    if (cs > 1) cg::this_cluster().sync();

    // ---- This thread's box and tile: interior rows ii0 .. ii0+TR-1, columns jj0, jj0+1.
    int q = -1;
    for (int b = 0; b < npack; ++b)
      if (warp >= pk[b].warp0 && warp < pk[b].warp0 + pk[b].nwarps) q = b;
    bool active = false, yshfl = false;
    ResDims d = res_geom<R, NC, SAC, ST, TR>(2 * R + 2, 1);
    int r0 = 0, S = 0, Ni = 1, ii0 = 0, jj0 = 0, obase = 0;
    float dtf = 0.f, csf = 0.f;
    if (q >= 0) {
      const PackBox& p = pk[q];
      const BoxDesc& bd = a.boxes[p.box];
      d = res_geom<R, NC, SAC, ST, TR>(bd.N, p.Sa);
      r0 = p.r0;
      S = p.S;
      Ni = bd.N - 2 * R;
      obase = p.base;
      const int t = (warp - p.warp0) * 32 + lane;
      ii0 = (t / d.CPp) * TR;          // row within the slab
      jj0 = 2 * (t % d.CPp);
      active = t < res_tiles(S, d.CPp, TR) && jj0 < Ni;
      yshfl = res_yshfl_ok(Ni, d.CPp);
      // lanes past the needed ones run the stencil on the last needed column and tile row
      if (yshfl) {
        jj0 = min(jj0, 2 * ((Ni + 1) / 2) + (R == 3 ? 2 : 0));
        ii0 = min(ii0, ((S + TR - 1) / TR - 1) * TR);
      }
      dtf = (float)bd.dt;
      csf = (float)(R == 3 ? 1.0 / ((24.0 * bd.dx) * (24.0 * bd.dx)) : 1.0 / (bd.dx * bd.dx));
    }
    const ResOffsets of = res_offsets(d);
    const int LD = d.LD, LDI = d.LDI, LDY = d.LDY, rows = d.rows;
    float* vA = fsm + obase + of.vA;
    float* vB = fsm + obase + of.vB;
    const float* miS = fsm + obase + of.mi;
    const float* hiS = fsm + obase + of.hi;
    const float* hwS = fsm + obase + of.hw;
    const float* afx = fsm + obase + of.afx;
    const float* afy = fsm + obase + of.afy;
    const int cstrV = rows * LD, cstrI = d.S * LDI;
    const int j0 = R + jj0;
    const bool col2 = jj0 + 1 < Ni;   // odd Ni: the tile's second column is ring
    const bool run = yshfl ? q >= 0 : active;   // lanes that run the stencil (whole warps if yshfl)
    const float2 cs2 = f2(csf, csf);
    const float2 dt2 = f2(dtf, dtf), hdt2 = f2(0.5f * dtf, 0.5f * dtf);
    const float2 half2 = f2(0.5f, 0.5f);
    if constexpr (ST == 0) {
      __nv_bfloat162 eB[3][TR], vlo[3][TR];
#pragma unroll
      for (int t = 0; t < TR; ++t)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          vlo[c][t] = __float2bfloat162_rn(0.f);
          eB[c][t] = __float2bfloat162_rn(0.f);
        }

      for (int n = 0; n < a.msteps; ++n) {
        const float om = a.om32[n + 1];
        if (run) {
          // Stage 1: k1 = f(m_init + v, H(m_init) + H(v)); vB = v + dt k1.
          float2 Hs[3][TR];
#pragma unroll
          for (int c = 0; c < 3; ++c)
            tile_stencil<R, TR>(vA + c * cstrV, LD, ii0 + R, j0, afx, LDI, jj0, afy, LDY, ii0, yshfl, Hs[c]);
#pragma unroll
          for (int t = 0; t < TR; ++t) {
            const int ii = ii0 + t;
            if (!active || ii >= S) continue;
            const int ro = ii * LDI + jj0;
            const int vo = (ii + R) * LD + j0 + 1;
            float2 v[3], m[3], H[3], f[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              v[c] = lds2(vA + c * cstrV + vo);
              m[c] = add2(lds2(miS + c * cstrI + ro), v[c]);
              H[c] = fma2(Hs[c][t], cs2, lds2(hiS + c * cstrI + ro));
            }
            ll_rhs2(m, H, alpha2, f);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              float2 vb = fma2(dt2, f[c], v[c]);
              // e_B / 2 = (v + dt k1 - v_B) / 2 (v_B - v is exact): stage 2 adds it to (v_B - v) / 2
              eB[c][t] = __float22bfloat162_rn(fma2(hdt2, f[c], mul2(half2, sub2(v[c], vb))));
              if (!col2) vb.y = 0.f;
              *reinterpret_cast<float2*>(vB + c * cstrV + vo) = vb;
            }
          }
        }
        __syncthreads();
        if (cs > 1) {
          push_halo<R, NC, SAC, ST, TR>(a, fsm, pk, 1, rank, cs);
          cg::this_cluster().sync();
        }
        float2 part2[3] = {f2(0.f, 0.f), f2(0.f, 0.f), f2(0.f, 0.f)};
        if (run) {
          // Stage 2: k2 = f(m_init + vB); v += dt/2 (k1 + k2) + projection, compensated.
          float2 Hs[3][TR];
#pragma unroll
          for (int c = 0; c < 3; ++c)
            tile_stencil<R, TR>(vB + c * cstrV, LD, ii0 + R, j0, afx, LDI, jj0, afy, LDY, ii0, yshfl, Hs[c]);
#pragma unroll
          for (int t = 0; t < TR; ++t) {
            const int ii = ii0 + t;
            if (!active || ii >= S) continue;
            const int ro = ii * LDI + jj0;
            const int vo = (ii + R) * LD + j0 + 1;
            float2 mi[3], m[3], H[3], k2[3], vh[3], dd[3], vt[3], vbo[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              mi[c] = lds2(miS + c * cstrI + ro);
              vbo[c] = lds2(vB + c * cstrV + vo);
              m[c] = add2(mi[c], vbo[c]);
              H[c] = fma2(Hs[c][t], cs2, lds2(hiS + c * cstrI + ro));
            }
            ll_rhs2(m, H, alpha2, k2);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              vh[c] = lds2(vA + c * cstrV + vo);
              // dt/2 (k1 + k2) with dt k1 = (v_B - v) + e_B
              dd[c] = fma2(hdt2, k2[c], fma2(half2, sub2(vbo[c], vh[c]), __bfloat1622float2(eB[c][t])));
              vt[c] = add2(vh[c], dd[c]);
            }
            const float2 hw = lds2(hwS + ro);
            // s = 2 m_init.vt + |vt|^2; c = -s / (sqrt(1+s)(1+sqrt(1+s)))
            float2 sdot = mul2(mi[0], vt[0]);
            sdot = fma2(mi[1], vt[1], sdot);
            sdot = fma2(mi[2], vt[2], sdot);
            float2 sq = mul2(vt[0], vt[0]);
            sq = fma2(vt[1], vt[1], sq);
            sq = fma2(vt[2], vt[2], sq);
            const float2 s = fma2(f2(2.f, 2.f), sdot, sq);
            // (c is a small correction, so the approximate quotient costs nothing measurable)
            const float rr0 = rsqrtf(1.f + s.x), rr1 = rsqrtf(1.f + s.y);
            const float2 cf = f2(__fdividef(-s.x * rr0 * rr0, 1.f + rr0), __fdividef(-s.y * rr1 * rr1, 1.f + rr1));
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              const float2 inc = add2(fma2(cf, add2(mi[c], vt[c]), dd[c]), __bfloat1622float2(vlo[c][t]));
              float2 nh = add2(vh[c], inc);
              vlo[c][t] = __float22bfloat162_rn(sub2(inc, sub2(nh, vh[c])));
              if (!col2) nh.y = 0.f;
              *reinterpret_cast<float2*>(vA + c * cstrV + vo) = nh;
              // H(W) times the exact change of the stored state (zero in a ring column)
              part2[c] = fma2(hw, sub2(nh, vh[c]), part2[c]);
            }
          }
        }
        if (om != 0.f) {
          float part[3] = {part2[0].x + part2[0].y, part2[1].x + part2[1].y, part2[2].x + part2[2].y};
          warp_kahan_add(kah, lane, om, part);
        }
        __syncthreads();
        if (cs > 1) {
          push_halo<R, NC, SAC, ST, TR>(a, fsm, pk, 0, rank, cs);
          cg::this_cluster().sync();
        }
      }
    } else {
      // RK4P (Section 3.1): k1 = f(v), k2 = f(v + dt/2 k1), k3 = f(v + dt/2 k2),
      // k4 = f(v + dt k3), v += dt/6 (k1 + 2 k2 + 2 k3 + k4) and the projection, both
      // written in the perturbation form and compensated as in HeunP (the carried
      // rounding error of v in bf16). The stage states alternate between vB and vC, so
      // that a stage reads one while it writes the other; k1 + 2 k2 + 2 k3 accumulates
      // per node in shared memory in thread order.
      float* vC = fsm + obase + of.vC;
      float2* accS = reinterpret_cast<float2*>(fsm + obase + of.acc);
      const int ntile = res_tiles(S, d.CPp, TR);
      const int tb = q >= 0 ? (warp - pk[q].warp0) * 32 + lane : 0;   // the tile's index in its slab
      const float2 sixth2 = f2(dtf / 6.f, dtf / 6.f), two2 = f2(2.f, 2.f);
      __nv_bfloat162 vlo[3][TR];
#pragma unroll
      for (int t = 0; t < TR; ++t)
#pragma unroll
        for (int c = 0; c < 3; ++c) vlo[c][t] = __float2bfloat162_rn(0.f);

      for (int n = 0; n < a.msteps; ++n) {
        const float om = a.om32[n + 1];
        float2 part2[3] = {f2(0.f, 0.f), f2(0.f, 0.f), f2(0.f, 0.f)};
#pragma unroll 1
        for (int st = 0; st < 4; ++st) {
          const float* in = st == 0 ? vA : (st == 2 ? vC : vB);   // this stage's state
          float* out = st == 1 ? vC : vB;                         // the next stage's state (st < 3)
          const float2 cnext = st == 2 ? dt2 : hdt2;              // its coefficient of k
          if (run) {
            float2 Hs[3][TR];
#pragma unroll
            for (int c = 0; c < 3; ++c)
              tile_stencil<R, TR>(in + c * cstrV, LD, ii0 + R, j0, afx, LDI, jj0, afy, LDY, ii0, yshfl, Hs[c]);
#pragma unroll
            for (int t = 0; t < TR; ++t) {
              const int ii = ii0 + t;
              if (!active || ii >= S) continue;
              const int ro = ii * LDI + jj0;
              const int vo = (ii + R) * LD + j0 + 1;
              float2 mi[3], v[3], m[3], H[3], k[3];
#pragma unroll
              for (int c = 0; c < 3; ++c) {
                mi[c] = lds2(miS + c * cstrI + ro);
                v[c] = lds2(vA + c * cstrV + vo);
                m[c] = add2(mi[c], st == 0 ? v[c] : lds2(in + c * cstrV + vo));
                H[c] = fma2(Hs[c][t], cs2, lds2(hiS + c * cstrI + ro));
              }
              ll_rhs2(m, H, alpha2, k);
              if (st < 3) {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                  float2* acc = accS + (c * TR + t) * ntile + tb;
                  *acc = st == 0 ? k[c] : fma2(two2, k[c], *acc);
                  float2 u = fma2(cnext, k[c], v[c]);
                  if (!col2) u.y = 0.f;
                  *reinterpret_cast<float2*>(out + c * cstrV + vo) = u;
                }
              } else {
                float2 dd[3], vt[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                  dd[c] = mul2(sixth2, add2(accS[(c * TR + t) * ntile + tb], k[c]));
                  vt[c] = add2(v[c], dd[c]);
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
                  const float2 inc = add2(fma2(cf, add2(mi[c], vt[c]), dd[c]), __bfloat1622float2(vlo[c][t]));
                  float2 nh = add2(v[c], inc);
                  vlo[c][t] = __float22bfloat162_rn(sub2(inc, sub2(nh, v[c])));
                  if (!col2) nh.y = 0.f;
                  *reinterpret_cast<float2*>(vA + c * cstrV + vo) = nh;
                  part2[c] = fma2(hw, sub2(nh, v[c]), part2[c]);
                }
              }
            }
          }
          __syncthreads();
          if (cs > 1) {
            push_halo<R, NC, SAC, ST, TR>(a, fsm, pk, st == 3 ? 0 : (st == 1 ? 2 : 1), rank, cs);
            cg::this_cluster().sync();
          }
        }
        if (om != 0.f) {
          float part[3] = {part2[0].x + part2[0].y, part2[1].x + part2[1].y, part2[2].x + part2[2].y};
          warp_kahan_add(kah, lane, om, part);
        }
      }
    }

    // ---- H_avg: s0 plus the Kahan sums of the box's warps; slabs of a cluster are
    // gathered on rank 0 and added in rank order.
    __syncthreads();
    if (tid < npack) {
      const PackBox& p = pk[tid];
      double acc[3] = {p.s0[0], p.s0[1], p.s0[2]};
      for (int w = p.warp0; w < p.warp0 + p.nwarps; ++w)
#pragma unroll
        for (int c = 0; c < 3; ++c) acc[c] += (double)kahA[6 * w + c] - (double)kahA[6 * w + 3 + c];
      if (cs == 1) {
        const BoxDesc& ob = a.boxes[p.box];
        const int pt = ob.p;
        double* out = ob.fax >= 0 ? a.Fout + (size_t)ob.fax * 3 * a.P : a.Havg;
        out[pt] = acc[0];
        out[a.P + pt] = acc[1];
        out[2 * a.P + pt] = acc[2];
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
        const BoxDesc& ob = a.boxes[pk[0].box];
        const int pt = ob.p;
        double* out = ob.fax >= 0 ? a.Fout + (size_t)ob.fax * 3 * a.P : a.Havg;
        out[pt] = acc[0];
        out[a.P + pt] = acc[1];
        out[2 * a.P + pt] = acc[2];
        if (!(isfinite(acc[0]) && isfinite(acc[1]) && isfinite(acc[2]))) atomicOr(a.err, kErrNonFinite);
      }
    }
  }
}

// A compiled instance of the kernel: radius, canvas (0: strides from the box) and
// the cluster size it is meant for (0: chosen per box).
struct ResVariant {
  int R, NC, SAC, cs;
  void (*fn)(MicroArgs, ResLaunch);
  int TZ;   // 3D: planes per thread tile (0 for 2D; -1: the z-column kernel, cs chosen per box)
  int stepper;   // micro stepper of the instance: 0 HeunP, 1 RK4P
  int tr;        // 2D: rows per thread tile (0: kResTR)
};

int res2d_variants_pack(const ResVariant** v);
int res2d_variants_cluster_a(const ResVariant** v);
int res2d_variants_cluster_b(const ResVariant** v);
int res2d_variants_any(const ResVariant** v);
int res2d_variants_rk4(const ResVariant** v);
int res2d_variants_tr2(const ResVariant** v);

}  // namespace hmm

// Batched FP32 micro kernel for 2D boxes held entirely on chip.
//
// Same mathematics and perturbation form as micro_fp32.cu (see there): v = m -
// m_init stepped by HeunP (Section 3.1) under H(m) = H(m_init) + H(v), the
// Dirichlet ring v = 0 (Section 4.2), the average of eq. upscaling evaluated as
// (sum_n w_n) sum_xi W H(m_init) + sum_n w_n sum_xi H(W)(xi) v^n(xi), by the
// symmetry of the discrete operator on fields that vanish on the ring.
//
// Layout: one CTA per box (atomic queue). The box's FP32 state lives in shared
// memory for all M steps: v^n (vA) and the stage state v^n + dt k1 (vB) on the
// whole box, m_init and H(m_init) on the interior, and the face coefficients of
// both axes. Each thread owns a tile of TR rows x 2 adjacent columns; the two
// columns are processed together with packed FP32x2 instructions. Per-node
// registers: k1 (stage 1 -> stage 2), the carried rounding error of v (v_lo, in
// bf16: it only has to carry a rounding error forward) and H(W) in FP32. The FP64 set-up (m_init, a^eps, H(m_init), H(W)) goes through
// the CTA's global arena once per box.
#include <cuda_bf16.h>

#include "micro_common.cuh"
#include "stencil.cuh"

namespace hmm {

constexpr int kResMaxInterior = 64;   // interior columns one warp covers (32 lanes x 2)
constexpr int kResLDI = 64;           // row stride of interior-only arrays (floats)
constexpr int kResLDY = 68;           // row stride of the y-face array (>= Ni + 3)

__host__ __device__ inline int res_ld(int nmax) { return (nmax + 4 + 1) & ~1; }

struct ResLayout {
  int LD;            // row stride of vA/vB
  size_t vA, vB, mi, hi, afx, afy, red;   // offsets in floats
  size_t total;      // floats
};

__host__ __device__ inline ResLayout res_layout(int nmax, int R) {
  ResLayout L;
  const int nimax = nmax - 2 * R;
  const int nfx = nimax + (R == 3 ? 3 : 1);
  L.LD = res_ld(nmax);
  size_t o = 0;
  L.vA = o; o += (size_t)3 * nmax * L.LD;
  L.vB = o; o += (size_t)3 * nmax * L.LD;
  L.mi = o; o += (size_t)3 * nimax * kResLDI;
  L.hi = o; o += (size_t)3 * nimax * kResLDI;
  L.afx = o; o += (size_t)nfx * kResLDI;
  L.afy = o; o += (size_t)nimax * kResLDY;
  o = (o + 1) & ~(size_t)1;          // 8-byte alignment for the doubles
  L.red = o; o += 2 * 96;
  L.total = o;
  return L;
}

size_t res2d_smem_bytes(int nmax, int R) { return res_layout(nmax, R).total * sizeof(float); }

// Set-up tables (FP64) overlay the vB region while a box is being set up.
bool res2d_setup_fits(int nmax, int R, int interp_k, int n_terms) {
  const ResLayout L = res_layout(nmax, R);
  return setup_smem_doubles(2, nmax, interp_k, n_terms) * 2 <= (size_t)3 * nmax * L.LD;
}

__host__ __device__ inline size_t res2d_arena_doubles(int nmax) { return (size_t)5 * nmax * nmax; }
size_t res2d_slot_bytes(int nmax) { return (res2d_arena_doubles(nmax) * 8 + 255) & ~(size_t)255; }

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, f2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 shift2(float2 a, float2 b) { return f2(a.y, b.x); }  // (a.y, b.x)

// Stencil of one component at the thread's TR x 2 tile. V: the component plane of
// vA or vB (row stride LD, column j at offset j + 1). Result H (unscaled) per row.
template <int R, int TR>
__device__ __forceinline__ void tile_stencil(const float* __restrict__ V, int LD, int N, int i0, int j0,
                                             const float* __restrict__ afx, int nf, int jj0,
                                             const float* __restrict__ afy_row0, int ii0, int Ni,
                                             float2* H) {
  constexpr int NP = TR + 2 * R;          // rows read
  float2 P[NP];
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    const int row = min(i0 - R + k, N - 1);
    P[k] = *reinterpret_cast<const float2*>(V + row * LD + j0 + 1);
  }
  // x direction (rows), faces between rows
  if (R == 3) {
    float2 F[TR + 3];
#pragma unroll
    for (int f = 0; f < TR + 3; ++f) {
      const float2 g = fma2(f2(27.f, 27.f), sub2(P[f + 2], P[f + 1]), sub2(P[f], P[f + 3]));
      const float2 ax = *reinterpret_cast<const float2*>(afx + min(ii0 + f, nf - 1) * kResLDI + jj0);
      F[f] = mul2(ax, g);
    }
#pragma unroll
    for (int t = 0; t < TR; ++t)
      H[t] = fma2(f2(27.f, 27.f), sub2(F[t + 2], F[t + 1]), sub2(F[t], F[t + 3]));
  } else {
    float2 F[TR + 1];
#pragma unroll
    for (int f = 0; f < TR + 1; ++f) {
      const float2 ax = *reinterpret_cast<const float2*>(afx + min(ii0 + f, nf - 1) * kResLDI + jj0);
      F[f] = mul2(ax, sub2(P[f + 1], P[f]));
    }
#pragma unroll
    for (int t = 0; t < TR; ++t) H[t] = sub2(F[t + 1], F[t]);
  }
  // y direction (columns), faces between columns, row by row
#pragma unroll
  for (int t = 0; t < TR; ++t) {
    const float* row = V + min(i0 + t, N - 1) * LD + j0 + 1;
    const float2 C = P[t + R];
    const float2 L1 = *reinterpret_cast<const float2*>(row - 2);
    const float2 R1 = *reinterpret_cast<const float2*>(row + 2);
    const float* ay = afy_row0 + min(ii0 + t, Ni - 1) * kResLDY + jj0;
    if (R == 3) {
      const float2 L2 = *reinterpret_cast<const float2*>(row - 4);
      const float r2x = row[4];
      const float2 a01 = *reinterpret_cast<const float2*>(ay);
      const float2 a23 = *reinterpret_cast<const float2*>(ay + 2);
      const float a4 = ay[4];
      // faces b = j0-2, j0-1 | j0, j0+1 | j0+2
      const float2 g01 = fma2(f2(27.f, 27.f), sub2(shift2(L1, C), L1), sub2(shift2(L2, L1), C));
      const float2 g23 = fma2(f2(27.f, 27.f), sub2(shift2(C, R1), C), sub2(shift2(L1, C), R1));
      const float g4 = (C.y - r2x) + 27.f * (R1.y - R1.x);
      const float2 F01 = mul2(a01, g01), F23 = mul2(a23, g23);
      const float F4 = a4 * g4;
      const float2 hy = fma2(f2(27.f, 27.f), sub2(F23, shift2(F01, F23)), sub2(F01, f2(F23.y, F4)));
      H[t] = add2(H[t], hy);
    } else {
      const float2 a01 = *reinterpret_cast<const float2*>(ay);
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
  const float2 p0 = sub2(mul2(m[1], H[2]), mul2(m[2], H[1]));
  const float2 p1 = sub2(mul2(m[2], H[0]), mul2(m[0], H[2]));
  const float2 p2 = sub2(mul2(m[0], H[1]), mul2(m[1], H[0]));
  const float2 d0 = sub2(mul2(m[1], p2), mul2(m[2], p1));
  const float2 d1 = sub2(mul2(m[2], p0), mul2(m[0], p2));
  const float2 d2 = sub2(mul2(m[0], p1), mul2(m[1], p0));
  const float2 mone = f2(-1.f, -1.f);
  f[0] = mul2(fma2(alpha, d0, p0), mone);
  f[1] = mul2(fma2(alpha, d1, p1), mone);
  f[2] = mul2(fma2(alpha, d2, p2), mone);
}

template <int R, int TR>
__global__ void __launch_bounds__(32 * ((kResMaxInterior + TR - 1) / TR))
micro_fp32_2d_kernel(MicroArgs a) {
  constexpr int D = 2;
  extern __shared__ __align__(16) float fsm[];
  __shared__ int s_box;
  const int nmax = a.nmax;
  const ResLayout Ly = res_layout(nmax, R);
  const int LD = Ly.LD;
  float* vA = fsm + Ly.vA;
  float* vB = fsm + Ly.vB;
  float* miS = fsm + Ly.mi;
  float* hiS = fsm + Ly.hi;
  float* afx = fsm + Ly.afx;
  float* afy = fsm + Ly.afy;
  double* red = reinterpret_cast<double*>(fsm + Ly.red);
  const SetupSmem sm = carve_setup(reinterpret_cast<double*>(vB), D, nmax, a.interp_k, a.n_terms);
  SetupSmem smr = sm;
  smr.red = red;

  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5;
  const size_t cap = (size_t)nmax * nmax;
  double* mi64 = reinterpret_cast<double*>(a.arena + (size_t)blockIdx.x * a.slot_bytes);
  double* af64 = mi64 + 3 * cap;
  const float am = (float)a.alpha_micro;
  const float2 alpha2 = f2(am, am);

  for (;;) {
    const int b = next_box(a.queue, &s_box);
    if (b >= a.n_boxes) break;
    const BoxDesc bd = a.boxes[b];
    const int N = bd.N, Ni = N - 2 * R;
    const int ntot = N * N;
    const Strides<D> st(N);
    box_setup_tables<D>(a, bd, smr);

    // ---- FP64 set-up through the arena: m_init (Section 4.1) and a^eps at the faces.
    int bad = 0;
    for (int idx = tid; idx < ntot; idx += nt) {
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
          v = face_coef<D>(a, smr, N, idx, k);
          bad |= !(v > 0.0);
        }
        af64[k * cap + idx] = v;
      }
    }
    if (bad) atomicOr(a.err, kErrCoefNonPositive);
    __syncthreads();   // the set-up tables (overlaying vB) are no longer needed

    // ---- Shared-memory fields: v = 0, m_init, face coefficients; H(m_init) below.
    for (int e = tid; e < 3 * nmax * LD; e += nt) {
      vA[e] = 0.f;
      vB[e] = 0.f;
    }
    const int f0 = R == 3 ? R - 2 : R - 1;     // first face row/column used by the stencil
    const int nf = Ni + (R == 3 ? 3 : 1);
    for (int e = tid; e < 3 * Ni * Ni; e += nt) {
      const int c = e / (Ni * Ni), r = e - c * Ni * Ni;
      const int ii = r / Ni, jj = r - ii * Ni;
      miS[(c * Ni + ii) * kResLDI + jj] = (float)mi64[c * cap + (ii + R) * N + (jj + R)];
    }
    for (int e = tid; e < nf * Ni; e += nt) {
      const int f = e / Ni, jj = e - f * Ni;
      afx[f * kResLDI + jj] = (float)af64[(f + f0) * N + (jj + R)];        // x-face between rows f+f0, f+f0+1
    }
    for (int e = tid; e < Ni * nf; e += nt) {
      const int ii = e / nf, g = e - ii * nf;
      afy[ii * kResLDY + g] = (float)af64[cap + (ii + R) * N + (g + f0)];   // y-face between columns g+f0, g+f0+1
    }

    // ---- Thread tile: rows i0.., columns j0, j0+1.
    const int ii0 = warp * TR;                 // first interior row of the tile
    const int i0 = R + ii0;
    const int jj0 = 2 * lane;
    const int j0 = R + jj0;
    const bool colok = jj0 < Ni;
    const bool tile_active = colok && ii0 < Ni;
    const float2 cmask = f2(1.f, (jj0 + 1 < Ni) ? 1.f : 0.f);   // odd Ni: the second column is ring
    const double cs64 = R == 3 ? 1.0 / ((24.0 * bd.dx) * (24.0 * bd.dx)) : 1.0 / (bd.dx * bd.dx);
    const double* W1d = a.W64 + bd.wofs;

    // H(m_init) (FP64) at the tile's nodes -> hiS; its weighted sum; H(W) -> registers.
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    float2 hw[TR];
#pragma unroll
    for (int t = 0; t < TR; ++t) {
      hw[t] = f2(0.f, 0.f);
      if (!tile_active || ii0 + t >= Ni) continue;
      float hwv[2] = {0.f, 0.f};
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        if (jj0 + q >= Ni) continue;
        const int idx = (i0 + t) * N + (j0 + q);
        double H[3];
        stencil_H<D, R, double>(mi64, af64, cap, st, idx, cs64, H);
        const double W = W1d[i0 + t] * W1d[j0 + q];
        s0 += W * H[0];
        s1 += W * H[1];
        s2 += W * H[2];
#pragma unroll
        for (int c = 0; c < 3; ++c) hiS[(c * Ni + ii0 + t) * kResLDI + jj0 + q] = (float)H[c];
        // H(W) with the same operator (W vanishes on and near the ring)
        double hwd = 0.0;
#pragma unroll
        for (int k = 0; k < D; ++k) {
          const int s = st.s[k];
          const double* af = af64 + k * cap;
          auto Wn = [&](int o) {
            const int id = idx + o * s;
            const int r_ = id / N, c_ = id - r_ * N;
            return W1d[r_] * W1d[c_];
          };
          if (R == 1) {
            hwd += af[idx] * (Wn(1) - Wn(0)) - af[idx - s] * (Wn(0) - Wn(-1));
          } else {
            const double m_3 = Wn(-3), m_2 = Wn(-2), m_1 = Wn(-1), m0 = Wn(0), m1 = Wn(1), m2 = Wn(2), m3 = Wn(3);
            hwd += (af[idx - 2 * s] * ((m_3 - m0) + 27.0 * (m_1 - m_2)) - af[idx + s] * ((m0 - m3) + 27.0 * (m2 - m1))) +
                   27.0 * (af[idx] * ((m_1 - m2) + 27.0 * (m1 - m0)) - af[idx - s] * ((m_2 - m1) + 27.0 * (m0 - m_1)));
          }
        }
        hwv[q] = (float)(hwd * cs64);
      }
      hw[t] = f2(hwv[0], hwv[1]);
    }
    {
      double wsum = 0.0;
      for (int n = 0; n <= a.msteps; ++n) wsum += a.w64[n];
      s0 *= wsum;
      s1 *= wsum;
      s2 *= wsum;
    }
    __syncthreads();

    // ---- Time loop.
    const float csf = (float)cs64;
    const float2 cs2 = f2(csf, csf);
    const float dtf = (float)bd.dt;
    const float2 dt2 = f2(dtf, dtf), hdt2 = f2(0.5f * dtf, 0.5f * dtf);
    float2 k1[3][TR];
    __nv_bfloat162 vlo[3][TR];
#pragma unroll
    for (int t = 0; t < TR; ++t)
#pragma unroll
      for (int c = 0; c < 3; ++c) vlo[c][t] = __float2bfloat162_rn(0.f);
    float ks[3] = {0.f, 0.f, 0.f}, kc[3] = {0.f, 0.f, 0.f};

    for (int n = 0; n <= a.msteps; ++n) {
      const float wn = a.w32[n];
      if (tile_active) {
        // The weighted sum of H(W) v^n (eq. upscaling through the operator's symmetry).
        float part[3] = {0.f, 0.f, 0.f};
        if (wn != 0.f) {
#pragma unroll
          for (int t = 0; t < TR; ++t) {
            if (ii0 + t >= Ni) continue;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              const float2 v = *reinterpret_cast<const float2*>(vA + (c * nmax + i0 + t) * LD + j0 + 1);
              const float2 p = mul2(hw[t], v);
              part[c] += p.x + p.y;
            }
          }
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const float y = wn * part[c] - kc[c];
            const float tt = ks[c] + y;
            kc[c] = (tt - ks[c]) - y;
            ks[c] = tt;
          }
        }
      }
      if (n == a.msteps) break;
      if (tile_active) {
        // Stage 1: k1 = f(m_init + v, H(m_init) + H(v)); vB = v + dt k1.
        float2 Hs[3][TR];
#pragma unroll
        for (int c = 0; c < 3; ++c)
          tile_stencil<R, TR>(vA + c * nmax * LD, LD, N, i0, j0, afx, nf, jj0, afy, ii0, Ni, Hs[c]);
#pragma unroll
        for (int t = 0; t < TR; ++t) {
          if (ii0 + t >= Ni) continue;
          float2 v[3], m[3], H[3], f[3];
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            v[c] = *reinterpret_cast<const float2*>(vA + (c * nmax + i0 + t) * LD + j0 + 1);
            m[c] = add2(*reinterpret_cast<const float2*>(miS + (c * Ni + ii0 + t) * kResLDI + jj0), v[c]);
            H[c] = fma2(Hs[c][t], cs2, *reinterpret_cast<const float2*>(hiS + (c * Ni + ii0 + t) * kResLDI + jj0));
          }
          ll_rhs2(m, H, alpha2, f);
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            k1[c][t] = f[c];
            *reinterpret_cast<float2*>(vB + (c * nmax + i0 + t) * LD + j0 + 1) = mul2(fma2(dt2, f[c], v[c]), cmask);
          }
        }
      }
      if (n == a.msteps) break;
      __syncthreads();
      if (tile_active) {
        // Stage 2: k2 = f(m_init + vB); v += dt/2 (k1 + k2) + projection, compensated.
        float2 Hs[3][TR];
#pragma unroll
        for (int c = 0; c < 3; ++c)
          tile_stencil<R, TR>(vB + c * nmax * LD, LD, N, i0, j0, afx, nf, jj0, afy, ii0, Ni, Hs[c]);
#pragma unroll
        for (int t = 0; t < TR; ++t) {
          if (ii0 + t >= Ni) continue;
          float2 mi[3], m[3], H[3], k2[3], vh[3], d[3], vt[3];
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            mi[c] = *reinterpret_cast<const float2*>(miS + (c * Ni + ii0 + t) * kResLDI + jj0);
            m[c] = add2(mi[c], *reinterpret_cast<const float2*>(vB + (c * nmax + i0 + t) * LD + j0 + 1));
            H[c] = fma2(Hs[c][t], cs2, *reinterpret_cast<const float2*>(hiS + (c * Ni + ii0 + t) * kResLDI + jj0));
          }
          ll_rhs2(m, H, alpha2, k2);
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            vh[c] = *reinterpret_cast<const float2*>(vA + (c * nmax + i0 + t) * LD + j0 + 1);
            d[c] = mul2(hdt2, add2(k1[c][t], k2[c]));
            vt[c] = add2(vh[c], d[c]);
          }
          // s = 2 m_init.vt + |vt|^2; c = -s / (sqrt(1+s)(1+sqrt(1+s)))
          float2 sdot = mul2(mi[0], vt[0]);
          sdot = fma2(mi[1], vt[1], sdot);
          sdot = fma2(mi[2], vt[2], sdot);
          float2 sq = mul2(vt[0], vt[0]);
          sq = fma2(vt[1], vt[1], sq);
          sq = fma2(vt[2], vt[2], sq);
          const float2 s = fma2(f2(2.f, 2.f), sdot, sq);
          const float r0 = rsqrtf(1.f + s.x), r1 = rsqrtf(1.f + s.y);
          const float2 cf = f2(-s.x * r0 * r0 / (1.f + r0), -s.y * r1 * r1 / (1.f + r1));
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const float2 inc = add2(fma2(cf, add2(mi[c], vt[c]), d[c]), __bfloat1622float2(vlo[c][t]));
            const float2 nh = add2(vh[c], inc);
            vlo[c][t] = __float22bfloat162_rn(sub2(inc, sub2(nh, vh[c])));
            *reinterpret_cast<float2*>(vA + (c * nmax + i0 + t) * LD + j0 + 1) = mul2(nh, cmask);
          }
        }
      }
      __syncthreads();
    }
    double acc0 = s0 + ((double)ks[0] - (double)kc[0]);
    double acc1 = s1 + ((double)ks[1] - (double)kc[1]);
    double acc2 = s2 + ((double)ks[2] - (double)kc[2]);
    block_sum3(acc0, acc1, acc2, red);
    if (tid == 0) {
      a.Havg[bd.p] = acc0;
      a.Havg[a.P + bd.p] = acc1;
      a.Havg[2 * a.P + bd.p] = acc2;
      if (!(isfinite(acc0) && isfinite(acc1) && isfinite(acc2))) atomicOr(a.err, kErrNonFinite);
    }
  }
}

constexpr int kResTR = 4;

int res2d_block(int nmax, int R) {
  const int ni = nmax - 2 * R;
  return 32 * ((ni + kResTR - 1) / kResTR);
}

template <int R>
static cudaError_t prepare_r(size_t smem, int* per_sm) {
  auto kern = micro_fp32_2d_kernel<R, kResTR>;
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, kern);
  if (e != cudaSuccess) return e;
  const int dyn_max = optin - (int)fa.sharedSizeBytes;
  if (smem > (size_t)dyn_max) return cudaErrorInvalidValue;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_max);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, kern, 32 * ((kResMaxInterior + kResTR - 1) / kResTR), smem);
}

cudaError_t prepare_micro_fp32_2d(int radius, size_t smem, int* ctas_per_sm) {
  return radius == 3 ? prepare_r<3>(smem, ctas_per_sm) : prepare_r<1>(smem, ctas_per_sm);
}

cudaError_t launch_micro_fp32_2d(const MicroArgs& a, int radius, int grid, int block, size_t smem,
                                 cudaStream_t st) {
  if (radius == 3) micro_fp32_2d_kernel<3, kResTR><<<grid, block, smem, st>>>(a);
  else micro_fp32_2d_kernel<1, kResTR><<<grid, block, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace hmm

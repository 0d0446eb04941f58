// Batched FP32 micro-batch kernel (perturbation form).
//
// The same mathematics as the FP64 kernel, stepped in FP32 on the perturbation
// v = m - m_init (0 on the Dirichlet ring, Section 4.2). Because the stencil is
// linear, H(m) = H(m_init) + H(v): H(m_init) is computed once per box in FP64
// from the FP64 m_init; the FP32 loop only sees H(v).
//
// Accuracy design (FP32 state, FP64 averages):
//  * The state is carried as v = v_hi + v_lo: each step forms its whole
//    increment (both Heun stages and the projection) in FP32, adds the carried
//    rounding error v_lo to it, and adds that to v_hi with an exact
//    (Fast2Sum) error term, which becomes the new v_lo. The stencil reads v_hi.
//  * The average (eq. upscaling) sum_n w_n sum_xi W H(m^n) equals, because the
//    discrete operator restricted to the interior is symmetric and W vanishes
//    on the ring, (sum_n w_n) sum_xi W H(m_init) + sum_xi H(W)(xi) V(xi) with
//    V = sum_n w_n v^n. V is accumulated per node in FP32 with Kahan
//    compensation; H(W) and both contractions are evaluated in FP64.
//  * MPE and MPEA (Section 3.1) keep h^n = H + alpha m x H per node for the next
//    steps and take the midpoint update in closed form (the Cayley transform, as
//    in the FP64 kernel); its increment goes through the same compensated sum.
//  * The HeunP projection (Section 3.1) is applied in perturbation form: with
//    u = m_init + v~ and s = |u|^2 - 1 (m_init taken as exactly unit, which its
//    FP64 value is), normalise(u) - m_init = v~ + c u, c = -s/(sqrt(1+s)(1+sqrt(1+s))),
//    so no O(1) component of m_init ever cancels in FP32.
#include "micro_common.cuh"
#include "stencil.cuh"

namespace hmm {

struct Fp32Slot {
  double* mi64;  // [3][cap] m_init, FP64 (set-up only)
  double* af64;  // [D][cap] face coefficients, FP64
  float* mi32;   // [3][cap]
  float* hi32;   // [3][cap] H(m_init) at interior nodes
  float* af32;   // [D][cap]
  float* vA;     // [3][cap] v_hi at step n
  float* vB;     // [3][cap] stage state v_hi + dt k1
  float* vlo;    // [3][cap] carried rounding error of v
  float* k1;     // [3][cap] stage-1 slope (RK4P: k1 + 2 k2 + 2 k3)
  float* V;      // [3][cap] sum_n w_n v_hi^n
  float* Vc;     // [3][cap] Kahan compensation of V
  float* vC;     // [3][cap] second stage state (RK4P)
  float* hX;     // [3][cap] MPE(A): h^{n-1} (only in slots sized for them)
  float* hY;     // [3][cap] MPE(A): h^{n-2}, overwritten by h^n
};

__host__ __device__ inline size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

__host__ __device__ inline size_t fp32_slot_bytes(int D, size_t cap, int stepper) {
  return align256(3 * cap * 8) + align256(D * cap * 8) + 2 * align256(3 * cap * 4) +
         align256(D * cap * 4) + (stepper >= 2 ? 9 : 7) * align256(3 * cap * 4);
}

__device__ inline Fp32Slot carve_fp32(char* base, int D, size_t cap) {
  Fp32Slot s;
  char* p = base;
  auto take = [&p](size_t bytes) { char* r = p; p += align256(bytes); return r; };
  s.mi64 = reinterpret_cast<double*>(take(3 * cap * 8));
  s.af64 = reinterpret_cast<double*>(take(D * cap * 8));
  s.mi32 = reinterpret_cast<float*>(take(3 * cap * 4));
  s.hi32 = reinterpret_cast<float*>(take(3 * cap * 4));
  s.af32 = reinterpret_cast<float*>(take(D * cap * 4));
  s.vA = reinterpret_cast<float*>(take(3 * cap * 4));
  s.vB = reinterpret_cast<float*>(take(3 * cap * 4));
  s.vlo = reinterpret_cast<float*>(take(3 * cap * 4));
  s.k1 = reinterpret_cast<float*>(take(3 * cap * 4));
  s.V = reinterpret_cast<float*>(take(3 * cap * 4));
  s.Vc = reinterpret_cast<float*>(take(3 * cap * 4));
  s.vC = reinterpret_cast<float*>(take(3 * cap * 4));
  s.hX = reinterpret_cast<float*>(take(3 * cap * 4));
  s.hY = reinterpret_cast<float*>(take(3 * cap * 4));
  return s;
}

// Spatial weight W(xi) at node idx (zero on and near the ring).
template <int D, typename T>
__device__ __forceinline__ T node_weight(const T* W1, int idx, int N) {
  int j[3];
  node_coords<D>(idx, N, j);
  T W = W1[j[0]];
  if (D > 1) W = W * W1[j[1]];
  if (D > 2) W = W * W1[j[2]];
  return W;
}

// H(W) at interior node idx in FP64 (the same staggered operator applied to W).
template <int D, int R>
__device__ __forceinline__ double stencil_of_weight(const double* W1, const double* af, size_t cap,
                                                    const Strides<D>& st, int idx, int N, double cs) {
  double acc = 0.0;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const int s = st.s[k];
    auto Wn = [&](int o) { return node_weight<D, double>(W1, idx + o * s, N); };
    const double* a = af + k * cap;
    if (R == 1) {
      acc += a[idx] * (Wn(1) - Wn(0)) - a[idx - s] * (Wn(0) - Wn(-1));
    } else {
      const double m_3 = Wn(-3), m_2 = Wn(-2), m_1 = Wn(-1), m0 = Wn(0), m1 = Wn(1), m2 = Wn(2), m3 = Wn(3);
      const double g_2 = (m_3 - m0) + 27.0 * (m_1 - m_2);
      const double g_1 = (m_2 - m1) + 27.0 * (m0 - m_1);
      const double g0 = (m_1 - m2) + 27.0 * (m1 - m0);
      const double g1 = (m0 - m3) + 27.0 * (m2 - m1);
      acc += (a[idx - 2 * s] * g_2 - a[idx + s] * g1) + 27.0 * (a[idx] * g0 - a[idx - s] * g_1);
    }
  }
  return acc * cs;
}

template <int D, int R>
__global__ void __launch_bounds__(256) micro_fp32_kernel(MicroArgs a) {
  const int nmax = a.nmax;
  extern __shared__ double smem[];
  __shared__ int s_box;
  const SetupSmem sm = carve_setup(smem, D, nmax, a.interp_k, a.n_terms);
  const int tid = threadIdx.x, nt = blockDim.x;
  const size_t cap = (size_t)ipow<D>(nmax);
  Fp32Slot sl = carve_fp32(a.arena + (size_t)blockIdx.x * a.slot_bytes, D, cap);
  const float am = (float)a.alpha_micro;

  for (;;) {
    const int b = next_box(a.queue, &s_box);
    if (b >= a.n_boxes) break;
    const BoxDesc bd = a.boxes[b];
    const int N = bd.N;
    const int ntot = ipow<D>(N);
    const Strides<D> st(N);
    box_setup_tables<D>(a, bd, sm);

    // FP64 set-up: m_init = Q_[2k] (Section 4.1) and a^eps at the faces; zero state.
    int bad = 0;
    for (int idx = tid; idx < ntot; idx += nt) {
      double P[3];
      interp_P<D>(a, sm, N, idx, P);
      const double inv = 1.0 / sqrt(P[0] * P[0] + P[1] * P[1] + P[2] * P[2]);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const double mv = P[c] * inv;
        const size_t o = c * cap + idx;
        sl.mi64[o] = mv;
        sl.mi32[o] = (float)mv;
        sl.vA[o] = 0.f;
        sl.vB[o] = 0.f;
        sl.vC[o] = 0.f;
        sl.vlo[o] = 0.f;
        sl.V[o] = 0.f;
        sl.Vc[o] = 0.f;
      }
      int j[3];
      node_coords<D>(idx, N, j);
#pragma unroll
      for (int k = 0; k < D; ++k) {
        double v = 0.0;
        if (j[k] < N - 1) {
          v = face_value<D>(a, bd, sm, N, idx, k);
          bad |= !(v > 0.0);
        }
        sl.af64[k * cap + idx] = v;
        sl.af32[k * cap + idx] = (float)v;
      }
    }
    if (bad) atomicOr(a.err, kErrCoefNonPositive);
    __syncthreads();

    const int nint = ipow<D>(N - 2 * R);
    const double cs64 = R == 3 ? 1.0 / ((24.0 * bd.dx) * (24.0 * bd.dx)) : 1.0 / (bd.dx * bd.dx);
    const float cs = (float)cs64;
    const double* W1d = a.W64 + bd.wofs;

    // H(m_init) in FP64 (stored in FP32 for the loop); sum_xi W H(m_init) in FP64.
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int t = tid; t < nint; t += nt) {
      const int idx = interior_node<D, R>(t, N);
      double H[3];
      stencil_H<D, R, double>(sl.mi64, sl.af64, cap, st, idx, cs64, H);
      const double W = node_weight<D, double>(W1d, idx, N);
      s0 += W * H[0];
      s1 += W * H[1];
      s2 += W * H[2];
#pragma unroll
      for (int c = 0; c < 3; ++c) sl.hi32[c * cap + idx] = (float)H[c];
    }
    double wsum = 0.0;
    for (int n = 0; n <= a.msteps; ++n) wsum += a.w64[n];
    // Flux model: the box averages the face flux along axis fax instead of H (the
    // face weights follow the node weights in the table); its m_init part in FP64.
    const int fax = bd.fax;
    const double cf = R == 3 ? 1.0 / (24.0 * bd.dx) : 1.0 / bd.dx;
    const int nsite = fax >= 0 ? nint / (N - 2 * R) * (N - 2 * R + 1) : 0;
    auto flux_sum = [&](const double* u, double& f0, double& f1, double& f2) {
      for (int t = tid; t < nsite; t += nt) {
        int j[3];
        const int idx = flux_site<D, R>(t, N, fax, j);
        double F[3];
        face_flux<R, double>(u, sl.af64 + (size_t)fax * cap, cap, idx, st.s[fax], cf, F);
        double W = 1.0;
#pragma unroll
        for (int ax = 0; ax < D; ++ax) W *= ax == fax ? W1d[N + j[ax]] : W1d[j[ax]];
        f0 += W * F[0];
        f1 += W * F[1];
        f2 += W * F[2];
      }
    };
    if (fax >= 0) {
      s0 = s1 = s2 = 0.0;
      flux_sum(sl.mi64, s0, s1, s2);
    }
    s0 *= wsum;
    s1 *= wsum;
    s2 *= wsum;
    __syncthreads();

    const float dt = (float)bd.dt, hdt = 0.5f * (float)bd.dt;
    const bool mpe = a.stepper >= 2;                 // MPE (2) or MPEA (3)
    const int nstart = a.stepper == 2 ? 1 : 2;       // their RK4P start-up steps
    const float e0 = a.stepper == 2 ? 1.5f : (float)(23.0 / 12.0), e1 = a.stepper == 2 ? -0.5f : (float)(-16.0 / 12.0),
                e2 = a.stepper == 2 ? 0.f : (float)(5.0 / 12.0);
    for (int n = 0; n < a.msteps; ++n) {
      const float wn = a.w32[n];
      const bool mp = mpe && n >= nstart;            // a midpoint step of MPE(A)
      const bool rk4 = a.stepper == 1 || (mpe && !mp);
      // HeunP: v_B = v + dt k1, d = dt/2 (k1 + k2). RK4P: v_B = v + dt/2 k1, the sum
      // k1 + 2 k2 + 2 k3 accumulated in sl.k1, d = dt/6 (k1 + 2 k2 + 2 k3 + k4).
      const float cb1 = rk4 ? hdt : dt, cdl = rk4 ? (float)(bd.dt / 6.0) : hdt;
      // Stage 1: k1 = f(m_init + v), v_B = v + dt k1, V += w_n v (Kahan).
      for (int t = tid; t < nint; t += nt) {
        const int idx = interior_node<D, R>(t, N);
        float Hv[3];
        stencil_H<D, R, float>(sl.vA, sl.af32, cap, st, idx, cs, Hv);
#pragma unroll
        for (int c = 0; c < 3; ++c) Hv[c] += sl.hi32[c * cap + idx];
        float v[3], m[3], k1[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          v[c] = sl.vA[c * cap + idx];
          m[c] = sl.mi32[c * cap + idx] + v[c];
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {   // V += w_n v^n (Kahan)
          const size_t o = c * cap + idx;
          const float y = wn * v[c] - sl.Vc[o];
          const float tV = sl.V[o] + y;
          sl.Vc[o] = (tV - sl.V[o]) - y;
          sl.V[o] = tV;
        }
        if (mpe) {
          // h^n (eq. h_term), kept as h^{n-1} for the next step (in hY, whose h^{n-2}
          // this step reads first)
          const float hn[3] = {Hv[0] + am * (m[1] * Hv[2] - m[2] * Hv[1]), Hv[1] + am * (m[2] * Hv[0] - m[0] * Hv[2]),
                               Hv[2] + am * (m[0] * Hv[1] - m[1] * Hv[0])};
          if (mp) {
            float w[3];
#pragma unroll
            for (int c = 0; c < 3; ++c)
              w[c] = hdt * (e0 * hn[c] + e1 * sl.hX[c * cap + idx] + e2 * sl.hY[c * cap + idx]);
            const float wm[3] = {w[1] * m[2] - w[2] * m[1], w[2] * m[0] - w[0] * m[2], w[0] * m[1] - w[1] * m[0]};
            const float g = 2.f / (1.f + (w[0] * w[0] + w[1] * w[1] + w[2] * w[2]));
            const float d[3] = {g * (wm[0] + (w[1] * wm[2] - w[2] * wm[1])), g * (wm[1] + (w[2] * wm[0] - w[0] * wm[2])),
                                g * (wm[2] + (w[0] * wm[1] - w[1] * wm[0]))};
#pragma unroll
            for (int c = 0; c < 3; ++c) {   // v^{n+1} = v^n + d, compensated, into vB
              const size_t o = c * cap + idx;
              const float inc = d[c] + sl.vlo[o];
              const float nh = v[c] + inc;
              sl.vlo[o] = inc - (nh - v[c]);
              sl.vB[o] = nh;
            }
          }
#pragma unroll
          for (int c = 0; c < 3; ++c) sl.hY[c * cap + idx] = hn[c];
          if (mp) continue;
        }
        ll_rhs(m, Hv, am, k1);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const size_t o = c * cap + idx;
          sl.k1[o] = k1[c];
          sl.vB[o] = v[c] + cb1 * k1[c];
        }
      }
      __syncthreads();
      if (mpe) {   // h^n becomes h^{n-1}, h^{n-1} becomes h^{n-2}
        float* t = sl.hX;
        sl.hX = sl.hY;
        sl.hY = t;
      }
      if (mp) {    // v^{n+1} was written to vB
        float* t = sl.vA;
        sl.vA = sl.vB;
        sl.vB = t;
        continue;
      }
      if (rk4) {
        // RK4P stages 2 and 3: k2 = f(m_init + v + dt/2 k1) (state in v_B), k3 =
        // f(m_init + v + dt/2 k2) (state in v_C); the last stage's state v + dt k3 goes to v_B.
        for (int stage = 2; stage <= 3; ++stage) {
          const float* src = stage == 2 ? sl.vB : sl.vC;
          float* dst = stage == 2 ? sl.vC : sl.vB;
          const float cn = stage == 2 ? hdt : dt;
          for (int t = tid; t < nint; t += nt) {
            const int idx = interior_node<D, R>(t, N);
            float Hv[3];
            stencil_H<D, R, float>(src, sl.af32, cap, st, idx, cs, Hv);
            float m[3], k[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              Hv[c] += sl.hi32[c * cap + idx];
              m[c] = sl.mi32[c * cap + idx] + src[c * cap + idx];
            }
            ll_rhs(m, Hv, am, k);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              const size_t o = c * cap + idx;
              sl.k1[o] += 2.f * k[c];
              dst[o] = sl.vA[o] + cn * k[c];
            }
          }
          __syncthreads();
        }
      }
      // Last stage: k = f(m_init + v_B); the step's increment d = cdl (sum of the
      // earlier slopes + k) plus the projection, added to v = v_hi + v_lo with an
      // exact error term.
      for (int t = tid; t < nint; t += nt) {
        const int idx = interior_node<D, R>(t, N);
        float Hv[3];
        stencil_H<D, R, float>(sl.vB, sl.af32, cap, st, idx, cs, Hv);
        float mi[3], m[3], k2[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          Hv[c] += sl.hi32[c * cap + idx];
          mi[c] = sl.mi32[c * cap + idx];
          m[c] = mi[c] + sl.vB[c * cap + idx];
        }
        ll_rhs(m, Hv, am, k2);
        float vh[3], d[3], vt[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          vh[c] = sl.vA[c * cap + idx];
          d[c] = cdl * (sl.k1[c * cap + idx] + k2[c]);
          vt[c] = vh[c] + d[c];
        }
        const float s = 2.f * (mi[0] * vt[0] + mi[1] * vt[1] + mi[2] * vt[2]) +
                        (vt[0] * vt[0] + vt[1] * vt[1] + vt[2] * vt[2]);
        const float r = rsqrtf(1.f + s);
        const float cf = -s * r * r / (1.f + r);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const size_t o = c * cap + idx;
          const float inc = (d[c] + cf * (mi[c] + vt[c])) + sl.vlo[o];
          const float nh = vh[c] + inc;
          sl.vlo[o] = inc - (nh - vh[c]);
          sl.vA[o] = nh;
        }
      }
      __syncthreads();
    }
    // The final state's weight w_M (zero for K0 in K0^{p,q}) and the contraction with H(W).
    const float wM = a.w32[a.msteps];
    if (fax >= 0) {
      // Flux model: sum_n w_n F(v^n) = F(V), V = sum_n w_n v^n, the face flux of the
      // accumulated state; V (zero on the ring) goes through the FP64 m_init scratch.
      for (int idx = tid; idx < ntot; idx += nt) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const size_t o = c * cap + idx;
          sl.mi64[o] = ((double)sl.V[o] - (double)sl.Vc[o]) + (double)wM * (double)sl.vA[o];
        }
      }
      __syncthreads();
      flux_sum(sl.mi64, s0, s1, s2);
    }
    for (int t = tid; t < (fax >= 0 ? 0 : nint); t += nt) {
      const int idx = interior_node<D, R>(t, N);
      const double hw = stencil_of_weight<D, R>(W1d, sl.af64, cap, st, idx, N, cs64);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const size_t o = c * cap + idx;
        const double Vt = ((double)sl.V[o] - (double)sl.Vc[o]) + (double)wM * (double)sl.vA[o];
        const double contrib = hw * Vt;
        if (c == 0) s0 += contrib;
        if (c == 1) s1 += contrib;
        if (c == 2) s2 += contrib;
      }
    }
    block_sum3(s0, s1, s2, sm.red);
    if (tid == 0) {
      double* out = fax >= 0 ? a.Fout + (size_t)fax * 3 * a.P : a.Havg;
      out[bd.p] = s0;
      out[a.P + bd.p] = s1;
      out[2 * a.P + bd.p] = s2;
      if (!(isfinite(s0) && isfinite(s1) && isfinite(s2))) atomicOr(a.err, kErrNonFinite);
    }
  }
}

template <int D, int R>
static cudaError_t launch_t(const MicroArgs& a, int grid, int block, size_t smem, cudaStream_t st) {
  micro_fp32_kernel<D, R><<<grid, block, smem, st>>>(a);
  return cudaGetLastError();
}

template <int D, int R>
static cudaError_t prepare_t(int block, size_t smem, int* per_sm) {
  auto kern = micro_fp32_kernel<D, R>;
  // Raise the kernel's limit to the device's opt-in maximum once, so that
  // handles with different table sizes never lower it for each other.
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
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, kern, block, smem);
}

#define HMM_DISPATCH(FN, ...)                                      \
  do {                                                              \
    if (radius == 3) {                                             \
      if (dim == 1) return FN<1, 3>(__VA_ARGS__);                  \
      if (dim == 2) return FN<2, 3>(__VA_ARGS__);                  \
      if (dim == 3) return FN<3, 3>(__VA_ARGS__);                  \
    } else if (radius == 1) {                                     \
      if (dim == 1) return FN<1, 1>(__VA_ARGS__);                  \
      if (dim == 2) return FN<2, 1>(__VA_ARGS__);                  \
      if (dim == 3) return FN<3, 1>(__VA_ARGS__);                  \
    }                                                              \
    return cudaErrorInvalidValue;                                  \
  } while (0)

cudaError_t launch_micro_fp32(const MicroArgs& a, int dim, int radius, int grid, int block,
                              size_t smem, cudaStream_t st) {
  HMM_DISPATCH(launch_t, a, grid, block, smem, st);
}

cudaError_t prepare_micro_fp32(int dim, int radius, int block, size_t smem, int* ctas_per_sm) {
  HMM_DISPATCH(prepare_t, block, smem, ctas_per_sm);
}

size_t micro_slot_bytes_fp32(int dim, int nmax, int stepper) {
  size_t cap = 1;
  for (int i = 0; i < dim; ++i) cap *= (size_t)nmax;
  return align256(fp32_slot_bytes(dim, cap, stepper));
}

}  // namespace hmm

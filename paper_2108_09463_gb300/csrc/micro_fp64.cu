// Plain FP64 micro-batch kernel: the micro problem (eq. micro) of every macro
// point, stepped by HeunP, RK4P, MPE or MPEA (Section 3.1) with the Dirichlet ring (Section 4.2),
// and reduced by the kernel-weighted average (Section 2.3, eq. upscaling), all
// in FP64 arithmetic. One CTA per box, boxes pulled from an atomic queue.
//
// The state is carried as v = m - m_init. Since H is linear, H(m) = H(m_init) +
// H(v) and the scheme is unchanged; what changes is the rounding: increments of
// size dt |f| are added to |v| ~ eps |grad m| instead of to |m| = 1, so the
// FP64 rounding floor of H_avg drops from ~1e-12 (the m-form) to ~1e-15.
// The projection m^{n+1} = m~/|m~| becomes v^{n+1} = v~ + c (m_init + v~) with
// s = |m_init + v~|^2 - 1 and c = -s / (sqrt(1+s) (1 + sqrt(1+s))).
//
// MPE and MPEA (eqs. h_mpe, h_mpea, mpe_update): after one (MPE) or two (MPEA)
// RK4P start-up steps, h^n = H(m^n) + alpha m^n x H(m^n) (eq. h_term) is kept per
// node for the next steps, h^{n+1/2} extrapolated from h^n, h^{n-1} (and h^{n-2}),
// and the midpoint update solved per node in closed form: with w = dt/2 h^{n+1/2},
// (I - [w]x) m' = (I + [w]x) m gives m' = m + 2/(1 + |w|^2) (w x m + w x (w x m))
// (the Cayley transform; (I - [w]x)^{-1} = I + ([w]x + [w]x^2)/(1 + |w|^2)).
#include "micro_common.cuh"
#include "stencil.cuh"

namespace hmm {

template <int D, int R>
__global__ void __launch_bounds__(256) micro_fp64_kernel(MicroArgs a) {
  const int nmax = a.nmax;
  extern __shared__ double smem[];
  __shared__ int s_box;
  const SetupSmem sm = carve_setup(smem, D, nmax, a.interp_k, a.n_terms);
  const int tid = threadIdx.x, nt = blockDim.x;
  const size_t cap = (size_t)ipow<D>(nmax);
  double* mi = reinterpret_cast<double*>(a.arena + (size_t)blockIdx.x * a.slot_bytes);
  double* hi = mi + 3 * cap;  // H(m_init)
  double* vA = hi + 3 * cap;
  double* vB = vA + 3 * cap;
  double* q = vB + 3 * cap;   // the step's accumulated state v + dt sum b_i k_i (MPE(A): v^{n+1})
  double* vC = q + 3 * cap;   // second stage state (RK4P)
  double* af = vC + 3 * cap;
  double* hX = af + D * cap;  // MPE(A): h^{n-1} (only in slots sized for them)
  double* hY = hX + 3 * cap;  // MPE(A): h^{n-2}, overwritten by h^n

  for (;;) {
    const int b = next_box(a.queue, &s_box);
    if (b >= a.n_boxes) break;
    const BoxDesc bd = a.boxes[b];
    const int N = bd.N;
    const int ntot = ipow<D>(N);
    const Strides<D> st(N);
    box_setup_tables<D>(a, bd, sm);

    // Initial data Q_[2k] at every node (Section 4.1), a^eps at every face, v = 0.
    int bad = 0;
    for (int idx = tid; idx < ntot; idx += nt) {
      double P[3];
      interp_P<D>(a, sm, N, idx, P);
      const double inv = 1.0 / sqrt(P[0] * P[0] + P[1] * P[1] + P[2] * P[2]);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        mi[c * cap + idx] = P[c] * inv;
        vA[c * cap + idx] = 0.0;
        vB[c * cap + idx] = 0.0;
        vC[c * cap + idx] = 0.0;
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
        af[k * cap + idx] = v;
      }
    }
    if (bad) atomicOr(a.err, kErrCoefNonPositive);
    __syncthreads();

    const double dt = bd.dt, hdt = 0.5 * bd.dt;
    const bool mpe = a.stepper >= 2;                 // MPE (2) or MPEA (3)
    const int nstart = a.stepper == 2 ? 1 : 2;       // their RK4P start-up steps
    const double e0 = a.stepper == 2 ? 1.5 : 23.0 / 12.0, e1 = a.stepper == 2 ? -0.5 : -16.0 / 12.0,
                 e2 = a.stepper == 2 ? 0.0 : 5.0 / 12.0;
    const double cs = R == 3 ? 1.0 / ((24.0 * bd.dx) * (24.0 * bd.dx)) : 1.0 / (bd.dx * bd.dx);
    const double* W1 = a.W64 + bd.wofs;
    const int nint = ipow<D>(N - 2 * R);
    double acc0 = 0.0, acc1 = 0.0, acc2 = 0.0;
    // Flux model: the box averages the face flux along axis fax (weights at the
    // face positions follow the node weights in the table) instead of H.
    const int fax = bd.fax;
    const double* Wf1 = W1 + N;
    const double cf = R == 3 ? 1.0 / (24.0 * bd.dx) : 1.0 / bd.dx;
    const int nsite = fax >= 0 ? ipow<D>(N - 2 * R) / (N - 2 * R) * (N - 2 * R + 1) : 0;
    auto flux_sum = [&](const double* u, double w, double& f0, double& f1, double& f2) {
      for (int t = tid; t < nsite; t += nt) {
        int j[3];
        const int idx = flux_site<D, R>(t, N, fax, j);
        double F[3];
        face_flux<R, double>(u, af + (size_t)fax * cap, cap, idx, st.s[fax], cf, F);
        double W = w;
#pragma unroll
        for (int ax = 0; ax < D; ++ax) W *= ax == fax ? Wf1[j[ax]] : W1[j[ax]];
        f0 += W * F[0];
        f1 += W * F[1];
        f2 += W * F[2];
      }
    };

    // H(m_init) and its weighted sum (times sum_n w_n).
    {
      double s0 = 0.0, s1 = 0.0, s2 = 0.0;
      for (int t = tid; t < nint; t += nt) {
        const int idx = interior_node<D, R>(t, N);
        double H[3];
        stencil_H<D, R, double>(mi, af, cap, st, idx, cs, H);
        int j[3];
        node_coords<D>(idx, N, j);
        double W = W1[j[0]];
        if (D > 1) W = W * W1[j[1]];
        if (D > 2) W = W * W1[j[2]];
        s0 += W * H[0];
        s1 += W * H[1];
        s2 += W * H[2];
#pragma unroll
        for (int c = 0; c < 3; ++c) hi[c * cap + idx] = H[c];
      }
      double wsum = 0.0;
      for (int n = 0; n <= a.msteps; ++n) wsum += a.w64[n];
      if (fax >= 0) {             // the flux of m_init instead of H(m_init)
        s0 = s1 = s2 = 0.0;
        flux_sum(mi, 1.0, s0, s1, s2);
      }
      acc0 = s0 * wsum;
      acc1 = s1 * wsum;
      acc2 = s2 * wsum;
    }
    __syncthreads();

    for (int n = 0; n <= a.msteps; ++n) {
      const double wn = a.w64[n];
      if (n == a.msteps && wn == 0.0) break;  // K0(1) = 0: no final stencil pass
      const bool mp = mpe && n >= nstart;      // a midpoint step of MPE(A)
      const bool rk4 = a.stepper == 1 || (mpe && !mp);
      // stage-1 coefficients: q = v + cq1 k1, vB = v + cb1 k1; the last stage adds cql k_last
      const double cq1 = rk4 ? dt / 6.0 : hdt, cb1 = rk4 ? hdt : dt, cql = rk4 ? dt / 6.0 : hdt;
      if (fax >= 0 && wn != 0.0) flux_sum(vA, wn, acc0, acc1, acc2);   // v^n is read-only in stage 1
      if (fax >= 0 && n == a.msteps) break;
      // Stage 1: H(m^n) = H(m_init) + H(v^n), its weighted sum, k1, v + dt k1, v + dt/2 k1.
      for (int t = tid; t < nint; t += nt) {
        const int idx = interior_node<D, R>(t, N);
        double Hv[3];
        stencil_H<D, R, double>(vA, af, cap, st, idx, cs, Hv);
        if (fax < 0 && wn != 0.0) {
          int j[3];
          node_coords<D>(idx, N, j);
          double W = W1[j[0]];
          if (D > 1) W = W * W1[j[1]];
          if (D > 2) W = W * W1[j[2]];
          const double ww = wn * W;
          acc0 += ww * Hv[0];
          acc1 += ww * Hv[1];
          acc2 += ww * Hv[2];
        }
        if (n == a.msteps) continue;
        double v[3], m[3], H[3], k1[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          v[c] = vA[c * cap + idx];
          m[c] = mi[c * cap + idx] + v[c];
          H[c] = hi[c * cap + idx] + Hv[c];
        }
        if (mpe) {
          // h^n (eq. h_term), kept as h^{n-1} for the next step (in hY, whose h^{n-2}
          // this step reads first)
          const double h0 = H[0] + a.alpha_micro * (m[1] * H[2] - m[2] * H[1]);
          const double h1 = H[1] + a.alpha_micro * (m[2] * H[0] - m[0] * H[2]);
          const double h2 = H[2] + a.alpha_micro * (m[0] * H[1] - m[1] * H[0]);
          if (mp) {
            double w[3];
            const double hn[3] = {h0, h1, h2};
#pragma unroll
            for (int c = 0; c < 3; ++c)
              w[c] = hdt * (e0 * hn[c] + e1 * hX[c * cap + idx] + e2 * hY[c * cap + idx]);
            const double wm0 = w[1] * m[2] - w[2] * m[1], wm1 = w[2] * m[0] - w[0] * m[2],
                         wm2 = w[0] * m[1] - w[1] * m[0];
            const double g = 2.0 / (1.0 + (w[0] * w[0] + w[1] * w[1] + w[2] * w[2]));
            q[idx] = v[0] + g * (wm0 + (w[1] * wm2 - w[2] * wm1));
            q[cap + idx] = v[1] + g * (wm1 + (w[2] * wm0 - w[0] * wm2));
            q[2 * cap + idx] = v[2] + g * (wm2 + (w[0] * wm1 - w[1] * wm0));
          }
          hY[idx] = h0;
          hY[cap + idx] = h1;
          hY[2 * cap + idx] = h2;
          if (mp) continue;
        }
        ll_rhs(m, H, a.alpha_micro, k1);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          q[c * cap + idx] = v[c] + cq1 * k1[c];
          vB[c * cap + idx] = v[c] + cb1 * k1[c];
        }
      }
      if (n == a.msteps) break;
      __syncthreads();
      if (mpe) {   // h^n becomes h^{n-1}, h^{n-1} becomes h^{n-2}
        double* t = hX;
        hX = hY;
        hY = t;
      }
      if (mp) {    // v^{n+1} was written to q
        double* t = vA;
        vA = q;
        q = t;
        continue;
      }
      if (rk4) {
        // RK4P stages 2 and 3: k2 = f(v + dt/2 k1) (state in vB), k3 = f(v + dt/2 k2)
        // (state in vC); q += dt/3 (k2 + k3); the last stage's state v + dt k3 goes to vB.
        for (int stage = 2; stage <= 3; ++stage) {
          const double* src = stage == 2 ? vB : vC;
          double* dst = stage == 2 ? vC : vB;
          const double cn = stage == 2 ? hdt : dt;
          for (int t = tid; t < nint; t += nt) {
            const int idx = interior_node<D, R>(t, N);
            double Hv[3];
            stencil_H<D, R, double>(src, af, cap, st, idx, cs, Hv);
            double m[3], H[3], k[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              m[c] = mi[c * cap + idx] + src[c * cap + idx];
              H[c] = hi[c * cap + idx] + Hv[c];
            }
            ll_rhs(m, H, a.alpha_micro, k);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              q[c * cap + idx] += (dt / 3.0) * k[c];
              dst[c * cap + idx] = vA[c * cap + idx] + cn * k[c];
            }
          }
          __syncthreads();
        }
      }
      // Last stage: k = f(m_init + vB), m^{n+1} = normalise(m_init + q + cql k), as v.
      for (int t = tid; t < nint; t += nt) {
        const int idx = interior_node<D, R>(t, N);
        double Hv[3];
        stencil_H<D, R, double>(vB, af, cap, st, idx, cs, Hv);
        double mv[3], m[3], H[3], k2[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          mv[c] = mi[c * cap + idx];
          m[c] = mv[c] + vB[c * cap + idx];
          H[c] = hi[c * cap + idx] + Hv[c];
        }
        ll_rhs(m, H, a.alpha_micro, k2);
        double vt[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) vt[c] = q[c * cap + idx] + cql * k2[c];
        const double s = 2.0 * (mv[0] * vt[0] + mv[1] * vt[1] + mv[2] * vt[2]) +
                         (vt[0] * vt[0] + vt[1] * vt[1] + vt[2] * vt[2]) +
                         ((mv[0] * mv[0] + mv[1] * mv[1] + mv[2] * mv[2]) - 1.0);
        const double rt = sqrt(1.0 + s);
        const double cf = -s / (rt * (1.0 + rt));
#pragma unroll
        for (int c = 0; c < 3; ++c) vA[c * cap + idx] = vt[c] + cf * (mv[c] + vt[c]);
      }
      __syncthreads();
    }
    block_sum3(acc0, acc1, acc2, sm.red);
    if (tid == 0) {
      double* out = fax >= 0 ? a.Fout + (size_t)fax * 3 * a.P : a.Havg;
      out[bd.p] = acc0;
      out[a.P + bd.p] = acc1;
      out[2 * a.P + bd.p] = acc2;
      if (!(isfinite(acc0) && isfinite(acc1) && isfinite(acc2))) atomicOr(a.err, kErrNonFinite);
    }
  }
}

template <int D, int R>
static cudaError_t launch_t(const MicroArgs& a, int grid, int block, size_t smem, cudaStream_t st) {
  micro_fp64_kernel<D, R><<<grid, block, smem, st>>>(a);
  return cudaGetLastError();
}

template <int D, int R>
static cudaError_t prepare_t(int block, size_t smem, int* per_sm) {
  auto kern = micro_fp64_kernel<D, R>;
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

cudaError_t launch_micro_fp64(const MicroArgs& a, int dim, int radius, int grid, int block,
                              size_t smem, cudaStream_t st) {
  HMM_DISPATCH(launch_t, a, grid, block, smem, st);
}

cudaError_t prepare_micro_fp64(int dim, int radius, int block, size_t smem, int* ctas_per_sm) {
  HMM_DISPATCH(prepare_t, block, smem, ctas_per_sm);
}

size_t micro_smem_bytes(int dim, int nmax, int interp_k, int n_terms) {
  return sizeof(double) * setup_smem_doubles(dim, nmax, interp_k, n_terms);
}

size_t micro_slot_bytes_fp64(int dim, int nmax, int stepper) {
  size_t cap = 1;
  for (int i = 0; i < dim; ++i) cap *= (size_t)nmax;
  size_t b = (size_t)(6 * 3 + dim + (stepper >= 2 ? 6 : 0)) * cap * sizeof(double);
  return (b + 255) & ~(size_t)255;
}

}  // namespace hmm

// Macro-side kernels of the field model (Section 2.2, eq. macro_disc), FP64,
// one thread per macro point:
//  - MPEA: h^j = H + alpha M x H (eq. h_term), h^{j+1/2} = 23/12 h^j - 16/12
//    h^{j-1} + 5/12 h^{j-2} (eq. h_mpea) (MPE: 3/2 h^j - 1/2 h^{j-1}, eq. h_mpe),
//    and the midpoint update
//    (M' - M)/dt = -(M + M')/2 x h^{j+1/2} (eq. mpe_update), solved in closed
//    form: with w = dt/2 h, (I - [w]x) M' = (I + [w]x) M, whose solution is
//    M' = M + 2/(1 + |w|^2) (w x M + w x (w x M)).
//  - RK4P stages (Section 3.1) with normalised stage states.
#include "hmm_internal.cuh"

namespace hmm {

__device__ __forceinline__ void cross3(const double* a, const double* b, double* c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

__device__ __forceinline__ void load3(const double* x, int P, int p, double* v) {
  v[0] = x[p];
  v[1] = x[P + p];
  v[2] = x[2 * P + p];
}

__device__ __forceinline__ void store3(double* x, int P, int p, const double* v) {
  x[p] = v[0];
  x[P + p] = v[1];
  x[2 * P + p] = v[2];
}

__global__ void h_term_kernel(const double* M, const double* H, double alpha, double* h, int P) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  double m[3], Hv[3], c[3];
  load3(M, P, p, m);
  load3(H, P, p, Hv);
  cross3(m, Hv, c);
  for (int i = 0; i < 3; ++i) c[i] = Hv[i] + alpha * c[i];
  store3(h, P, p, c);
}

__global__ void mpea_kernel(double* M, const double* H, double* hist, double alpha, double dt, double c0, double c1,
                            double c2, int P) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  double m[3], Hv[3], c[3], h1[3], h2[3], hj[3], w[3];
  load3(M, P, p, m);
  load3(H, P, p, Hv);
  load3(hist, P, p, h1);
  load3(hist + 3 * (size_t)P, P, p, h2);
  cross3(m, Hv, c);
  for (int i = 0; i < 3; ++i) hj[i] = Hv[i] + alpha * c[i];
  for (int i = 0; i < 3; ++i)
    w[i] = 0.5 * dt * (c0 * hj[i] + c1 * h1[i] + c2 * h2[i]);
  double wm[3], wwm[3];
  cross3(w, m, wm);
  cross3(w, wm, wwm);
  const double f = 2.0 / (1.0 + w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
  double out[3];
  for (int i = 0; i < 3; ++i) out[i] = m[i] + f * (wm[i] + wwm[i]);
  store3(M, P, p, out);
  store3(hist + 3 * (size_t)P, P, p, h1);
  store3(hist, P, p, hj);
}

// RK4P stage s (1..4). Ms: the (normalised) stage state whose micro batch gave H.
// Stage 1 also shifts the MPEA history and stores h^j = H + alpha M x H.
__global__ void rk4_stage_kernel(const double* M, const double* Ms, const double* H, double alpha,
                                 double dt, int stage, double* acc, double* Mnext, double* hist,
                                 int P) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  double m[3], ms[3], Hv[3], mxH[3], mmxH[3], k[3];
  load3(M, P, p, m);
  load3(Ms, P, p, ms);
  load3(H, P, p, Hv);
  cross3(ms, Hv, mxH);
  cross3(ms, mxH, mmxH);
  for (int i = 0; i < 3; ++i) k[i] = -mxH[i] - alpha * mmxH[i];
  double a[3];
  if (stage == 1) {
    double hj[3], old[3];
    for (int i = 0; i < 3; ++i) hj[i] = Hv[i] + alpha * mxH[i];
    load3(hist, P, p, old);
    store3(hist + 3 * (size_t)P, P, p, old);
    store3(hist, P, p, hj);
    for (int i = 0; i < 3; ++i) a[i] = k[i];
  } else {
    load3(acc, P, p, a);
    const double wk = stage == 4 ? 1.0 : 2.0;
    for (int i = 0; i < 3; ++i) a[i] += wk * k[i];
  }
  store3(acc, P, p, a);
  double u[3];
  if (stage == 4) {
    for (int i = 0; i < 3; ++i) u[i] = m[i] + (dt / 6.0) * a[i];
  } else {
    const double c = stage == 3 ? dt : 0.5 * dt;
    for (int i = 0; i < 3; ++i) u[i] = m[i] + c * k[i];
  }
  const double inv = 1.0 / sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
  for (int i = 0; i < 3; ++i) u[i] *= inv;
  store3(Mnext, P, p, u);
}

__global__ void check_finite_kernel(const double* x, int n, int* err) {
  int bad = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    bad |= !isfinite(x[i]);
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(err, kErrNonFinite);
}

// Flux model (eq. macro_flux): H_i = sum_k D_k F_k at macro point i, F_k's entry i
// the flux column k at x_i + (DX_k/2) e_k. Order 4: (F_{i-3/2} - 27 F_{i-1/2} +
// 27 F_{i+1/2} - F_{i+3/2}) / (24 DX_k); order 2: (F_{i+1/2} - F_{i-1/2}) / DX_k;
// indices periodic.
__global__ void flux_div_kernel(const double* F, double* H, int dim, int n0, int n1, int n2,
                                double DX0, double DX1, double DX2, int order, int P) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  const int nm[3] = {n0, n1, n2};
  const double DX[3] = {DX0, DX1, DX2};
  int ci[3] = {0, 0, 0}, rem = p;
  for (int k = dim - 1; k >= 0; --k) {
    ci[k] = rem % nm[k];
    rem /= nm[k];
  }
  double out[3] = {0.0, 0.0, 0.0};
  for (int k = 0; k < dim; ++k) {
    // linear index of the point shifted by s along axis k (periodic)
    int stride = 1;
    for (int a = dim - 1; a > k; --a) stride *= nm[a];
    auto at = [&](int s) {
      int i = (ci[k] + s) % nm[k];
      if (i < 0) i += nm[k];
      return p + (i - ci[k]) * stride;
    };
    const double* Fk = F + (size_t)k * 3 * P;
    for (int c = 0; c < 3; ++c) {
      const double* f = Fk + (size_t)c * P;
      double v;
      if (order == 2) v = (f[at(0)] - f[at(-1)]) / DX[k];
      else v = (((f[at(-2)] - 27.0 * f[at(-1)]) + 27.0 * f[at(0)]) - f[at(1)]) / (24.0 * DX[k]);
      out[c] += v;
    }
  }
  for (int c = 0; c < 3; ++c) H[(size_t)c * P + p] = out[c];
}

static inline int nblk(int P) { return (P + 255) / 256; }

cudaError_t launch_flux_divergence(const double* F, double* H, int dim, const int* nmac, const double* DX,
                                   int order, int P, cudaStream_t st) {
  flux_div_kernel<<<nblk(P), 256, 0, st>>>(F, H, dim, nmac[0], dim > 1 ? nmac[1] : 1, dim > 2 ? nmac[2] : 1,
                                           DX[0], dim > 1 ? DX[1] : 1.0, dim > 2 ? DX[2] : 1.0, order, P);
  return cudaGetLastError();
}

cudaError_t launch_h_term(const double* M, const double* H, double alpha, double* h, int P,
                          cudaStream_t st) {
  h_term_kernel<<<nblk(P), 256, 0, st>>>(M, H, alpha, h, P);
  return cudaGetLastError();
}

cudaError_t launch_mpea_update(double* M, const double* H, double* hist, double alpha, double dt,
                               int scheme, int P, cudaStream_t st) {
  // extrapolation coefficients of h^j, h^{j-1}, h^{j-2}: MPE (scheme 1), else MPEA
  const double c0 = scheme == 1 ? 1.5 : 23.0 / 12.0;
  const double c1 = scheme == 1 ? -0.5 : -16.0 / 12.0;
  const double c2 = scheme == 1 ? 0.0 : 5.0 / 12.0;
  mpea_kernel<<<nblk(P), 256, 0, st>>>(M, H, hist, alpha, dt, c0, c1, c2, P);
  return cudaGetLastError();
}

cudaError_t launch_rk4_stage(const double* M, const double* Ms, const double* H, double alpha,
                             double dt, int stage, double* acc, double* Mnext, double* hist0,
                             int P, cudaStream_t st) {
  rk4_stage_kernel<<<nblk(P), 256, 0, st>>>(M, Ms, H, alpha, dt, stage, acc, Mnext, hist0, P);
  return cudaGetLastError();
}

cudaError_t launch_check_finite(const double* x, int n, int* err, cudaStream_t st) {
  check_finite_kernel<<<64, 256, 0, st>>>(x, n, err);
  return cudaGetLastError();
}

}  // namespace hmm

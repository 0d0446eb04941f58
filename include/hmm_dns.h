/*
 * hmm_dns.h -- C ABI of the direct simulation resolving eps: eq. prob
 * (Section 2.1) on a periodic grid fine enough to resolve a^eps, the reference
 * solver of the paper's Section 5 examples (the locally periodic 1D example
 * with 15 grid points per eps, the quasi-periodic 2D example with dx = 1/1500),
 * time-stepped by MPEA.
 *
 * Discretisation (the same stencil as the micro problems of hmm.h, with
 * periodic wrap instead of the Dirichlet ring):
 *  - nodes x_j = j*dx_k along axis k, dx_k = L/n[k], periodic;
 *  - H = sum_k D_s(a_f D_s m) along each axis, D_s the staggered difference of
 *    order 2 (Section 2.3) or 4, a_f = a^eps at the face x_j + (dx_k/2) e_k;
 *  - steps j = 0 and 1 by RK4P (Section 3.1) with normalised stage states,
 *    then MPEA (eqs. h_term, h_mpea, mpe_update): h^j = H^j + alpha m^j x H^j,
 *    h^{j+1/2} = (23 h^j - 16 h^{j-1} + 5 h^{j-2})/12 and the midpoint update
 *    m^{j+1} = m^j + 2/(1+|w|^2) (w x m^j + w x (w x m^j)), w = (dt/2) h^{j+1/2},
 *    which solves (m^{j+1} - m^j)/dt = -(m^j + m^{j+1})/2 x h^{j+1/2} exactly.
 *
 * Two forms, like hmm.h's precision modes:
 *  - HMM_FP64_PLAIN: FP64 state, history and arithmetic;
 *  - HMM_FP32_BATCHED: the state held as an unevaluated sum of two floats per
 *    component (hi + lo, about 48 significant bits), every difference of the
 *    stencil taken on hi and lo separately so that it keeps FP32 relative
 *    accuracy, FP32 arithmetic and history, and the midpoint increment added
 *    to (hi, lo) by an error-free two-sum. The start-up steps run in FP64.
 *
 * Conventions as in hmm.h: a field is G = n[0]*...*n[d-1] points, FP64, SoA
 * (component c of point p at [c*G + p], p the C-order index, last axis
 * fastest); "_dev" pointers are device pointers, "_host" ordinary host memory;
 * the caller owns what it passes; work runs on the stream given at init and
 * every call that returns a result synchronises it; no call throws.
 */
#ifndef HMM_GB300_DNS_H
#define HMM_GB300_DNS_H

#include "hmm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int dim;                      /* d = 1 or 2                                      */
  int n[3];                     /* grid points per axis, 4 <= n[k] <= 2^20, and
                                   G <= 2^31 - 1 (entries >= dim ignored)          */
  double L;                     /* periodic domain [0, L]^d                        */
  double alpha;                 /* damping, 0 <= alpha <= 1                        */
  double dt;                    /* time step; <= 0: dt_safety * s_AB3(alpha) /
                                   omega_max, s_AB3 the stability limit of the AB3
                                   extrapolation on the ray (-alpha + i) R+ and
                                   omega_max = a_max * lambda_s * sum_k 1/dx_k^2,
                                   lambda_s = 4 (order 2) or 49/9 (order 4),
                                   a_max = c0 + sum |amp| (or the table maximum)   */
  double dt_safety;             /* <= 0: 0.5                                       */
  double c0;                    /* a(x) = c0 + sum of terms (as in hmm_params)     */
  int n_terms;                  /* 0..8                                            */
  const hmm_coef_term* terms;   /* host array, copied                              */
  double eps;                   /* eps of the fast variable x/eps                  */
  int stencil_order;            /* 2 or 4; <= 0: 4                                 */
  int precision;                /* hmm_precision (see above)                       */
  int reserved[4];              /* must be zero                                    */
} hmm_dns_params;

/* Validates the parameters (including a > 0 at every face, (A1)), tabulates
 * a^eps at every face (d x G values, FP64 and FP32 copies), picks the time step
 * and allocates the state: 2 state buffers and 3 history buffers of G points
 * (FP64: 24 B per point each; FP32 form: 24 B state, 12 B history) plus 4 FP64
 * start-up buffers.
 * cuda_stream: a cudaStream_t (NULL = the legacy default stream). */
hmm_status hmm_dns_init(const hmm_dns_params* params, void* cuda_stream, void** handle_out);

/* Replaces c0 + terms by tabulated face values, for coefficients that are not
 * sums of separable terms (for example eq. coeff_loc2D). table_host: FP64,
 * n_values = d*G: block k (G values, C order) holds a at x_j + (dx_k/2) e_k.
 * Every value must be positive and finite. The time step is recomputed from the
 * table's maximum when params.dt <= 0, and the stepper restarts (j = 0). */
hmm_status hmm_dns_set_face_table(void* handle, const double* table_host, long long n_values);

/* n_steps >= 0 time steps, in place on M_dev (SoA 3 x G FP64 device buffer).
 * The handle keeps the step count j and the MPEA history between calls, so
 * consecutive calls continue one trajectory when each passes the M the previous
 * call returned. Returns HMM_ERR_NONFINITE if a non-finite value appeared. */
hmm_status hmm_dns_step(void* handle, double* M_dev, int n_steps);

/* As hmm_dns_step with M in host memory (copied in and out once per call). */
hmm_status hmm_dns_step_host(void* handle, double* M_host, int n_steps);

/* Forgets the history: the next step is an RK4P start-up step again (j = 0). */
hmm_status hmm_dns_reset(void* handle);

/* The time step, the step count j and the device time of the last
 * hmm_dns_step call in ms. Any pointer may be NULL. */
hmm_status hmm_dns_info(void* handle, double* dt, long long* j, double* last_ms);

/* The work plan of the time-stepping kernel: warp strips along the fast axis,
 * rows per work item (chunk) and work items. The chunk starts as the longest
 * that keeps every resident warp busy in one wave; the first time step after the
 * RK4P start-up autotunes it (times the kernel for a few chunk lengths on the
 * handle's own grid and keeps the fastest). Any pointer may be NULL. */
hmm_status hmm_dns_plan(void* handle, int* strips, int* chunk, int* items);

/* One-line description of the last failure on this handle ("" if none);
 * NULL handle: the last hmm_dns_init failure. */
const char* hmm_dns_last_error(void* handle);

/* Frees all memory of the handle (synchronises its stream). */
void hmm_dns_destroy(void* handle);

#ifdef __cplusplus
}
#endif
#endif /* HMM_GB300_DNS_H */

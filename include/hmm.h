/*
 * hmm.h -- C ABI of the GB300 library for the heterogeneous multiscale method
 * (HMM) for the Landau-Lifshitz equation with an oscillatory exchange
 * coefficient a^eps (Leitenmaier & Runborg, "Heterogeneous multiscale methods
 * for the Landau-Lifshitz equation").
 *
 * The problem (Section 2.1, eq. prob): on the periodic domain [0, L]^d find M
 * with dM/dt = -M x H - alpha M x (M x H), H = div(a^eps grad M), |M| = 1.
 * HMM (Section 2.2) evolves a coarse macro grid x_i = i*DX with the field model
 * (eq. macro_disc) dM_i/dt = -M_i x H_avg,i - alpha M_i x (M_i x H_avg,i), where
 * H_avg,i comes from a micro problem around x_i (eq. micro) averaged by the
 * kernel-weighted space-time average (Section 2.3, eq. upscaling).
 *
 * Conventions shared by every call:
 *  - A macro field is P = n_macro[0]*...*n_macro[d-1] points, FP64, stored SoA:
 *    component c of point p at [c*P + p]; p is the C-order linear index of the
 *    multi-index (i_1, ..., i_d) with i_d fastest. Both precision modes keep the
 *    macro fields in FP64; only the micro state of HMM_FP32_BATCHED is FP32.
 *  - "_dev" pointers are device pointers on the device that was current at
 *    hmm_init; "_host" pointers are ordinary host memory (pinned or pageable).
 *    The caller owns every buffer it passes; the library never frees or
 *    retains them beyond the call (except host arrays inside hmm_params, which
 *    hmm_init copies).
 *  - All work is enqueued on the stream given to hmm_init, and every call that
 *    returns a result synchronises that stream before returning.
 *  - No call throws. Every call returns an hmm_status; hmm_last_error() gives
 *    a one-line reason for the last failure on a handle.
 *  - A handle is not thread safe: calls on one handle must not overlap.
 */
#ifndef HMM_GB300_H
#define HMM_GB300_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HMM_OK = 0,
  HMM_ERR_INVALID_ARG = 1,     /* a parameter or pointer is out of its domain   */
  HMM_ERR_UNSTABLE_DT = 2,     /* a given time step exceeds the stability bound */
  HMM_ERR_OUT_OF_MEMORY = 3,   /* a device allocation failed                    */
  HMM_ERR_CUDA = 4,            /* a CUDA runtime call failed                    */
  HMM_ERR_TIMEOUT = 5,         /* reserved: the kernels contain no spin waits   */
  HMM_ERR_NONFINITE = 6,       /* a non-finite value or |m| blow-up on device   */
  HMM_ERR_NOT_INITIALISED = 7  /* null or destroyed handle                      */
} hmm_status;

typedef enum {
  HMM_FP64_PLAIN = 0,    /* micro state and arithmetic in FP64                */
  HMM_FP32_BATCHED = 1   /* FP32 perturbation-form micro state, FP64 averages */
} hmm_precision;

/* Time integrator of the micro problems (Section 3.1): HeunP, the paper's choice
 * with artificial damping (Section 3.4), or RK4P, whose stability region holds
 * part of the imaginary axis and which is cheaper per unit of micro time for
 * small micro damping (Section 3.2); or the multi-step midpoint methods MPE and
 * MPEA (eqs. h_mpe, h_mpea, mpe_update: one stencil evaluation per step, after one
 * (MPE) or two (MPEA) RK4P start-up steps), whose time step follows the stability
 * regions of AB2 and AB3 (Section 3.2, eq. mpe_update_ab). MPE and MPEA run on the
 * generic kernels (both precisions). */
typedef enum {
  HMM_HEUNP = 0,
  HMM_RK4P = 1,
  HMM_MICRO_MPE = 2,
  HMM_MICRO_MPEA = 3
} hmm_micro_stepper;

/* Macro time stepper (Section 3.1): MPEA, the extrapolation of eq. h_mpea in the
 * midpoint update of eq. mpe_update, with two RK4P start-up steps; or MPE, the
 * extrapolation of eq. h_mpe (3/2 h^j - 1/2 h^{j-1}) with one RK4P start-up step.
 * Both are second order; the paper prefers MPEA (better stability for low damping,
 * Section 3.2, and third order observed on its 1D example). */
typedef enum {
  HMM_MPEA = 0,
  HMM_MPE = 1
} hmm_macro_stepper;

/* The HMM macro model (Section 2.2). The field model averages H = div(a^eps grad m)
 * over each micro problem (eq. upscaling) and steps eq. macro_disc with it. The
 * flux model (eq. macro_flux) averages the flux a^eps grad m instead: column k of
 * F_avg at the staggered point x_i + (DX_k/2) e_k, from a micro problem centred
 * there (d micro problems per macro point), and steps the macro equation with
 * div F_avg, the staggered difference of order interp_order (2 or 4) of those
 * columns, in place of H_avg. The flux model runs on the generic kernels (both
 * precision forms; kernel_variant 0 or 1) with the separable coefficient terms. */
typedef enum {
  HMM_FIELD_MODEL = 0,
  HMM_FLUX_MODEL = 1
} hmm_model;

/* One term of the material coefficient (Section 2.1 (A1); the examples of
 * Section 2.4 and Section 5 are sums of such terms):
 *     amp * prod_{k<d} g_k(2*pi*omega[k]*s_k + phase[k]),
 * g_k = 1 (kind 0), sin (kind 1) or cos (kind 2); s_k = x_k/eps (scale 0, the
 * fast variable) or s_k = x_k (scale 1, the slow variable). */
typedef struct {
  double amp;
  int kind[3];
  int scale[3];
  double omega[3];
  double phase[3];
} hmm_coef_term;

/* Parameters of one HMM problem (copied by hmm_init). Section references:
 * damping alpha (A2) and the artificial micro damping alpha_micro (Section 2.3,
 * end; Section 4.3); box half-width mu' and averaging half-width mu (eq.
 * upscaling, Section 4.3); micro grid dx = eps/pts_per_eps (Section 4.4);
 * kernel parameters p, q (Definition of K^{p,q}); interpolation order 2k
 * (Section 4.1, eq. Q_k). */
typedef struct {
  int dim;                      /* d = 1, 2 or 3                                   */
  int n_macro[3];               /* macro points per axis (entries >= dim ignored)  */
  double L;                     /* domain length; DX = L/n_macro[k]                */
  double alpha;                 /* macro damping, 0 < alpha <= 1 (A2)              */
  double alpha_micro;           /* micro damping, 0 < alpha_micro <= 4             */
  double dt_macro;              /* macro step; <= 0: 0.06*DX^2/(d*a_max)          */
  double c0;                    /* a(x) = c0 + sum of terms                        */
  int n_terms;                  /* 0..8                                            */
  const hmm_coef_term* terms;   /* host array of n_terms terms                     */
  double eps;                   /* uniform eps (used when eps_field is NULL)       */
  const double* eps_field;      /* host array of P eps_i values, or NULL           */
  int box_n;                    /* micro nodes per axis N, ring included           */
  const int* box_n_field;       /* host array of P values N_i, or NULL             */
  double pts_per_eps;           /* K: micro grid spacing dx = eps_i/K              */
  double mu_over_eps;           /* mu/eps; <= 0: mu = 0.8*mu', mu' = (N-1)dx/2     */
  int micro_steps;              /* M micro time steps (eta = M*dt_micro)           */
  double dt_safety;             /* dt_micro as a fraction of the stepper's stability
                                   limit (eq. Cstab); <= 0: 0.8                    */
  int px, qx, pt, qt;           /* kernel parameters; <= 0: 3, 7, 3, 7             */
  int interp_order;             /* 2k in {2, 4}; <= 0: 4                           */
  int stencil_order;            /* 2 or 4; <= 0: 4                                 */
  int precision;                /* hmm_precision                                   */
  int kernel_variant;           /* HMM_FP32_BATCHED kernel: 0 automatic (the
                                   shared-memory-resident kernels when every box
                                   fits them: d = 2, N up to the 8-CTA cluster
                                   limit (HeunP or RK4P); d = 3, order 4, N <= 32,
                                   HeunP; else the generic arena kernel), 1 generic,
                                   2 resident                                      */
  int micro_stepper;            /* hmm_micro_stepper; with RK4P the automatic kernel
                                   choice takes the resident kernel in 2D and the
                                   generic kernel in 3D; MPE and MPEA take the
                                   generic kernel                                  */
  int model;                    /* hmm_model                                       */
  int macro_stepper;            /* hmm_macro_stepper (0: MPEA, 1: MPE)             */
  int tile_rows;                /* resident 2D kernel, rows per thread tile: 0 the
                                   autotuner chooses (2 or 4 per box size), 2 or 4
                                   fixes it                                        */
} hmm_params;

/* Set-up (host only, plus device allocations on the current device).
 * Validates the parameters: 0 < alpha <= 1, 0 < alpha_micro <= 4, eps > 0,
 * n_macro >= 2k+1 per axis, 2r+2 <= N <= 1024/256/64 for d = 1/2/3, a > 0 at
 * every micro face (checked on the device during each micro batch), and that
 * the averaging box [-mu, mu]^d stays inside the interior (off the Dirichlet
 * ring of width r = 1 or 3). Computes the smoothing kernels, the quadrature
 * weight tables, the micro time step of each box (dt = dt_safety *
 * s_max(alpha_micro) dx^2 / (a_max d lambda_s), s_max the stability limit of the
 * micro stepper on the ray (-alpha_micro + i) R+), sorts the boxes by cost
 * (longest first) and allocates the per-CTA arenas.
 * cuda_stream: a cudaStream_t (NULL = the legacy default stream).
 * On success *handle_out owns all library memory until hmm_destroy. */
hmm_status hmm_init(const hmm_params* params, void* cuda_stream, void** handle_out);

/* The batched micro-problem solve (the hot path): for every macro point x_i,
 * build m_init = Q_[2k](x_i + xi) from M (Section 4.1), time-step the micro
 * problem (eq. micro) with HeunP on [-mu', mu']^d with m - m_init = 0 on the
 * ring (Section 4.2), and reduce H = div(a^eps grad m) by the kernel-weighted
 * average (eq. upscaling) into H_avg,i. M_dev and Havg_dev: SoA 3 x P FP64
 * device buffers; Havg_dev is overwritten. Pure: the macro history is not
 * touched. Returns HMM_ERR_NONFINITE if a micro state blew up.
 * With the flux model, Havg_dev receives div F_avg (see hmm_model). */
hmm_status hmm_micro_batch(void* handle, const double* M_dev, double* Havg_dev);

/* The micro batch on a subset of the macro points (field model): H_avg,i of
 * eq. upscaling for the n_points macro points listed in points_host (a host
 * array of distinct indices in [0, P)), written to Havg_dev at those points; the
 * other entries of Havg_dev are left as they were. The boxes run on the generic
 * persistent kernel of the handle's precision form (the shared-memory-resident
 * kernels' work plans cover whole batches), so the FP64 method and the FP32 form
 * can be sampled on batches too large to solve whole (accuracy checks at full
 * size, timing the FP64 method on a sample). hmm_stats' last_batch_ms is this
 * call's device time. Allocates (and keeps until hmm_destroy) a box table and an
 * arena sized for the largest subset so far. HMM_ERR_INVALID_ARG for a flux-model
 * handle, an index out of range or listed twice. Synchronises the stream. */
hmm_status hmm_micro_batch_points(void* handle, const double* M_dev, double* Havg_dev, const int* points_host,
                                  int n_points);

/* Flux model only: the averaged fluxes themselves. F_dev: d x 3 x P FP64 device
 * buffer; entry [(k*3 + c)*P + p] is component c of column k of F_avg at
 * x_p + (DX_k/2) e_k, averaging a^eps D_s m along axis k over that axis's faces
 * with the spatial kernel at the face positions. HMM_ERR_INVALID_ARG for a
 * field-model handle. */
hmm_status hmm_flux_batch(void* handle, const double* M_dev, double* F_dev);

/* As hmm_micro_batch, with host buffers: copies M_host to the device, runs the
 * batch and copies H_avg back, all on the handle's stream. */
hmm_status hmm_micro_batch_host(void* handle, const double* M_host, double* Havg_host);

/* n_steps macro steps of the field model (eq. macro_disc), in place on M_dev
 * (SoA 3 x P FP64). The start-up steps (j = 0 and 1 for MPEA, j = 0 for MPE) use
 * RK4P (Section 3.1) with one micro batch per stage at the normalised stage
 * state; later steps use MPEA (eqs. h_term, h_mpea, mpe_update) or MPE (eq. h_mpe
 * in place of eq. h_mpea), one micro batch per step, replayed from a CUDA graph
 * captured on first use for this M_dev. */
hmm_status hmm_macro_step(void* handle, double* M_dev, int n_steps);

/* As hmm_macro_step with M in host memory (copied in and out once per call). */
hmm_status hmm_macro_step_host(void* handle, double* M_host, int n_steps);

/* One MPEA (or MPE) macro step of eq. macro_disc taken in n_waves calls, for
 * batches whose micro problems are too many to solve in one call of bounded
 * length. The micro problems are independent (Section 4.4), so the micro batch
 * of the step is split into n_waves contiguous shares of the handle's work list
 * (each launch group's items, longest first, or the generic kernel's box list):
 * call `wave` = 0, 1, ..., n_waves-1 in order with the same M_dev and n_waves.
 * Each call solves its share's micro problems from M_dev (read only) and keeps
 * their H_avg (field model) or flux columns (flux model) in the handle; the call
 * with wave = n_waves-1 then takes the macro update of every point (eqs. h_term,
 * h_mpea or h_mpe, mpe_update; div F_avg first for the flux model) in place on
 * M_dev and advances the step count. The n_waves calls together give the same
 * M_dev and history as hmm_macro_step(handle, M_dev, 1), bit for bit.
 * Needs the multistep history (step count >= 2 for MPEA, >= 1 for MPE: take the
 * RK4P start-up steps with hmm_macro_step first); 1 <= n_waves <= the number of
 * micro problems; HMM_ERR_INVALID_ARG otherwise or when a wave comes out of order.
 * Any other micro-batch or macro-step call on the handle between two waves, and
 * hmm_set_state, abandons the step in progress (M_dev is untouched until the
 * last wave; the next call must be wave 0). Synchronises the library's stream;
 * hmm_stats' last time is the wave's micro batch. This entry point is an addition
 * of this library; the paper solves each macro step's micro problems at once. */
hmm_status hmm_macro_step_wave(void* handle, double* M_dev, int wave, int n_waves);

/* Restart state of the macro stepper: the history hist (2 x 3 x P FP64 device
 * buffer: h^{j-1} then h^{j-2}, eq. h_term; MPE reads only h^{j-1}) and the step
 * count j. The macro field itself is the caller's M. get copies out, set copies in. */
hmm_status hmm_get_state(void* handle, double* hist_dev, long long* j);
hmm_status hmm_set_state(void* handle, const double* hist_dev, long long j);

/* Lattice updates (micro nodes x micro steps, interior nodes only) of one
 * micro batch, and the device time of the last micro batch in ms. */
hmm_status hmm_stats(void* handle, double* lattice_updates_per_batch, double* last_batch_ms);

/* Per-box quantities as the library computed them, host arrays of length P in
 * macro-point order: dt_micro, mu, dx and N. Any pointer may be NULL. */
hmm_status hmm_box_info(void* handle, double* dt, double* mu, double* dx, int* n);

/* Replaces the coefficient of hmm_params (c0 and terms) by tabulated values of
 * a^eps at every staggered face of every micro box, for coefficients that are
 * not sums of separable terms (for example the locally periodic 2D coefficient
 * of Section 5, eq. coeff_loc2D). table_host: FP64 host array, copied. The boxes
 * follow one another in macro-point order; box p holds d blocks of N_p^d values,
 * block k for the faces along axis k: entry idx (the C-order multi-index j of a
 * box node, last axis fastest) is a^eps at x_p + xi_j + (dx/2) e_k, the face
 * between node j and its +1 neighbour along axis k, with xi_j as in hmm_init
 * (entries with j_k = N_p - 1 are not used). n_values: the array length, which
 * must equal sum_p d N_p^d. Every used value must be positive and finite (A1).
 * The micro time step of each box is recomputed from the maximum of its values,
 * and the macro time step from the global maximum when dt_macro <= 0. A macro
 * step graph captured earlier is discarded. Synchronises the handle's stream. */
hmm_status hmm_set_face_table(void* handle, const double* table_host, long long n_values);

/* The macro time step the handle uses. */
hmm_status hmm_macro_dt(void* handle, double* dt_macro);

/* Allocation-free variant of hmm_micro_batch. This entry point is an addition of
 * this library; the paper has no counterpart.
 *
 * It is for callers that must not allocate device memory: code that runs inside
 * a memory allocator's own callbacks (where cudaMalloc would re-enter the
 * allocator), and applications whose device memory is fully reserved up front by
 * another framework's memory pool (so cudaMalloc fails).
 * It takes the problem directly (no handle), runs the same batched FP32 micro
 * solve as hmm_micro_batch with kernel_variant 1, and calls no cudaMalloc,
 * cudaFree or other allocating routine: every buffer it needs (box table,
 * weight tables, work counter, error word, per-CTA arenas) is carved out of one
 * fixed device array of 32 MiB inside the library, reserved on every GPU that
 * loads the library and held until the process exits.
 *
 * Limits: precision must be HMM_FP32_BATCHED; eps_field and box_n_field must be
 * NULL (uniform boxes); micro_steps <= 16384; the box table, weight tables and
 * at least one box's arena must fit in the 32 MiB (else HMM_ERR_INVALID_ARG with
 * the sizes in hmm_last_error(NULL)). Fewer CTAs run than with hmm_init when the
 * arenas of a full grid do not fit, so large batches run slower.
 * M_dev, Havg_dev: SoA 3 x P FP64 device buffers as for hmm_micro_batch;
 * cuda_stream: the stream to run on (NULL = legacy default stream); the call
 * synchronises it before returning. Errors are reported through
 * hmm_last_error(NULL).
 *
 * The call copies host data to the device, reads the error word back and
 * synchronises its stream; on a stream that is being captured it returns
 * HMM_ERR_INVALID_ARG before enqueuing anything, and the capture stays valid.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) once for that device; make that first call before
 * any stream capture begins. All calls share the one array and each call
 * overwrites it: calls that overlap on the GPU (other threads, other streams)
 * race and must be serialised by the caller. hmm_last_error(NULL) is cleared
 * by a successful call. */
hmm_status hmm_micro_batch_noalloc(const hmm_params* params, const double* M_dev, double* Havg_dev,
                                   void* cuda_stream);

/* The resident-plan autotuner's record for this handle: one line per box size
 * N of the batch that more than one resident-kernel instance can hold, with the
 * device time of each candidate (canvas size or box stride, CTAs per cluster)
 * on a sample of that size's boxes and the index of the one kept. hmm_init runs
 * the autotuner when it picks the resident 2D kernel; "" when there was
 * nothing to choose or another kernel runs. The string is owned by the handle
 * and valid until hmm_destroy. NULL handle: "". This entry point is an addition
 * of this library; the paper has no counterpart. */
const char* hmm_plan_report(void* handle);

/* The current device's FP32 fused multiply-add rate in flop/s (an FMA = 2 flops),
 * measured: a kernel that fills every SM runs eight independent FMA chains per
 * thread for a few milliseconds, as scalar FP32 FMAs (packed = 0) or as the paired
 * FP32x2 FMAs that the micro kernels issue (packed = 1), timed with CUDA events on a
 * stream of its own (synchronised before returning). A denominator for the roofline
 * of the FP32 micro kernels, which are bound by instruction issue rather than by
 * memory; the paper has no counterpart. It allocates one float of device memory
 * for the duration of the call. HMM_ERR_INVALID_ARG for a null output or packed not
 * 0/1; HMM_ERR_OUT_OF_MEMORY if that allocation fails; HMM_ERR_CUDA if another CUDA
 * call fails (hmm_last_error(NULL) says which kind). */
hmm_status hmm_fp32_fma_rate(int packed, double* flops_per_s);

/* One-line description of the last failure on this handle ("" if none). Valid
 * until the next call on the handle. NULL handle: the last hmm_init failure. */
const char* hmm_last_error(void* handle);

/* Frees all library memory of the handle (synchronises its stream). */
void hmm_destroy(void* handle);

#ifdef __cplusplus
}
#endif
#endif /* HMM_GB300_H */

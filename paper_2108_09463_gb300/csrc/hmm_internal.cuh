// Internal declarations shared by the library's translation units.
#pragma once
#include <map>
#include <string>
#include <utility>
#include <vector>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <string>
#include <vector>

namespace hmm {

constexpr int kMaxTerms = 8;
constexpr double kPi = 3.141592653589793238462643383279502884;

// Error bits raised by kernels in the device error word.
enum : int { kErrNonFinite = 1, kErrCoefNonPositive = 2, kErrConfig = 4 };

struct TermDev {
  double amp;
  int kind[3];
  int scale[3];
  double omega[3];
  double phase[3];
};

// One micro problem (one macro point). Sorted longest-first in the work queue.
struct BoxDesc {
  int p;        // macro point (C-order linear index)
  int ci[3];    // macro multi-index
  int N;        // micro nodes per axis, Dirichlet ring included
  int wofs;     // offset of this box's spatial weight table (length N)
  double eps;   // eps_i
  double dx;    // micro grid spacing
  double dt;    // micro time step
  double xc[3]; // box centre: x_i, or x_i + (DX_k/2) e_k for a flux box
  int fax;      // flux model: the axis k of the flux column this box averages; -1: field model
};

struct MicroArgs {
  const BoxDesc* boxes;
  int n_boxes;
  int* queue;            // work counter (reset to 0 before each launch)
  int* err;              // error word (bits above)
  const double* M;       // macro field, SoA 3 x P
  double* Havg;          // output, SoA 3 x P
  double* Fout;          // flux model output, d x 3 x P
  int P;
  int nmac[3];
  double DX[3];
  int interp_k;          // k of Q_[2k]
  int msteps;            // M micro steps
  int stepper;           // 0: HeunP, 1: RK4P (generic kernels)
  const double* faces;   // tabulated a^eps at the faces (NULL: c0 + terms), see hmm_set_face_table
  const long long* face_off;   // offset of macro point p's block in faces
  double alpha_micro;
  const double* W64;     // spatial weight tables (per size class)
  const float* W32;
  const double* w64;     // time weights, msteps + 1
  const float* w32;
  const float* om32;     // tail sums Omega_j = sum_{n >= j} w_n, j = 0..msteps + 1
  double c0;
  int n_terms;
  TermDev terms[kMaxTerms];
  char* arena;           // per-CTA scratch
  size_t slot_bytes;
  int nmax;              // largest N of the batch (sizes the arena and tables)
};

// Launchers (one per precision); dim in {1,2,3}, radius in {1,3}.
// Flux model: H_i = sum_k D_k F_k, the staggered difference of order 2 or 4 of
// the flux columns F (d x 3 x P, column k at x_i + (DX_k/2) e_k), periodic.
cudaError_t launch_flux_divergence(const double* F, double* H, int dim, const int* nmac, const double* DX,
                                   int order, int P, cudaStream_t st);
cudaError_t launch_micro_fp64(const MicroArgs& a, int dim, int radius, int grid, int block,
                              size_t smem, cudaStream_t st);
cudaError_t launch_micro_fp32(const MicroArgs& a, int dim, int radius, int grid, int block,
                              size_t smem, cudaStream_t st);
// Per-CTA arena bytes for boxes of up to nmax nodes per axis.
size_t micro_slot_bytes_fp64(int dim, int nmax, int stepper);   // stepper >= 2: MPE(A) history
size_t micro_slot_bytes_fp32(int dim, int nmax, int stepper);
// Dynamic shared memory of the set-up tables.
size_t micro_smem_bytes(int dim, int nmax, int interp_k, int n_terms);
// Set the kernel's dynamic shared-memory limit and return resident CTAs per SM.
cudaError_t prepare_micro_fp64(int dim, int radius, int block, size_t smem, int* ctas_per_sm);
cudaError_t prepare_micro_fp32(int dim, int radius, int block, size_t smem, int* ctas_per_sm);

// Resident 2D FP32 kernel (micro_fp32_2d.cu). The sorted box table is cut into
// work items (first box, box count): packs of small boxes sharing one CTA, or single
// boxes shared by a cluster of cs CTAs; items of one cluster size form a group, run
// as one persistent launch with its own queue counter.
struct Res2dGroup {
  int cs;           // CTAs per cluster (1: packs)
  int variant;      // compiled instance of the kernel
  int first_item;
  int n_items;
  int grid;         // CTAs launched (a multiple of cs), set by res2d_prepare
  int threads;      // threads per CTA
  int aux;          // z-column 3D kernel: row stride of its planes; 0 otherwise
  int N;            // z-column 3D kernel: the group's box size; 0 otherwise
};
struct Res2dPlan {
  std::vector<int2> items;
  std::vector<Res2dGroup> groups;
  size_t smem = 0;  // dynamic shared memory per CTA
  int dim = 2;      // 2: micro_fp32_2d_kernel instances, 3: micro_fp32_3d_kernel instances
};
// False (with the reason) when some box fits no cluster of the portable size.
// pick: per box size N, the (instance, cluster size) to use instead of the
// heuristic's choice (the autotuner's result), or NULL.
// allow_col3: 3D boxes may run on the z-column kernel, which evaluates separable
// coefficient terms in its time loop (false once a face table is set).
// stepper: the micro stepper (0 HeunP, 1 RK4P: 2D only) whose instances serve the boxes;
// tr: the heuristic's rows per thread tile (0: 4).
bool res2d_make_plan(int dim, const BoxDesc* boxes, int n, int R, int interp_k, int n_terms, size_t smem_bytes,
                     Res2dPlan* plan, std::string* why,
                     const std::map<int, std::pair<int, int>>* pick = nullptr, bool allow_col3 = true,
                     int stepper = 0, int tr = 0);
// True when a 3D plan runs any group on the z-column kernel.
bool res3d_plan_uses_col3(const Res2dPlan& plan);
// The (instance, cluster size) pairs that hold a 2D box of N nodes, the
// heuristic's choice first; the canvas size of an instance (0: box stride).
// tr: rows per thread tile (0: the instances of every tile height; the heuristic's
// pick first, which has 4-row tiles)
std::vector<std::pair<int, int>> res2d_candidates(int N, int R, int interp_k, int n_terms, size_t smem_bytes,
                                                  int stepper = 0, int tr = 0);
int res2d_variant_canvas(int vi);
int res2d_variant_rows(int vi);   // rows per thread tile of a 2D instance
cudaError_t res2d_prepare(int radius, Res2dPlan* plan, int num_sms);
int res2d_max_grid(const Res2dPlan& plan);
size_t res2d_slot_bytes(int nmax);
size_t res3d_slot_bytes(int nmax);
cudaError_t res2d_launch(const MicroArgs& a, int radius, const Res2dPlan& plan, const int2* d_items,
                         int* d_queues, cudaStream_t st);

// Macro-side kernels (FP64, pointwise over P points).
cudaError_t launch_h_term(const double* M, const double* H, double alpha, double* h, int P,
                          cudaStream_t st);
// scheme: hmm_macro_stepper (0 MPEA, 1 MPE), which fixes the extrapolation of h^{j+1/2}.
cudaError_t launch_mpea_update(double* M, const double* H, double* hist, double alpha,
                               double dt, int scheme, int P, cudaStream_t st);
// RK4P: k = f(Ms, H); acc += wk*k (acc = 0 when first); Mnext = normalise(M + c*k).
cudaError_t launch_rk4_stage(const double* M, const double* Ms, const double* H, double alpha,
                             double dt, int stage, double* acc, double* Mnext, double* hist0,
                             int P, cudaStream_t st);
cudaError_t launch_check_finite(const double* x, int n, int* err, cudaStream_t st);

// Message returned by hmm_last_error(NULL) (copied into a fixed buffer).
void set_null_handle_error(const char* msg);

// Host-side set-up shared by hmm_init and the allocation-free entry point.
namespace host {
constexpr int kMaxKernelP = 6;
bool kernel_coeffs(int p, int q, bool one_sided, double* out);   // out[p + 1]
double eval_kernel(const double* c, int p, int q, double x);
double eval_kernel0(const double* c, int p, int q, double t);
double heun_limit(double alpha);
// Largest s with |1 + z + z^2/2 + z^3/6 + z^4/24| <= 1 on z = s(-alpha + i) (RK4P).
double rk4_limit(double alpha);
// Largest s with every root of AB2's (k = 2) or AB3's (k = 3) characteristic polynomial
// in the unit disc on z = s(-alpha + i) (MPE, MPEA).
double ab_limit(double alpha, int k);
double micro_dt(double dt_safety, double alpha_micro, double a_max, int dim, int stencil_order, double dx,
                int stepper);
}  // namespace host

}  // namespace hmm

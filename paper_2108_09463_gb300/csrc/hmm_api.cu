// Host side of the C ABI declared in include/hmm.h.
//
// hmm_init validates the problem, builds the smoothing kernels exactly (moment
// conditions of Section 2.3's Definition solved in 128-bit rationals from
// Beta-function moments), the quadrature tables, every box's geometry and
// micro time step (eq. Cstab with the HeunP limit on the eigenvalue ray of
// Section 3.2), sorts boxes longest first, and allocates the per-CTA arenas.
// hmm_micro_batch launches the persistent micro kernel; hmm_macro_step drives
// RK4P start-up steps and graph-captured MPEA steps (Section 3.1).
#include <cuda_runtime.h>

#include <algorithm>
#include <complex>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "../../include/hmm.h"
#include "hmm_internal.cuh"

using namespace hmm;

namespace {

thread_local char g_init_error[512] = "";   // last failure of a call without a handle

// ---------------------------------------------------------------- rationals
struct Rat {
  __int128 n, d;  // d > 0, gcd(n, d) = 1
};

__int128 gcd128(__int128 a, __int128 b) {
  if (a < 0) a = -a;
  if (b < 0) b = -b;
  while (b != 0) {
    __int128 t = a % b;
    a = b;
    b = t;
  }
  return a;
}

bool rat_make(__int128 n, __int128 d, Rat* r) {
  if (d == 0) return false;
  if (d < 0) { n = -n; d = -d; }
  __int128 g = gcd128(n, d);
  if (g == 0) g = 1;
  r->n = n / g;
  r->d = d / g;
  return true;
}

bool mul128(__int128 a, __int128 b, __int128* out) { return !__builtin_mul_overflow(a, b, out); }

bool rat_mul(const Rat& a, const Rat& b, Rat* r) {
  // cross-reduce first to keep the numbers small
  __int128 g1 = gcd128(a.n, b.d), g2 = gcd128(b.n, a.d);
  if (g1 == 0) g1 = 1;
  if (g2 == 0) g2 = 1;
  __int128 n, d;
  if (!mul128(a.n / g1, b.n / g2, &n) || !mul128(a.d / g2, b.d / g1, &d)) return false;
  return rat_make(n, d, r);
}

bool rat_add(const Rat& a, const Rat& b, Rat* r) {
  __int128 g = gcd128(a.d, b.d);
  __int128 x, y, d;
  if (!mul128(a.n, b.d / g, &x) || !mul128(b.n, a.d / g, &y) || !mul128(a.d / g, b.d, &d)) return false;
  __int128 n;
  if (__builtin_add_overflow(x, y, &n)) return false;
  return rat_make(n, d, r);
}

bool rat_div(const Rat& a, const Rat& b, Rat* r) {
  if (b.n == 0) return false;
  Rat inv;
  if (!rat_make(b.d, b.n, &inv)) return false;
  return rat_mul(a, inv, r);
}

long double rat_ld(const Rat& a) { return (long double)a.n / (long double)a.d; }

// Beta-function moments as exact rationals.
//  two-sided: int_{-1}^{1} (1-x^2)^{q+1} x^n dx = B((n+1)/2, q+2) for even n (0 for odd n)
//             = (q+1)! 2^{q+2} / prod_{i=0}^{q+1} (n+1+2i)
//  one-sided: int_0^1 t^{q+1+n} (1-t)^{q+1} dt = B(q+2+n, q+2) = (q+1+n)! (q+1)! / (2q+3+n)!
bool moment_two_sided(int q, int n, Rat* r) {
  if (n % 2) return rat_make(0, 1, r);
  Rat acc;
  rat_make(1, 1, &acc);
  for (int i = 1; i <= q + 1; ++i) {
    Rat f;
    rat_make(i, 1, &f);
    if (!rat_mul(acc, f, &acc)) return false;
  }
  for (int i = 0; i <= q + 1; ++i) {
    Rat f;
    rat_make(2, n + 1 + 2 * i, &f);
    if (!rat_mul(acc, f, &acc)) return false;
  }
  *r = acc;
  return true;
}

bool moment_one_sided(int q, int n, Rat* r) {
  Rat acc;
  rat_make(1, 1, &acc);
  // (q+1+n)! (q+1)! / (2q+3+n)! = (q+1)! / prod_{i=q+2+n}^{2q+3+n} i
  for (int i = 1; i <= q + 1; ++i) {
    Rat f;
    rat_make(i, 1, &f);
    if (!rat_mul(acc, f, &acc)) return false;
  }
  for (int i = q + 2 + n; i <= 2 * q + 3 + n; ++i) {
    Rat f;
    rat_make(1, i, &f);
    if (!rat_mul(acc, f, &acc)) return false;
  }
  *r = acc;
  return true;
}

}  // namespace

namespace hmm {
namespace host {

// Solve sum_k c_k mom(k + r) = delta_{r0}, r = 0..p, in exact rationals (p <= kMaxKernelP).
bool kernel_coeffs(int p, int q, bool one_sided, double* out) {
  if (p < 0 || p > kMaxKernelP) return false;
  const int n = p + 1;
  Rat A[kMaxKernelP + 1][kMaxKernelP + 2];
  for (int r = 0; r < n; ++r) {
    for (int k = 0; k < n; ++k) {
      bool ok = one_sided ? moment_one_sided(q, k + r, &A[r][k]) : moment_two_sided(q, k + r, &A[r][k]);
      if (!ok) return false;
    }
    rat_make(r == 0 ? 1 : 0, 1, &A[r][n]);
  }
  for (int col = 0; col < n; ++col) {
    int piv = -1;
    for (int r = col; r < n; ++r)
      if (A[r][col].n != 0) { piv = r; break; }
    if (piv < 0) return false;
    if (piv != col)
      for (int c = 0; c <= n; ++c) std::swap(A[col][c], A[piv][c]);
    for (int r = 0; r < n; ++r) {
      if (r == col || A[r][col].n == 0) continue;
      Rat fac;
      if (!rat_div(A[r][col], A[col][col], &fac)) return false;
      for (int c = col; c <= n; ++c) {
        Rat t;
        if (!rat_mul(fac, A[col][c], &t)) return false;
        t.n = -t.n;
        if (!rat_add(A[r][c], t, &A[r][c])) return false;
      }
    }
  }
  for (int i = 0; i < n; ++i) {
    Rat c;
    if (!rat_div(A[i][n], A[i][i], &c)) return false;
    out[i] = (double)rat_ld(c);
  }
  return true;
}

double eval_kernel(const double* c, int p, int q, double x) {  // K, support (-1, 1)
  if (!(std::fabs(x) < 1.0)) return 0.0;
  double poly = 0.0;
  for (int k = p; k >= 0; --k) poly = poly * x + c[k];
  return std::pow(1.0 - x * x, q + 1) * poly;
}

double eval_kernel0(const double* c, int p, int q, double t) {  // K0, support (0, 1)
  if (!(t > 0.0 && t < 1.0)) return 0.0;
  double poly = 0.0;
  for (int k = p; k >= 0; --k) poly = poly * t + c[k];
  return std::pow(t * (1.0 - t), q + 1) * poly;
}

// Largest s with |1 + z + z^2/2| <= 1 on z = s(-alpha + i): |R|^2 - 1 = s g(s) with
// g(s) = (1+a^2)^2/4 s^3 - a(1+a^2) s^2 + 2 a^2 s - 2a; its smallest positive root.
double heun_limit(double a) {
  auto g = [a](double s) {
    const double b = 1.0 + a * a;
    return ((0.25 * b * b * s - a * b) * s + 2.0 * a * a) * s - 2.0 * a;
  };
  double lo = 0.0, hi = 1e-3;
  while (g(hi) < 0.0) {
    lo = hi;
    hi += 1e-3;
    if (hi > 20.0) return 0.0;
  }
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (g(mid) < 0.0) lo = mid; else hi = mid;
  }
  return lo;
}

double rk4_limit(double a) {
  // scan outward from s = 0 for the first exit from the unit disc, then bisect
  auto amp = [a](double s) {
    const std::complex<double> z = s * std::complex<double>(-a, 1.0);
    return std::abs(1.0 + z * (1.0 + z * (0.5 + z * (1.0 / 6.0 + z / 24.0))));
  };
  double lo = 0.0, hi = 1e-3;
  while (amp(hi) <= 1.0) {
    lo = hi;
    hi += 1e-3;
    if (hi > 20.0) return 0.0;
  }
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (amp(mid) <= 1.0) lo = mid; else hi = mid;
  }
  return lo;
}

// Largest root modulus of the characteristic polynomial rho(zeta) - z sigma(zeta) of
// AB2 (k = 2) or AB3 (k = 3), the methods Section 3.2 relates MPE and MPEA to
// (eq. mpe_update_ab): zeta^2 - (1 + 3z/2) zeta + z/2 and
// zeta^3 - (1 + 23z/12) zeta^2 + (16z/12) zeta - 5z/12; roots by Durand-Kerner.
double ab_growth(std::complex<double> z, int k) {
  using C = std::complex<double>;
  C c[4];   // monic, c[0] zeta^k + c[1] zeta^(k-1) + ...
  if (k == 2) {
    c[0] = 1.0; c[1] = -(1.0 + 1.5 * z); c[2] = 0.5 * z;
  } else {
    c[0] = 1.0; c[1] = -(1.0 + (23.0 / 12.0) * z); c[2] = (16.0 / 12.0) * z; c[3] = -(5.0 / 12.0) * z;
  }
  auto P = [&](C x) {
    C v = c[0];
    for (int i = 1; i <= k; ++i) v = v * x + c[i];
    return v;
  };
  C r[3];
  for (int i = 0; i < k; ++i) r[i] = std::pow(C(0.4, 0.9), i);
  for (int it = 0; it < 500; ++it) {
    for (int i = 0; i < k; ++i) {
      C den = 1.0;
      for (int j = 0; j < k; ++j)
        if (j != i) den *= r[i] - r[j];
      r[i] -= P(r[i]) / den;
    }
  }
  double g = 0.0;
  for (int i = 0; i < k; ++i) g = std::max(g, std::abs(r[i]));
  return g;
}

double ab_limit(double a, int k) {
  const std::complex<double> ray(-a, 1.0);
  double lo = 0.0, hi = 1e-3;
  while (ab_growth(hi * ray, k) <= 1.0) {
    lo = hi;
    hi += 1e-3;
    if (hi > 20.0) return 0.0;
  }
  for (int it = 0; it < 100; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (ab_growth(mid * ray, k) <= 1.0) lo = mid; else hi = mid;
  }
  return lo;
}

double stepper_limit(double alpha_micro, int stepper) {
  switch (stepper) {
    case HMM_RK4P: return rk4_limit(alpha_micro);
    case HMM_MICRO_MPE: return ab_limit(alpha_micro, 2);
    case HMM_MICRO_MPEA: return ab_limit(alpha_micro, 3);
    default: return heun_limit(alpha_micro);
  }
}

double micro_dt(double dt_safety, double alpha_micro, double a_max, int dim, int stencil_order, double dx,
                int stepper) {
  const double lam = stencil_order == 2 ? 4.0 : (28.0 / 12.0) * (28.0 / 12.0);
  const double omega = a_max * dim * lam / (dx * dx);
  return dt_safety * stepper_limit(alpha_micro, stepper) / omega;
}

}  // namespace host

void set_null_handle_error(const char* msg) {
  std::snprintf(g_init_error, sizeof g_init_error, "%s", msg);
}

}  // namespace hmm

namespace {

constexpr double kMacroDtConstant = 0.06;
constexpr int kQueues = 32;           // queue counters (one per resident-kernel launch group)

}  // namespace

// ---------------------------------------------------------------- handle
struct HmmHandle {
  hmm_params p{};
  std::vector<hmm_coef_term> terms;
  std::vector<double> eps_field;
  std::vector<int> n_field;
  int dim = 0, P = 0, nmac[3] = {1, 1, 1};
  double DX[3] = {0, 0, 0};
  int radius = 3, interp_k = 2;
  double a_max = 0;
  cudaStream_t user_stream = nullptr;  // the caller's stream (may be the legacy stream)
  cudaStream_t stream = nullptr;       // the library's own non-blocking stream
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  int device = 0, num_sms = 0;
  // host copies
  std::vector<BoxDesc> boxes;      // sorted longest first
  std::vector<double> box_dt, box_mu, box_dx;
  std::vector<int> box_n;
  double lu_per_batch = 0;
  int nmax = 0;
  double dt_macro = 0;
  // device
  BoxDesc* d_boxes = nullptr;
  int nb = 0;                      // boxes: P (field model) or d P (flux model)
  std::string plan_report;         // the resident-plan autotuner's timings
  double* d_F = nullptr;           // flux model: F_avg, d x 3 x P
  double* d_W64 = nullptr;
  float* d_W32 = nullptr;
  double* d_w64 = nullptr;
  float* d_w32 = nullptr;
  float* d_om32 = nullptr;
  char* d_arena = nullptr;
  size_t slot_bytes = 0;
  int grid = 0, block = 256;
  size_t smem = 0;
  bool res2d = false;        // resident 2D FP32 kernel
  Res2dPlan plan;            // its work items and launches
  int2* d_items = nullptr;
  double* d_faces = nullptr;      // tabulated face coefficients (hmm_set_face_table)
  long long* d_face_off = nullptr;
  int* d_queue = nullptr;
  int* d_err = nullptr;
  int* h_err = nullptr;      // pinned
  double* d_H = nullptr;     // 3P
  double* d_hist = nullptr;  // 2 x 3P
  double* d_acc = nullptr;   // 3P (RK4 accumulator)
  double* d_stage = nullptr; // 3P (RK4 stage state)
  double* d_Mhost = nullptr; // 3P (host-buffer entry points)
  double* d_Hhost = nullptr; // 3P
  long long j = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  double last_ms = 0;
  cudaGraphExec_t graph = nullptr;
  const double* graph_M = nullptr;
  // hmm_macro_step_wave: the next wave expected, the wave count and M of the macro
  // step in progress (wave_next = 0: none)
  int wave_next = 0, wave_n = 0;
  const double* wave_M = nullptr;
  std::string err;
  MicroArgs args{};
  // hmm_micro_batch_points: box table and generic-kernel arena of the last subset
  std::vector<int> box_of_point;   // index into boxes of macro point p's box (field model)
  BoxDesc* d_sub_boxes = nullptr;
  int sub_cap = 0;
  char* d_sub_arena = nullptr;
  size_t sub_arena_bytes = 0;
};

namespace {

hmm_status fail(HmmHandle* h, hmm_status s, const std::string& msg) {
  if (h) h->err = msg; else hmm::set_null_handle_error(msg.c_str());
  return s;
}

hmm_status cuda_fail(HmmHandle* h, cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorString(e);
  return fail(h, e == cudaErrorMemoryAllocation ? HMM_ERR_OUT_OF_MEMORY : HMM_ERR_CUDA, m);
}

#define HMM_CUDA(h, call)                                    \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return cuda_fail((h), e_, #call); \
  } while (0)

void free_all(HmmHandle* h) {
  if (h->graph) cudaGraphExecDestroy(h->graph);
  void* ptrs[] = {h->d_boxes, h->d_F, h->d_W64, h->d_W32, h->d_w64, h->d_w32, h->d_om32, h->d_arena, h->d_queue, h->d_items, h->d_faces, h->d_face_off,
                  h->d_err, h->d_H, h->d_hist, h->d_acc, h->d_stage, h->d_Mhost, h->d_Hhost,
                  h->d_sub_boxes, h->d_sub_arena};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (h->h_err) cudaFreeHost(h->h_err);
  if (h->ev0) cudaEventDestroy(h->ev0);
  if (h->ev1) cudaEventDestroy(h->ev1);
  if (h->ev_in) cudaEventDestroy(h->ev_in);
  if (h->ev_out) cudaEventDestroy(h->ev_out);
  if (h->stream) cudaStreamDestroy(h->stream);
}

int max_n_for_dim(int d) { return d == 1 ? 1024 : (d == 2 ? 256 : 64); }

// Autotuner of the resident 2D plan. For every box size of the batch with more
// than one kernel instance that holds it (compile-time canvases, the box-stride
// instance, cluster sizes), the micro kernel is timed for each candidate on a
// sample of that size's boxes (up to 8 per SM): a constant macro field, the
// first min(M, 32) micro steps, one warm-up and two timed launches; the fastest
// candidate is kept and the real plan is rebuilt with it. The results are kept
// as text (hmm_plan_report).
hmm_status tune_resident_plan(HmmHandle* h) {
  const int R = h->radius, k = h->interp_k, nt = h->p.n_terms;
  const size_t smem = h->plan.smem;
  std::map<int, std::pair<int, int>> pick;
  std::string report;
  double* d_M = nullptr;
  double* d_out = nullptr;
  BoxDesc* d_sb = nullptr;
  int2* d_it = nullptr;
  char* d_ar = nullptr;
  size_t ar_bytes = 0;
  auto release = [&]() {
    void* ptrs[] = {d_M, d_out, d_sb, d_it, d_ar};
    for (void* q : ptrs)
      if (q) cudaFree(q);
  };
  auto tune = [&]() -> hmm_status {
    const size_t f3 = sizeof(double) * 3 * (size_t)h->P;
    HMM_CUDA(h, cudaMalloc(&d_M, f3));
    HMM_CUDA(h, cudaMalloc(&d_out, f3 * h->dim));
    {
      std::vector<double> mz(3 * (size_t)h->P, 0.0);
      for (int q = 0; q < h->P; ++q) mz[2 * (size_t)h->P + q] = 1.0;   // M = e_z
      HMM_CUDA(h, cudaMemcpy(d_M, mz.data(), f3, cudaMemcpyHostToDevice));
    }
    const int cap_sample = 8 * h->num_sms;
    HMM_CUDA(h, cudaMalloc(&d_sb, sizeof(BoxDesc) * cap_sample));
    HMM_CUDA(h, cudaMalloc(&d_it, sizeof(int2) * cap_sample));
    int lo = 0;
    while (lo < h->nb) {
      const int N = h->boxes[lo].N;
      int hi = lo;
      while (hi < h->nb && h->boxes[hi].N == N) ++hi;
      const int count = hi - lo;
      const auto cand = res2d_candidates(N, R, k, nt, smem, h->p.micro_stepper, h->p.tile_rows);
      lo = hi;
      if (cand.size() < 2) continue;
      const int ns = std::min(count, cap_sample);
      HMM_CUDA(h, cudaMemcpy(d_sb, h->boxes.data() + (hi - count), sizeof(BoxDesc) * ns, cudaMemcpyHostToDevice));
      float best_ms = 1e30f;
      int best = 0;
      std::string line = "N=" + std::to_string(N) + ":";
      for (size_t c = 0; c < cand.size(); ++c) {
        std::map<int, std::pair<int, int>> one{{N, cand[c]}};
        Res2dPlan pl;
        std::string why;
        if (!res2d_make_plan(h->dim, h->boxes.data() + (hi - count), ns, R, k, nt, smem, &pl, &why, &one, true,
                             h->p.micro_stepper, h->p.tile_rows))
          continue;
        if ((int)pl.groups.size() > kQueues) continue;
        if (res2d_prepare(R, &pl, h->num_sms) != cudaSuccess) {
          cudaGetLastError();
          continue;
        }
        const size_t need = h->slot_bytes * (size_t)res2d_max_grid(pl);
        if (need > ar_bytes) {
          if (d_ar) cudaFree(d_ar);
          d_ar = nullptr;
          HMM_CUDA(h, cudaMalloc(&d_ar, need));
          ar_bytes = need;
        }
        HMM_CUDA(h, cudaMemcpy(d_it, pl.items.data(), sizeof(int2) * pl.items.size(), cudaMemcpyHostToDevice));
        MicroArgs a = h->args;
        a.boxes = d_sb;
        a.n_boxes = ns;
        a.M = d_M;
        a.Havg = d_out;
        a.Fout = d_out;
        a.msteps = std::min(h->args.msteps, 32);
        a.arena = d_ar;
        float ms = 0;
        for (int r = 0; r < 3; ++r) {
          HMM_CUDA(h, cudaMemsetAsync(h->d_queue, 0, sizeof(int) * kQueues, h->stream));
          if (r == 1) HMM_CUDA(h, cudaEventRecord(h->ev0, h->stream));
          HMM_CUDA(h, res2d_launch(a, R, pl, d_it, h->d_queue, h->stream));
        }
        HMM_CUDA(h, cudaEventRecord(h->ev1, h->stream));
        HMM_CUDA(h, cudaEventSynchronize(h->ev1));
        HMM_CUDA(h, cudaEventElapsedTime(&ms, h->ev0, h->ev1));
        char buf[96];
        snprintf(buf, sizeof buf, " %s%d x%d tr%d %.3f ms", res2d_variant_canvas(cand[c].first) ? "canvas " : "stride ",
                 res2d_variant_canvas(cand[c].first), cand[c].second, res2d_variant_rows(cand[c].first), ms / 2);
        line += buf;
        if (ms < best_ms) {
          best_ms = ms;
          best = (int)c;
        }
      }
      if (best_ms < 1e30f) {
        pick[N] = cand[best];
        line += " -> " + std::to_string(best + 1) + "\n";
        report += line;
      }
    }
    HMM_CUDA(h, cudaMemset(h->d_err, 0, sizeof(int)));
    if (pick.empty()) return HMM_OK;
    // the real plan with the tuned instances
    Res2dPlan pl;
    std::string why;
    if (!res2d_make_plan(h->dim, h->boxes.data(), h->nb, R, k, nt, smem, &pl, &why, &pick, true, h->p.micro_stepper,
                         h->p.tile_rows) ||
        (int)pl.groups.size() > kQueues || res2d_prepare(R, &pl, h->num_sms) != cudaSuccess) {
      cudaGetLastError();
      return HMM_OK;                // keep the heuristic plan
    }
    const int grid = res2d_max_grid(pl);
    if (grid > h->grid) {
      char* ar = nullptr;
      HMM_CUDA(h, cudaMalloc(&ar, h->slot_bytes * (size_t)grid));
      cudaFree(h->d_arena);
      h->d_arena = ar;
      h->args.arena = ar;
      h->grid = grid;
    }
    int2* it = nullptr;
    HMM_CUDA(h, cudaMalloc(&it, sizeof(int2) * pl.items.size()));
    const cudaError_t e = cudaMemcpy(it, pl.items.data(), sizeof(int2) * pl.items.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      cudaFree(it);
      return cuda_fail(h, e, "cudaMemcpy(tuned work items)");
    }
    cudaFree(h->d_items);
    h->d_items = it;
    h->plan = pl;
    return HMM_OK;
  };
  const hmm_status st = tune();
  release();
  h->plan_report = report;
  return st;
}

hmm_status build(HmmHandle* h) {
  hmm_params& p = h->p;
  if (p.dim < 1 || p.dim > 3) return fail(h, HMM_ERR_INVALID_ARG, "dim must be 1, 2 or 3");
  if (p.tile_rows != 0 && p.tile_rows != 2 && p.tile_rows != 4)
    return fail(h, HMM_ERR_INVALID_ARG, "tile_rows must be 0 (tuned), 2 or 4");
  if (p.macro_stepper != HMM_MPEA && p.macro_stepper != HMM_MPE)
    return fail(h, HMM_ERR_INVALID_ARG, "macro_stepper must be 0 (MPEA) or 1 (MPE)");
  if (p.model != HMM_FIELD_MODEL && p.model != HMM_FLUX_MODEL)
    return fail(h, HMM_ERR_INVALID_ARG, "model must be 0 (field) or 1 (flux)");

  if (p.micro_stepper < HMM_HEUNP || p.micro_stepper > HMM_MICRO_MPEA)
    return fail(h, HMM_ERR_INVALID_ARG, "micro_stepper must be 0 (HeunP), 1 (RK4P), 2 (MPE) or 3 (MPEA)");
  h->dim = p.dim;
  if (!(p.L > 0)) p.L = 1.0;
  if (p.px <= 0) p.px = 3;
  if (p.qx <= 0) p.qx = 7;
  if (p.pt <= 0) p.pt = 3;
  if (p.qt <= 0) p.qt = 7;
  if (p.interp_order <= 0) p.interp_order = 4;
  if (p.stencil_order <= 0) p.stencil_order = 4;
  if (!(p.dt_safety > 0)) p.dt_safety = 0.8;
  if (p.interp_order != 2 && p.interp_order != 4)
    return fail(h, HMM_ERR_INVALID_ARG, "interp_order must be 2 or 4");
  if (p.stencil_order != 2 && p.stencil_order != 4)
    return fail(h, HMM_ERR_INVALID_ARG, "stencil_order must be 2 or 4");
  if (p.precision != HMM_FP64_PLAIN && p.precision != HMM_FP32_BATCHED)
    return fail(h, HMM_ERR_INVALID_ARG, "precision must be HMM_FP64_PLAIN or HMM_FP32_BATCHED");
  if (p.kernel_variant < 0 || p.kernel_variant > 2)
    return fail(h, HMM_ERR_INVALID_ARG, "kernel_variant must be 0, 1 or 2");
  if (!(p.alpha > 0 && p.alpha <= 1)) return fail(h, HMM_ERR_INVALID_ARG, "alpha must be in (0, 1] (A2)");
  if (!(p.alpha_micro > 0 && p.alpha_micro <= 4))
    return fail(h, HMM_ERR_INVALID_ARG, "alpha_micro must be in (0, 4]");
  if (p.n_terms < 0 || p.n_terms > kMaxTerms) return fail(h, HMM_ERR_INVALID_ARG, "n_terms must be 0..8");
  if (p.n_terms > 0 && !p.terms) return fail(h, HMM_ERR_INVALID_ARG, "terms is NULL");
  if (!(p.pts_per_eps > 0)) return fail(h, HMM_ERR_INVALID_ARG, "pts_per_eps must be > 0");
  if (p.micro_steps < 1 || p.micro_steps > 1000000) return fail(h, HMM_ERR_INVALID_ARG, "micro_steps out of range");
  if (p.px > 6 || p.pt > 6 || p.qx > 12 || p.qt > 12)
    return fail(h, HMM_ERR_INVALID_ARG, "kernel parameters must satisfy p <= 6, q <= 12");
  h->radius = p.stencil_order == 2 ? 1 : 3;
  h->interp_k = p.interp_order / 2;
  long long P = 1;
  for (int k = 0; k < h->dim; ++k) {
    if (p.n_macro[k] < 2 * h->interp_k + 1)
      return fail(h, HMM_ERR_INVALID_ARG, "n_macro must be >= interp_order + 1 on every axis");
    h->nmac[k] = p.n_macro[k];
    h->DX[k] = p.L / p.n_macro[k];
    P *= p.n_macro[k];
  }
  if (P > (1LL << 30)) return fail(h, HMM_ERR_INVALID_ARG, "too many macro points");
  h->P = (int)P;
  h->terms.assign(p.terms, p.terms + p.n_terms);
  for (const auto& t : h->terms)
    for (int k = 0; k < 3; ++k) {
      if (t.kind[k] < 0 || t.kind[k] > 2 || t.scale[k] < 0 || t.scale[k] > 1)
        return fail(h, HMM_ERR_INVALID_ARG, "coefficient term kind/scale out of range");
      if (k >= h->dim && t.kind[k] != 0)
        return fail(h, HMM_ERR_INVALID_ARG, "coefficient factor on an axis beyond dim");
    }
  p.terms = nullptr;
  if (p.eps_field) h->eps_field.assign(p.eps_field, p.eps_field + h->P);
  if (p.box_n_field) h->n_field.assign(p.box_n_field, p.box_n_field + h->P);
  p.eps_field = nullptr;
  p.box_n_field = nullptr;
  h->a_max = p.c0;
  for (const auto& t : h->terms) h->a_max += std::fabs(t.amp);
  if (!(h->a_max > 0)) return fail(h, HMM_ERR_INVALID_ARG, "coefficient upper bound must be positive");

  // Smoothing kernels (exact rationals).
  double cK[host::kMaxKernelP + 1], cK0[host::kMaxKernelP + 1];
  if (!host::kernel_coeffs(p.px, p.qx, false, cK) || !host::kernel_coeffs(p.pt, p.qt, true, cK0))
    return fail(h, HMM_ERR_INVALID_ARG, "kernel moment system overflowed 128-bit rationals");

  // Time weights w_n = K0(n/M), normalised to sum 1.
  const int M = p.micro_steps;
  std::vector<double> w(M + 1);
  double ws = 0;
  for (int n = 0; n <= M; ++n) ws += (w[n] = host::eval_kernel0(cK0, p.pt, p.qt, (double)n / (double)M));
  if (!(ws != 0)) return fail(h, HMM_ERR_INVALID_ARG, "time weights vanish");
  for (auto& v : w) v /= ws;

  // Boxes.

  // Field model: one box per macro point. Flux model: one box per macro point
  // and axis k, centred at x_i + (DX_k/2) e_k (the staggered point of column k).
  const bool flux = p.model == HMM_FLUX_MODEL;
  const int naxes = flux ? h->dim : 1;
  h->nb = h->P * naxes;
  const int nlim = max_n_for_dim(h->dim);
  std::map<int, int> class_ofs;
  std::vector<double> W64;
  h->boxes.resize(h->nb);
  h->box_dt.resize(h->P);
  h->box_mu.resize(h->P);
  h->box_dx.resize(h->P);
  h->box_n.resize(h->P);
  h->nmax = 0;
  h->lu_per_batch = 0;
  for (int bi = 0; bi < h->nb; ++bi) {
    const int pi = bi % h->P;
    BoxDesc bd{};
    bd.p = pi;
    bd.fax = flux ? bi / h->P : -1;
    int rem = pi;
    for (int k = h->dim - 1; k >= 0; --k) {
      bd.ci[k] = rem % h->nmac[k];
      rem /= h->nmac[k];
    }
    for (int k = 0; k < h->dim; ++k) bd.xc[k] = bd.ci[k] * h->DX[k] + (k == bd.fax ? 0.5 * h->DX[k] : 0.0);
    bd.eps = h->eps_field.empty() ? p.eps : h->eps_field[pi];
    bd.N = h->n_field.empty() ? p.box_n : h->n_field[pi];
    if (!(bd.eps > 0)) return fail(h, HMM_ERR_INVALID_ARG, "eps must be > 0");
    if (bd.N < 2 * h->radius + 2 || bd.N > nlim)
      return fail(h, HMM_ERR_INVALID_ARG, "box_n out of range for this dimension and stencil");
    bd.dx = bd.eps / p.pts_per_eps;
    const double mup = (bd.N - 1) * bd.dx / 2.0;
    const double mu = p.mu_over_eps > 0 ? p.mu_over_eps * bd.eps : 0.8 * mup;
    bd.dt = host::micro_dt(p.dt_safety, p.alpha_micro, h->a_max, h->dim, p.stencil_order, bd.dx, p.micro_stepper);
    if (!(bd.dt > 0)) return fail(h, HMM_ERR_INVALID_ARG, "micro time step is not positive");
    auto it = class_ofs.find(bd.N);
    if (it == class_ofs.end()) {
      // spatial weights W_j = K(xi_j/mu), normalised; xi_j = (j - (N-1)/2) dx
      const int ofs = (int)W64.size();
      double s = 0;
      for (int jn = 0; jn < bd.N; ++jn) {
        const double xi = (jn - (bd.N - 1) / 2.0) * bd.dx;
        const double v = host::eval_kernel(cK, p.px, p.qx, xi / mu);
        W64.push_back(v);
        s += v;
      }
      if (!(s != 0)) return fail(h, HMM_ERR_INVALID_ARG, "spatial weights vanish (mu too small)");
      for (int jn = 0; jn < bd.N; ++jn) W64[ofs + jn] /= s;
      for (int jn = 0; jn < h->radius; ++jn)
        if (W64[ofs + jn] != 0.0 || W64[ofs + bd.N - 1 - jn] != 0.0)
          return fail(h, HMM_ERR_INVALID_ARG, "averaging box [-mu, mu] reaches the Dirichlet ring");
      if (flux) {
        // the flux model's face weights K(xi_f/mu), xi_f = xi_j + dx/2, j = 0..N-2,
        // normalised (entry N-1 unused); with the ring off the averaging box only
        // faces that touch an interior node carry weight
        double sf = 0;
        for (int jn = 0; jn < bd.N; ++jn) {
          const double xf = (jn + 0.5 - (bd.N - 1) / 2.0) * bd.dx;
          const double v = jn < bd.N - 1 ? host::eval_kernel(cK, p.px, p.qx, xf / mu) : 0.0;
          W64.push_back(v);
          sf += v;
        }
        if (!(sf != 0)) return fail(h, HMM_ERR_INVALID_ARG, "face weights vanish (mu too small)");
        for (int jn = 0; jn < bd.N; ++jn) W64[ofs + bd.N + jn] /= sf;
      }
      it = class_ofs.emplace(bd.N, ofs).first;
    }
    bd.wofs = it->second;
    h->boxes[bi] = bd;
    h->box_dt[pi] = bd.dt;
    h->box_mu[pi] = mu;
    h->box_dx[pi] = bd.dx;
    h->box_n[pi] = bd.N;
    h->nmax = std::max(h->nmax, bd.N);
    double lu = M;
    for (int k = 0; k < h->dim; ++k) lu *= (bd.N - 2 * h->radius);
    h->lu_per_batch += lu;
  }
  std::stable_sort(h->boxes.begin(), h->boxes.end(),
                   [](const BoxDesc& x, const BoxDesc& y) { return x.N > y.N; });
  if (p.dt_macro > 0) {
    h->dt_macro = p.dt_macro;
  } else {
    double dX = h->DX[0];
    for (int k = 1; k < h->dim; ++k) dX = std::min(dX, h->DX[k]);
    h->dt_macro = kMacroDtConstant * dX * dX / (h->dim * h->a_max);
  }

  // Device side.
  HMM_CUDA(h, cudaGetDevice(&h->device));
  HMM_CUDA(h, cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device));
  std::vector<float> W32(W64.begin(), W64.end()), w32(w.begin(), w.end());
  std::vector<float> om32(w.size() + 1, 0.f);   // Omega_j = sum_{n >= j} w_n (suffix sums in FP64)
  {
    double tail = 0.0;
    for (size_t j = w.size(); j-- > 0;) {
      tail += w[j];
      om32[j] = (float)tail;
    }
  }
  HMM_CUDA(h, cudaMalloc(&h->d_boxes, sizeof(BoxDesc) * h->nb));
  HMM_CUDA(h, cudaMalloc(&h->d_W64, sizeof(double) * W64.size()));
  HMM_CUDA(h, cudaMalloc(&h->d_W32, sizeof(float) * W32.size()));
  HMM_CUDA(h, cudaMalloc(&h->d_w64, sizeof(double) * w.size()));
  HMM_CUDA(h, cudaMalloc(&h->d_w32, sizeof(float) * w32.size()));
  HMM_CUDA(h, cudaMalloc(&h->d_om32, sizeof(float) * om32.size()));
  HMM_CUDA(h, cudaMemcpy(h->d_boxes, h->boxes.data(), sizeof(BoxDesc) * h->nb, cudaMemcpyHostToDevice));
  HMM_CUDA(h, cudaMemcpy(h->d_W64, W64.data(), sizeof(double) * W64.size(), cudaMemcpyHostToDevice));
  HMM_CUDA(h, cudaMemcpy(h->d_W32, W32.data(), sizeof(float) * W32.size(), cudaMemcpyHostToDevice));
  HMM_CUDA(h, cudaMemcpy(h->d_w64, w.data(), sizeof(double) * w.size(), cudaMemcpyHostToDevice));
  HMM_CUDA(h, cudaMemcpy(h->d_w32, w32.data(), sizeof(float) * w32.size(), cudaMemcpyHostToDevice));
  HMM_CUDA(h, cudaMemcpy(h->d_om32, om32.data(), sizeof(float) * om32.size(), cudaMemcpyHostToDevice));
  HMM_CUDA(h, cudaMalloc(&h->d_queue, sizeof(int) * kQueues));
  HMM_CUDA(h, cudaMalloc(&h->d_err, sizeof(int)));
  HMM_CUDA(h, cudaMemset(h->d_err, 0, sizeof(int)));
  HMM_CUDA(h, cudaMallocHost(&h->h_err, sizeof(int)));
  const size_t f3 = sizeof(double) * 3 * (size_t)h->P;
  HMM_CUDA(h, cudaMalloc(&h->d_H, f3));
  HMM_CUDA(h, cudaMalloc(&h->d_hist, 2 * f3));
  HMM_CUDA(h, cudaMemset(h->d_hist, 0, 2 * f3));
  HMM_CUDA(h, cudaMalloc(&h->d_acc, f3));
  HMM_CUDA(h, cudaMalloc(&h->d_stage, f3));
  if (flux) HMM_CUDA(h, cudaMalloc(&h->d_F, f3 * h->dim));
  HMM_CUDA(h, cudaEventCreate(&h->ev0));
  HMM_CUDA(h, cudaEventCreate(&h->ev1));
  HMM_CUDA(h, cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming));
  HMM_CUDA(h, cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming));
  HMM_CUDA(h, cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));

  // Kernel choice: the resident 2D FP32 kernel when the box fits one SM.
  int optin = 0;
  HMM_CUDA(h, cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device));
  std::string why = "the resident kernels need the FP32 form and d = 2 (HeunP or RK4P) or d = 3 (HeunP)";
  const bool res_ok = p.precision == HMM_FP32_BATCHED && h->dim >= 2 && p.micro_stepper <= HMM_RK4P &&
                      (p.micro_stepper == HMM_HEUNP || h->dim == 2) &&
                      res2d_make_plan(h->dim, h->boxes.data(), h->nb, h->radius, h->interp_k, p.n_terms,
                                      (size_t)optin - 256, &h->plan, &why, nullptr, true, p.micro_stepper,
                                      p.tile_rows) &&
                      (int)h->plan.groups.size() <= kQueues;
  if (p.kernel_variant == 2 && !res_ok) return fail(h, HMM_ERR_INVALID_ARG, why.c_str());
  h->res2d = res_ok && p.kernel_variant != 1;

  // Launch shape: persistent grid of (CTAs per SM x SMs), capped by the box count.
  int per_sm = 0;
  if (h->res2d) {
    HMM_CUDA(h, res2d_prepare(h->radius, &h->plan, h->num_sms));
    h->slot_bytes = h->dim == 3 ? res3d_slot_bytes(h->nmax) : res2d_slot_bytes(h->nmax);
    HMM_CUDA(h, cudaMalloc(&h->d_items, sizeof(int2) * h->plan.items.size()));
    HMM_CUDA(h, cudaMemcpy(h->d_items, h->plan.items.data(), sizeof(int2) * h->plan.items.size(),
                           cudaMemcpyHostToDevice));
    per_sm = 1;
  } else {
    h->block = 256;
    h->smem = micro_smem_bytes(h->dim, h->nmax, h->interp_k, p.n_terms);
    HMM_CUDA(h, p.precision == HMM_FP64_PLAIN
                    ? prepare_micro_fp64(h->dim, h->radius, h->block, h->smem, &per_sm)
                    : prepare_micro_fp32(h->dim, h->radius, h->block, h->smem, &per_sm));
    h->slot_bytes = p.precision == HMM_FP64_PLAIN ? micro_slot_bytes_fp64(h->dim, h->nmax, p.micro_stepper)
                                                  : micro_slot_bytes_fp32(h->dim, h->nmax, p.micro_stepper);
  }
  if (per_sm < 1) return fail(h, HMM_ERR_INVALID_ARG, "micro kernel does not fit on an SM for this box size");
  h->grid = h->res2d ? res2d_max_grid(h->plan) : std::min(h->nb, per_sm * h->num_sms);
  HMM_CUDA(h, cudaMalloc(&h->d_arena, h->slot_bytes * (size_t)h->grid));

  MicroArgs& a = h->args;
  a.boxes = h->d_boxes;
  a.n_boxes = h->nb;
  a.Fout = h->d_F;
  a.queue = h->d_queue;
  a.err = h->d_err;
  a.P = h->P;
  for (int k = 0; k < 3; ++k) {
    a.nmac[k] = h->nmac[k];
    a.DX[k] = h->DX[k];
  }
  a.interp_k = h->interp_k;
  a.msteps = M;
  a.stepper = p.micro_stepper;
  a.alpha_micro = p.alpha_micro;
  a.W64 = h->d_W64;
  a.W32 = h->d_W32;
  a.w64 = h->d_w64;
  a.w32 = h->d_w32;
  a.om32 = h->d_om32;
  a.c0 = p.c0;
  a.n_terms = p.n_terms;
  for (int t = 0; t < p.n_terms; ++t) {
    const auto& s = h->terms[t];
    TermDev& d = a.terms[t];
    d.amp = s.amp;
    for (int k = 0; k < 3; ++k) {
      d.kind[k] = s.kind[k];
      d.scale[k] = s.scale[k];
      d.omega[k] = s.omega[k];
      d.phase[k] = s.phase[k];
    }
  }
  a.arena = h->d_arena;
  a.slot_bytes = h->slot_bytes;
  a.nmax = h->nmax;
  if (h->res2d && h->dim == 2) {
    const hmm_status st = tune_resident_plan(h);
    if (st != HMM_OK) return st;
  }
  if (h->res2d && h->dim == 3) {
    // the 3D launch groups: kernel, box size, CTAs per cluster (chosen by occupancy for
    // the z-column kernel), CTAs launched, threads per CTA
    std::string rep;
    for (const Res2dGroup& g : h->plan.groups) {
      char line[160];
      std::snprintf(line, sizeof line, "3D %s: N=%d cluster=%d grid=%d threads=%d items=%d\n",
                    g.N > 0 ? "z-column kernel" : "z-slab kernel", g.N > 0 ? g.N : h->boxes[h->plan.items[g.first_item].x].N,
                    g.cs, g.grid, g.threads, g.n_items);
      rep += line;
    }
    h->plan_report = rep;
  }
  return HMM_OK;
}

// Enqueue one micro batch (no synchronisation). It overwrites what a macro step in
// waves has gathered so far, so it abandons such a step.
hmm_status enqueue_micro(HmmHandle* h, const double* M, double* Havg) {
  h->wave_next = 0;
  HMM_CUDA(h, cudaMemsetAsync(h->d_queue, 0, sizeof(int) * kQueues, h->stream));
  MicroArgs a = h->args;
  a.M = M;
  a.Havg = Havg;
  cudaError_t e = h->res2d ? res2d_launch(a, h->radius, h->plan, h->d_items, h->d_queue, h->stream)
                 : h->p.precision == HMM_FP64_PLAIN
                      ? launch_micro_fp64(a, h->dim, h->radius, h->grid, h->block, h->smem, h->stream)
                      : launch_micro_fp32(a, h->dim, h->radius, h->grid, h->block, h->smem, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "micro kernel launch");
  if (h->p.model == HMM_FLUX_MODEL && Havg) {
    e = launch_flux_divergence(h->d_F, Havg, h->dim, h->nmac, h->DX, h->p.interp_order, h->P, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "flux divergence launch");
  }
  return HMM_OK;
}

// Enqueue the micro batch of wave w of n: a contiguous share of every resident launch
// group's work items (each group's share keeps its longest-first order), or of the
// generic kernel's box list. The kernels write H_avg (field model) or F (flux model)
// at the macro points of the wave's boxes only.
hmm_status enqueue_micro_wave(HmmHandle* h, const double* M, double* Havg, int w, int n) {
  HMM_CUDA(h, cudaMemsetAsync(h->d_queue, 0, sizeof(int) * kQueues, h->stream));
  MicroArgs a = h->args;
  a.M = M;
  a.Havg = Havg;
  cudaError_t e = cudaSuccess;
  if (h->res2d) {
    Res2dPlan pl;
    pl.smem = h->plan.smem;
    pl.dim = h->plan.dim;
    for (const Res2dGroup& g : h->plan.groups) {
      const long long lo = (long long)g.n_items * w / n, hi = (long long)g.n_items * (w + 1) / n;
      if (hi == lo) continue;
      Res2dGroup s = g;
      s.first_item = g.first_item + (int)lo;
      s.n_items = (int)(hi - lo);
      pl.groups.push_back(s);
    }
    if (!pl.groups.empty()) e = res2d_launch(a, h->radius, pl, h->d_items, h->d_queue, h->stream);
  } else {
    const long long lo = (long long)h->nb * w / n, hi = (long long)h->nb * (w + 1) / n;
    a.boxes = h->d_boxes + lo;
    a.n_boxes = (int)(hi - lo);
    const int grid = std::min(h->grid, a.n_boxes);
    e = h->p.precision == HMM_FP64_PLAIN ? launch_micro_fp64(a, h->dim, h->radius, grid, h->block, h->smem, h->stream)
                                         : launch_micro_fp32(a, h->dim, h->radius, grid, h->block, h->smem, h->stream);
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "micro kernel launch");
  return HMM_OK;
}

hmm_status check_error_word(HmmHandle* h) {
  HMM_CUDA(h, cudaMemcpyAsync(h->h_err, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  HMM_CUDA(h, cudaStreamSynchronize(h->stream));
  const int e = *h->h_err;
  if (e) {
    HMM_CUDA(h, cudaMemsetAsync(h->d_err, 0, sizeof(int), h->stream));
    HMM_CUDA(h, cudaStreamSynchronize(h->stream));
    if (e & kErrCoefNonPositive) return fail(h, HMM_ERR_INVALID_ARG, "coefficient a^eps <= 0 at a micro face (A1)");
    return fail(h, HMM_ERR_NONFINITE, "non-finite value in the micro solve or macro state");
  }
  return HMM_OK;
}

hmm_status enqueue_mpea_step(HmmHandle* h, double* M) {
  hmm_status s = enqueue_micro(h, M, h->d_H);
  if (s != HMM_OK) return s;
  cudaError_t e = launch_mpea_update(M, h->d_H, h->d_hist, h->p.alpha, h->dt_macro, h->p.macro_stepper, h->P,
                                     h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "mpea kernel launch");
  return HMM_OK;
}

hmm_status enqueue_rk4_step(HmmHandle* h, double* M) {
  const double* states[4] = {M, h->d_stage, h->d_stage, h->d_stage};
  for (int stage = 1; stage <= 4; ++stage) {
    hmm_status s = enqueue_micro(h, states[stage - 1], h->d_H);
    if (s != HMM_OK) return s;
    double* next = stage == 4 ? M : h->d_stage;
    cudaError_t e = launch_rk4_stage(M, states[stage - 1], h->d_H, h->p.alpha, h->dt_macro, stage,
                                     h->d_acc, next, h->d_hist, h->P, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "rk4 stage launch");
  }
  return HMM_OK;
}

hmm_status ensure_graph(HmmHandle* h, double* M) {
  if (h->graph && h->graph_M == M) return HMM_OK;
  if (h->graph) {
    cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
  }
  cudaGraph_t g;
  HMM_CUDA(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
  hmm_status s = enqueue_mpea_step(h, M);
  cudaError_t e = cudaStreamEndCapture(h->stream, &g);
  if (s != HMM_OK) return s;
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(&h->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphInstantiate");
  h->graph_M = M;
  return HMM_OK;
}

HmmHandle* as_handle(void* p) { return static_cast<HmmHandle*>(p); }

// Order the library's stream after the work already queued on the caller's stream.
hmm_status begin_call(HmmHandle* h) {
  HMM_CUDA(h, cudaEventRecord(h->ev_in, h->user_stream));
  HMM_CUDA(h, cudaStreamWaitEvent(h->stream, h->ev_in, 0));
  return HMM_OK;
}

// Order the caller's stream after the library's work.
hmm_status end_call(HmmHandle* h) {
  HMM_CUDA(h, cudaEventRecord(h->ev_out, h->stream));
  HMM_CUDA(h, cudaStreamWaitEvent(h->user_stream, h->ev_out, 0));
  return HMM_OK;
}

#define HMM_TRY(expr)                 \
  do {                                \
    hmm_status s_ = (expr);           \
    if (s_ != HMM_OK) return s_;      \
  } while (0)

}  // namespace

// ------------------------------------------------------------------ C ABI
extern "C" {

hmm_status hmm_init(const hmm_params* params, void* cuda_stream, void** handle_out) {
  g_init_error[0] = 0;
  if (!params || !handle_out) return fail(nullptr, HMM_ERR_INVALID_ARG, "null params or handle_out");
  *handle_out = nullptr;
  HmmHandle* h = new (std::nothrow) HmmHandle();
  if (!h) return fail(nullptr, HMM_ERR_OUT_OF_MEMORY, "host allocation failed");
  h->p = *params;
  h->user_stream = static_cast<cudaStream_t>(cuda_stream);
  hmm_status s = build(h);
  if (s != HMM_OK) {
    hmm::set_null_handle_error(h->err.c_str());
    free_all(h);
    delete h;
    return s;
  }
  *handle_out = h;
  return HMM_OK;
}

hmm_status hmm_micro_batch(void* handle, const double* M_dev, double* Havg_dev) {
  HmmHandle* h = as_handle(handle);
  if (!h) return fail(nullptr, HMM_ERR_NOT_INITIALISED, "null handle");
  if (!M_dev || !Havg_dev) return fail(h, HMM_ERR_INVALID_ARG, "null device pointer");
  HMM_TRY(begin_call(h));
  HMM_CUDA(h, cudaEventRecord(h->ev0, h->stream));
  hmm_status s = enqueue_micro(h, M_dev, Havg_dev);
  if (s != HMM_OK) return s;
  HMM_CUDA(h, cudaEventRecord(h->ev1, h->stream));
  HMM_TRY(end_call(h));
  s = check_error_word(h);
  float ms = 0;
  cudaEventElapsedTime(&ms, h->ev0, h->ev1);
  h->last_ms = ms;
  return s;
}

hmm_status hmm_flux_batch(void* handle, const double* M_dev, double* F_dev) {
  HmmHandle* h = as_handle(handle);
  if (!h) return fail(nullptr, HMM_ERR_NOT_INITIALISED, "null handle");
  if (!M_dev || !F_dev) return fail(h, HMM_ERR_INVALID_ARG, "null device pointer");
  if (h->p.model != HMM_FLUX_MODEL) return fail(h, HMM_ERR_INVALID_ARG, "hmm_flux_batch needs a flux-model handle");
  HMM_TRY(begin_call(h));
  HMM_CUDA(h, cudaEventRecord(h->ev0, h->stream));
  hmm_status s = enqueue_micro(h, M_dev, nullptr);
  if (s != HMM_OK) return s;
  HMM_CUDA(h, cudaEventRecord(h->ev1, h->stream));
  HMM_CUDA(h, cudaMemcpyAsync(F_dev, h->d_F, sizeof(double) * 3 * (size_t)h->P * h->dim, cudaMemcpyDeviceToDevice,
                              h->stream));
  HMM_TRY(end_call(h));
  s = check_error_word(h);
  float ms = 0;
  cudaEventElapsedTime(&ms, h->ev0, h->ev1);
  h->last_ms = ms;
  return s;
}

hmm_status hmm_micro_batch_points(void* handle, const double* M_dev, double* Havg_dev, const int* points_host,
                                  int n_points) {
  HmmHandle* h = as_handle(handle);
  if (!h) return fail(nullptr, HMM_ERR_NOT_INITIALISED, "null handle");
  if (!M_dev || !Havg_dev || (n_points > 0 && !points_host))
    return fail(h, HMM_ERR_INVALID_ARG, "null pointer");
  if (h->p.model != HMM_FIELD_MODEL) return fail(h, HMM_ERR_INVALID_ARG, "hmm_micro_batch_points needs a field-model handle");
  h->wave_next = 0;   // like every other micro batch, it abandons a macro step in waves
  if (n_points < 0 || n_points > h->P) return fail(h, HMM_ERR_INVALID_ARG, "n_points must be 0..P");
  if (h->box_of_point.empty()) {
    h->box_of_point.assign(h->P, -1);
    for (int b = 0; b < h->nb; ++b) h->box_of_point[h->boxes[b].p] = b;
  }
  std::vector<char> seen(h->P, 0);
  std::vector<BoxDesc> sub;
  sub.reserve(n_points);
  int nmax = 0;
  for (int i = 0; i < n_points; ++i) {
    const int pt = points_host[i];
    if (pt < 0 || pt >= h->P) return fail(h, HMM_ERR_INVALID_ARG, "macro point index out of range");
    if (seen[pt]) return fail(h, HMM_ERR_INVALID_ARG, "macro point listed twice");
    seen[pt] = 1;
    sub.push_back(h->boxes[h->box_of_point[pt]]);
    nmax = std::max(nmax, sub.back().N);
  }
  if (n_points == 0) return HMM_OK;
  std::stable_sort(sub.begin(), sub.end(), [](const BoxDesc& x, const BoxDesc& y) { return x.N > y.N; });
  // The generic persistent kernel of the handle's precision over just these boxes.
  const int block = 256;
  const size_t smem = micro_smem_bytes(h->dim, nmax, h->interp_k, h->p.n_terms);
  int per_sm = 0;
  HMM_CUDA(h, h->p.precision == HMM_FP64_PLAIN ? prepare_micro_fp64(h->dim, h->radius, block, smem, &per_sm)
                                                : prepare_micro_fp32(h->dim, h->radius, block, smem, &per_sm));
  if (per_sm < 1) return fail(h, HMM_ERR_INVALID_ARG, "micro kernel does not fit on an SM for this box size");
  const size_t slot = h->p.precision == HMM_FP64_PLAIN ? micro_slot_bytes_fp64(h->dim, nmax, h->p.micro_stepper)
                                                        : micro_slot_bytes_fp32(h->dim, nmax, h->p.micro_stepper);
  const int grid = std::min(n_points, per_sm * h->num_sms);
  HMM_TRY(begin_call(h));
  if (n_points > h->sub_cap) {
    HMM_CUDA(h, cudaStreamSynchronize(h->stream));
    if (h->d_sub_boxes) cudaFree(h->d_sub_boxes);
    h->d_sub_boxes = nullptr;
    h->sub_cap = 0;
    HMM_CUDA(h, cudaMalloc(&h->d_sub_boxes, sizeof(BoxDesc) * n_points));
    h->sub_cap = n_points;
  }
  if (slot * grid > h->sub_arena_bytes) {
    HMM_CUDA(h, cudaStreamSynchronize(h->stream));
    if (h->d_sub_arena) cudaFree(h->d_sub_arena);
    h->d_sub_arena = nullptr;
    h->sub_arena_bytes = 0;
    HMM_CUDA(h, cudaMalloc(&h->d_sub_arena, slot * grid));
    h->sub_arena_bytes = slot * grid;
  }
  HMM_CUDA(h, cudaMemcpyAsync(h->d_sub_boxes, sub.data(), sizeof(BoxDesc) * n_points, cudaMemcpyHostToDevice,
                              h->stream));
  HMM_CUDA(h, cudaStreamSynchronize(h->stream));   // the host vector goes out of scope
  HMM_CUDA(h, cudaMemsetAsync(h->d_queue, 0, sizeof(int) * kQueues, h->stream));
  MicroArgs a = h->args;
  a.boxes = h->d_sub_boxes;
  a.n_boxes = n_points;
  a.arena = h->d_sub_arena;
  a.slot_bytes = slot;
  a.nmax = nmax;
  a.M = M_dev;
  a.Havg = Havg_dev;
  HMM_CUDA(h, cudaEventRecord(h->ev0, h->stream));
  cudaError_t e = h->p.precision == HMM_FP64_PLAIN ? launch_micro_fp64(a, h->dim, h->radius, grid, block, smem, h->stream)
                                                    : launch_micro_fp32(a, h->dim, h->radius, grid, block, smem, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "micro kernel launch");
  HMM_CUDA(h, cudaEventRecord(h->ev1, h->stream));
  HMM_TRY(end_call(h));
  hmm_status s = check_error_word(h);
  float ms = 0;
  cudaEventElapsedTime(&ms, h->ev0, h->ev1);
  h->last_ms = ms;
  return s;
}

hmm_status hmm_micro_batch_host(void* handle, const double* M_host, double* Havg_host) {
  HmmHandle* h = as_handle(handle);
  if (!h) return fail(nullptr, HMM_ERR_NOT_INITIALISED, "null handle");
  if (!M_host || !Havg_host) return fail(h, HMM_ERR_INVALID_ARG, "null host pointer");
  const size_t f3 = sizeof(double) * 3 * (size_t)h->P;
  if (!h->d_Mhost) HMM_CUDA(h, cudaMalloc(&h->d_Mhost, f3));
  if (!h->d_Hhost) HMM_CUDA(h, cudaMalloc(&h->d_Hhost, f3));
  HMM_TRY(begin_call(h));
  HMM_CUDA(h, cudaMemcpyAsync(h->d_Mhost, M_host, f3, cudaMemcpyHostToDevice, h->stream));
  hmm_status s = enqueue_micro(h, h->d_Mhost, h->d_Hhost);
  if (s != HMM_OK) return s;
  HMM_CUDA(h, cudaMemcpyAsync(Havg_host, h->d_Hhost, f3, cudaMemcpyDeviceToHost, h->stream));
  return check_error_word(h);
}

hmm_status hmm_macro_step(void* handle, double* M_dev, int n_steps) {
  HmmHandle* h = as_handle(handle);
  if (!h) return fail(nullptr, HMM_ERR_NOT_INITIALISED, "null handle");
  if (!M_dev || n_steps < 0) return fail(h, HMM_ERR_INVALID_ARG, "null M_dev or negative n_steps");
  HMM_TRY(begin_call(h));
  for (int s = 0; s < n_steps; ++s) {
    hmm_status st;
    if (h->j < (h->p.macro_stepper == HMM_MPE ? 1 : 2)) {
      st = enqueue_rk4_step(h, M_dev);
    } else {
      st = ensure_graph(h, M_dev);
      if (st == HMM_OK) {
        cudaError_t e = cudaGraphLaunch(h->graph, h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphLaunch");
      }
    }
    if (st != HMM_OK) return st;
    h->j += 1;
  }
  cudaError_t e = launch_check_finite(M_dev, 3 * h->P, h->d_err, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "finite check launch");
  HMM_TRY(end_call(h));
  return check_error_word(h);
}

hmm_status hmm_macro_step_host(void* handle, double* M_host, int n_steps) {
  HmmHandle* h = as_handle(handle);
  if (!h) return fail(nullptr, HMM_ERR_NOT_INITIALISED, "null handle");
  if (!M_host) return fail(h, HMM_ERR_INVALID_ARG, "null host pointer");
  const size_t f3 = sizeof(double) * 3 * (size_t)h->P;
  if (!h->d_Mhost) HMM_CUDA(h, cudaMalloc(&h->d_Mhost, f3));
  HMM_CUDA(h, cudaMemcpyAsync(h->d_Mhost, M_host, f3, cudaMemcpyHostToDevice, h->stream));
  hmm_status s = hmm_macro_step(handle, h->d_Mhost, n_steps);
  if (s != HMM_OK) return s;
  HMM_CUDA(h, cudaMemcpyAsync(M_host, h->d_Mhost, f3, cudaMemcpyDeviceToHost, h->stream));
  HMM_CUDA(h, cudaStreamSynchronize(h->stream));
  return HMM_OK;
}

hmm_status hmm_macro_step_wave(void* handle, double* M_dev, int wave, int n_waves) {
  HmmHandle* h = as_handle(handle);
  if (!h) return fail(nullptr, HMM_ERR_NOT_INITIALISED, "null handle");
  if (!M_dev) return fail(h, HMM_ERR_INVALID_ARG, "null M_dev");
  if (n_waves < 1 || n_waves > h->nb || wave < 0 || wave >= n_waves)
    return fail(h, HMM_ERR_INVALID_ARG, "need 1 <= n_waves <= the number of micro problems and 0 <= wave < n_waves");
  if (h->j < (h->p.macro_stepper == HMM_MPE ? 1 : 2))
    return fail(h, HMM_ERR_INVALID_ARG,
                "a macro step in waves needs the multistep history: take the RK4P start-up steps with hmm_macro_step");
  if (wave != h->wave_next || (wave > 0 && (n_waves != h->wave_n || M_dev != h->wave_M)))
    return fail(h, HMM_ERR_INVALID_ARG,
                "the waves of one macro step come in the order 0 .. n_waves-1, with the same n_waves and M_dev");
  h->wave_next = 0;
  HMM_TRY(begin_call(h));
  HMM_CUDA(h, cudaEventRecord(h->ev0, h->stream));
  hmm_status s = enqueue_micro_wave(h, M_dev, h->d_H, wave, n_waves);
  if (s != HMM_OK) return s;
  HMM_CUDA(h, cudaEventRecord(h->ev1, h->stream));
  const bool last = wave == n_waves - 1;
  if (last) {
    cudaError_t e = cudaSuccess;
    if (h->p.model == HMM_FLUX_MODEL)
      e = launch_flux_divergence(h->d_F, h->d_H, h->dim, h->nmac, h->DX, h->p.interp_order, h->P, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "flux divergence launch");
    e = launch_mpea_update(M_dev, h->d_H, h->d_hist, h->p.alpha, h->dt_macro, h->p.macro_stepper, h->P, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "mpea kernel launch");
    e = launch_check_finite(M_dev, 3 * h->P, h->d_err, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "finite check launch");
  }
  HMM_TRY(end_call(h));
  s = check_error_word(h);
  float ms = 0;
  cudaEventElapsedTime(&ms, h->ev0, h->ev1);
  h->last_ms = ms;
  if (s != HMM_OK) return s;
  if (last) {
    h->j += 1;
  } else {
    h->wave_next = wave + 1;
    h->wave_n = n_waves;
    h->wave_M = M_dev;
  }
  return HMM_OK;
}

hmm_status hmm_get_state(void* handle, double* hist_dev, long long* j) {
  HmmHandle* h = as_handle(handle);
  if (!h) return fail(nullptr, HMM_ERR_NOT_INITIALISED, "null handle");
  if (hist_dev) {
    HMM_TRY(begin_call(h));
    HMM_CUDA(h, cudaMemcpyAsync(hist_dev, h->d_hist, sizeof(double) * 6 * (size_t)h->P,
                                cudaMemcpyDeviceToDevice, h->stream));
    HMM_CUDA(h, cudaStreamSynchronize(h->stream));
  }
  if (j) *j = h->j;
  return HMM_OK;
}

hmm_status hmm_set_state(void* handle, const double* hist_dev, long long j) {
  HmmHandle* h = as_handle(handle);
  if (!h) return fail(nullptr, HMM_ERR_NOT_INITIALISED, "null handle");
  if (j < 0) return fail(h, HMM_ERR_INVALID_ARG, "negative step count");
  h->wave_next = 0;
  if (hist_dev) {
    HMM_TRY(begin_call(h));
    HMM_CUDA(h, cudaMemcpyAsync(h->d_hist, hist_dev, sizeof(double) * 6 * (size_t)h->P,
                                cudaMemcpyDeviceToDevice, h->stream));
    HMM_CUDA(h, cudaStreamSynchronize(h->stream));
  } else if (j >= 1) {
    return fail(h, HMM_ERR_INVALID_ARG, "a step count >= 1 needs the history");
  }
  h->j = j;
  return HMM_OK;
}

hmm_status hmm_stats(void* handle, double* lattice_updates_per_batch, double* last_batch_ms) {
  HmmHandle* h = as_handle(handle);
  if (!h) return fail(nullptr, HMM_ERR_NOT_INITIALISED, "null handle");
  if (lattice_updates_per_batch) *lattice_updates_per_batch = h->lu_per_batch;
  if (last_batch_ms) *last_batch_ms = h->last_ms;
  return HMM_OK;
}

hmm_status hmm_box_info(void* handle, double* dt, double* mu, double* dx, int* n) {
  HmmHandle* h = as_handle(handle);
  if (!h) return fail(nullptr, HMM_ERR_NOT_INITIALISED, "null handle");
  if (dt) std::memcpy(dt, h->box_dt.data(), sizeof(double) * h->P);
  if (mu) std::memcpy(mu, h->box_mu.data(), sizeof(double) * h->P);
  if (dx) std::memcpy(dx, h->box_dx.data(), sizeof(double) * h->P);
  if (n) std::memcpy(n, h->box_n.data(), sizeof(int) * h->P);
  return HMM_OK;
}

hmm_status hmm_set_face_table(void* handle, const double* table_host, long long n_values) {
  HmmHandle* h = as_handle(handle);
  if (!h) return fail(nullptr, HMM_ERR_NOT_INITIALISED, "null handle");
  if (!table_host) return fail(h, HMM_ERR_INVALID_ARG, "null face table");
  if (h->p.model == HMM_FLUX_MODEL)
    return fail(h, HMM_ERR_INVALID_ARG, "tabulated coefficients are not available with the flux model");
  const int d = h->dim;
  std::vector<long long> off(h->P);
  long long total = 0;
  for (int q = 0; q < h->P; ++q) {
    long long nd = 1;
    for (int k = 0; k < d; ++k) nd *= h->box_n[q];
    off[q] = total;
    total += d * nd;
  }
  if (n_values != total) {
    char msg[160];
    std::snprintf(msg, sizeof msg, "face table has %lld values, the boxes need %lld", n_values, total);
    return fail(h, HMM_ERR_INVALID_ARG, msg);
  }
  // each box's maximum over the faces the stencil uses (node index j_k < N - 1); (A1)
  std::vector<double> bmax(h->P, 0.0);
  double gmax = 0.0;
  for (int q = 0; q < h->P; ++q) {
    const int N = h->box_n[q];
    long long nd = 1;
    for (int k = 0; k < d; ++k) nd *= N;
    for (int k = 0; k < d; ++k) {
      long long stride = 1;
      for (int a = k + 1; a < d; ++a) stride *= N;
      const double* blk = table_host + off[q] + k * nd;
      for (long long idx = 0; idx < nd; ++idx) {
        if ((idx / stride) % N == N - 1) continue;
        const double v = blk[idx];
        if (!(v > 0.0) || !std::isfinite(v))
          return fail(h, HMM_ERR_INVALID_ARG, "face table: a^eps must be positive and finite at every used face (A1)");
        bmax[q] = std::max(bmax[q], v);
      }
    }
    gmax = std::max(gmax, bmax[q]);
  }
  HMM_CUDA(h, cudaStreamSynchronize(h->stream));   // no batch in flight reads the old table
  if (h->d_faces) cudaFree(h->d_faces);
  if (h->d_face_off) cudaFree(h->d_face_off);
  h->d_faces = nullptr;
  h->d_face_off = nullptr;
  HMM_CUDA(h, cudaMalloc(&h->d_faces, sizeof(double) * (size_t)total));
  HMM_CUDA(h, cudaMalloc(&h->d_face_off, sizeof(long long) * (size_t)h->P));
  HMM_CUDA(h, cudaMemcpy(h->d_faces, table_host, sizeof(double) * (size_t)total, cudaMemcpyHostToDevice));
  HMM_CUDA(h, cudaMemcpy(h->d_face_off, off.data(), sizeof(long long) * (size_t)h->P, cudaMemcpyHostToDevice));
  // micro time steps from each box's maximum; the macro step from the global one when
  // the library chose it
  const hmm_params& p = h->p;
  for (BoxDesc& bd : h->boxes) {
    bd.dt = host::micro_dt(p.dt_safety, p.alpha_micro, bmax[bd.p], d, p.stencil_order, bd.dx, p.micro_stepper);
    h->box_dt[bd.p] = bd.dt;
  }
  HMM_CUDA(h, cudaMemcpy(h->d_boxes, h->boxes.data(), sizeof(BoxDesc) * h->nb, cudaMemcpyHostToDevice));
  h->a_max = gmax;
  if (!(p.dt_macro > 0)) {
    double dX = h->DX[0];
    for (int k = 1; k < d; ++k) dX = std::min(dX, h->DX[k]);
    h->dt_macro = kMacroDtConstant * dX * dX / (d * gmax);
  }
  h->args.faces = h->d_faces;
  h->args.face_off = h->d_face_off;
  if (h->res2d && h->dim == 3 && res3d_plan_uses_col3(h->plan)) {
    // the z-column kernel evaluates separable coefficient terms in its time loop:
    // tabulated coefficients run on the z-slab kernel, which reads the set-up's faces
    Res2dPlan pl;
    std::string why;
    if (!res2d_make_plan(3, h->boxes.data(), h->nb, h->radius, h->interp_k, p.n_terms, h->plan.smem, &pl, &why,
                         nullptr, false))
      return fail(h, HMM_ERR_INVALID_ARG, why);
    HMM_CUDA(h, res2d_prepare(h->radius, &pl, h->num_sms));
    const int grid = res2d_max_grid(pl);
    if (grid > h->grid) {
      char* ar = nullptr;
      HMM_CUDA(h, cudaMalloc(&ar, h->slot_bytes * (size_t)grid));
      cudaFree(h->d_arena);
      h->d_arena = ar;
      h->args.arena = ar;
      h->grid = grid;
    }
    if (pl.items.size() != h->plan.items.size()) return fail(h, HMM_ERR_INVALID_ARG, "3D work items changed size");
    HMM_CUDA(h, cudaMemcpy(h->d_items, pl.items.data(), sizeof(int2) * pl.items.size(), cudaMemcpyHostToDevice));
    h->plan = pl;
  }
  if (h->graph) {   // captured with the old arguments
    cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
    h->graph_M = nullptr;
  }
  return HMM_OK;
}

hmm_status hmm_macro_dt(void* handle, double* dt_macro) {
  HmmHandle* h = as_handle(handle);
  if (!h) return fail(nullptr, HMM_ERR_NOT_INITIALISED, "null handle");
  if (!dt_macro) return fail(h, HMM_ERR_INVALID_ARG, "null pointer");
  *dt_macro = h->dt_macro;
  return HMM_OK;
}

const char* hmm_plan_report(void* handle) {
  HmmHandle* h = as_handle(handle);
  return h ? h->plan_report.c_str() : "";
}

const char* hmm_last_error(void* handle) {
  HmmHandle* h = as_handle(handle);
  return h ? h->err.c_str() : g_init_error;
}

void hmm_destroy(void* handle) {
  HmmHandle* h = as_handle(handle);
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  free_all(h);
  delete h;
}

}  // extern "C"

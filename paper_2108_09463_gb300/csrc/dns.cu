// Host side and point-wise kernels of the direct simulation resolving eps
// (include/hmm_dns.h). The stencil kernels are in dns_kernels.cuh.
//
// hmm_dns_init validates the problem, tabulates the separable factors of the
// coefficient per axis (FP64 and FP32 copies), picks the time step from the
// AB3 stability limit (the linearisation of MPEA's extrapolated midpoint step)
// and allocates the state. hmm_dns_step runs the RK4P start-up steps (FP64, a
// field kernel per stage and a point-wise stage kernel) and then one fused
// MPEA kernel per step, ping-ponging the state and rotating three history
// buffers.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/hmm_dns.h"
#include "dns_kernels.cuh"

using namespace hmm_dns;

namespace {

thread_local std::string g_dns_init_error;
constexpr int kMaxTerms = 8;   // coefficient terms accepted (as in hmm_params)

struct DnsHandle {
  hmm_dns_params p{};
  std::vector<hmm_coef_term> terms;
  cudaStream_t user = nullptr;    // the caller's stream
  cudaStream_t stream = nullptr;  // the library's own non-blocking stream (capturable)
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  cudaGraphExec_t graph[2][3] = {};   // six MPEA steps, by (cur, j mod 3) at their start
  int d = 1, n0 = 1, n1 = 1, order = 4, precision = 0;
  long long G = 0;
  double dx[2] = {0, 0};          // slow, fast axis spacing
  double dt = 0, a_max = 0;
  long long j = 0;
  int cur = 0;                    // state buffer holding the current state
  Args base{};
  // device memory
  double* d_face64 = nullptr;     // ax | ay (G each): faces along the fast, the slow axis
  float* d_face32 = nullptr;
  void* d_state[2] = {nullptr, nullptr};   // FP64: 3G doubles; FF: 6G floats
  void* d_hist[3] = {nullptr, nullptr, nullptr};
  double* d_m64 = nullptr;        // start-up state (FF form)
  double* d_stage = nullptr;      // RK4P stage state
  double* d_H = nullptr;          // RK4P stage field
  double* d_acc = nullptr;        // RK4P accumulator
  double* d_host_io = nullptr;    // staging for hmm_dns_step_host
  int* d_err = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  double last_ms = 0;
  bool tuned = false;             // the work plan has been autotuned
  std::string err;
};

hmm_status fail(DnsHandle* h, hmm_status s, const std::string& msg) {
  if (h) h->err = msg; else g_dns_init_error = msg;
  return s;
}

hmm_status cuda_fail(DnsHandle* h, cudaError_t e, const char* where) {
  return fail(h, e == cudaErrorMemoryAllocation ? HMM_ERR_OUT_OF_MEMORY : HMM_ERR_CUDA,
              std::string(where) + ": " + cudaGetErrorString(e));
}

#define DNS_CUDA(h, call)                                    \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return cuda_fail((h), e_, #call); \
  } while (0)

#define DNS_TRY(expr)                  \
  do {                                 \
    hmm_status s_ = (expr);            \
    if (s_ != HMM_OK) return s_;       \
  } while (0)

// ------------------------------------------------------------ time step rule
// Largest modulus of the roots of zeta^3 - (1 + 23z/12) zeta^2 + (16z/12) zeta
// - 5z/12 (the AB3 recurrence for y' = lambda y, z = lambda dt), by the
// Durand-Kerner simultaneous iteration.
double ab3_root_modulus(std::complex<double> z) {
  using C = std::complex<double>;
  const C a2 = -(1.0 + 23.0 * z / 12.0), a1 = 16.0 * z / 12.0, a0 = -5.0 * z / 12.0;
  auto poly = [&](C x) { return ((x + a2) * x + a1) * x + a0; };
  C r[3] = {C(0.4, 0.9), C(0.4, 0.9) * C(0.4, 0.9), C(0.4, 0.9) * C(0.4, 0.9) * C(0.4, 0.9)};
  for (int it = 0; it < 500; ++it) {
    double change = 0;
    for (int k = 0; k < 3; ++k) {
      C den(1.0, 0.0);
      for (int m = 0; m < 3; ++m)
        if (m != k) den *= (r[k] - r[m]);
      if (std::abs(den) == 0) den = C(1e-300, 0);
      C step = poly(r[k]) / den;
      r[k] -= step;
      change = std::max(change, std::abs(step));
    }
    if (change < 1e-16) break;
  }
  return std::max({std::abs(r[0]), std::abs(r[1]), std::abs(r[2])});
}

// Largest s with all AB3 roots in the closed unit disc for z = s(-alpha + i):
// outward scan from 0 in steps of 1e-3, then bisection.
double ab3_stability_limit(double alpha) {
  const std::complex<double> w(-alpha, 1.0);
  auto ok = [&](double s) { return ab3_root_modulus(s * w) <= 1.0 + 1e-12; };
  double s = 0.0, ds = 1e-3;
  while (ok(s + ds)) {
    s += ds;
    if (s > 10.0) return -1.0;
  }
  double lo = s, hi = s + ds;
  for (int i = 0; i < 60; ++i) {
    double mid = 0.5 * (lo + hi);
    if (ok(mid)) lo = mid; else hi = mid;
  }
  return lo;
}

// ------------------------------------------------------------ coefficient
double factor(int kind, double th) { return kind == 1 ? std::sin(th) : kind == 2 ? std::cos(th) : 1.0; }

// g_tk(x) for term t on axis k at coordinate x (without amp)
double term_factor(const hmm_coef_term& t, int k, double x, double eps) {
  if (t.kind[k] == 0) return 1.0;
  const double s = t.scale[k] == 0 ? x / eps : x;
  return factor(t.kind[k], 2.0 * M_PI * t.omega[k] * s + t.phase[k]);
}

// ------------------------------------------------------------ point-wise kernels
// Start-up stage s (1..4) of RK4P (Section 3.1) at one point, FP64:
// k_s = f(M_s, H) = -M_s x H - alpha M_s x (M_s x H); acc accumulates
// k1 + 2 k2 + 2 k3 + k4; stages 1-3 write the next (normalised) stage state,
// stage 4 the new state. Stage 1 also stores h^j = H + alpha M x H.
__global__ void dns_rk4_stage(int stage, long long G, double alpha, double dt, double* M, double* Ms,
                              const double* H, double* acc, double* hist64, float* hist32) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= G) return;
  double m[3], s[3], h[3], k[3];
  for (int c = 0; c < 3; ++c) {
    m[c] = M[c * G + i];
    s[c] = stage == 1 ? m[c] : Ms[c * G + i];
    h[c] = H[c * G + i];
  }
  double q[3] = {s[1] * h[2] - s[2] * h[1], s[2] * h[0] - s[0] * h[2], s[0] * h[1] - s[1] * h[0]};
  double r[3] = {s[1] * q[2] - s[2] * q[1], s[2] * q[0] - s[0] * q[2], s[0] * q[1] - s[1] * q[0]};
  for (int c = 0; c < 3; ++c) k[c] = -q[c] - alpha * r[c];
  if (stage == 1) {
    for (int c = 0; c < 3; ++c) {
      double hv = h[c] + alpha * q[c];     // s = M at stage 1: q = M x H
      if (hist64) hist64[c * G + i] = hv;
      if (hist32) hist32[c * G + i] = (float)hv;
    }
  }
  double a[3];
  for (int c = 0; c < 3; ++c) {
    double prev = stage == 1 ? 0.0 : acc[c * G + i];
    a[c] = stage == 1 ? k[c] : prev + ((stage == 4) ? k[c] : 2.0 * k[c]);
    acc[c * G + i] = a[c];
  }
  double u[3];
  if (stage < 4) {
    const double f = stage == 3 ? dt : 0.5 * dt;
    for (int c = 0; c < 3; ++c) u[c] = m[c] + f * k[c];
  } else {
    const double f = dt / 6.0;
    for (int c = 0; c < 3; ++c) u[c] = m[c] + f * a[c];
  }
  const double nrm = std::sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
  double* out = stage < 4 ? Ms : M;
  for (int c = 0; c < 3; ++c) out[c * G + i] = u[c] / nrm;
}

// FP64 state -> float-float state (hi = fl(m), lo = fl(m - hi), one float2 per
// component) and back.
__global__ void dns_split(long long G, const double* M, float2* S) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= G) return;
  for (int c = 0; c < 3; ++c) {
    double v = M[c * G + i];
    float hi = (float)v;
    S[c * G + i] = make_float2(hi, (float)(v - (double)hi));
  }
}

__global__ void dns_join(long long G, const float2* S, double* M) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= G) return;
  for (int c = 0; c < 3; ++c) {
    const float2 v = S[c * G + i];
    M[c * G + i] = (double)v.x + (double)v.y;
  }
}

int pw_blocks(long long G) { return (int)((G + 255) / 256); }

// ------------------------------------------------------------ stencil launch
template <int ORDER, bool TWO_D>
cudaError_t launch_mode(int mode, const Args& a, cudaStream_t st) {
  const int blocks = (a.items + kWarps - 1) / kWarps;
  if (mode == kField) dns_kernel<ORDER, TWO_D, kField><<<blocks, 32 * kWarps, 0, st>>>(a);
  else if (mode == kMpea64) dns_kernel<ORDER, TWO_D, kMpea64><<<blocks, 32 * kWarps, 0, st>>>(a);
  else dns_kernel<ORDER, TWO_D, kMpeaFF><<<blocks, 32 * kWarps, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_stencil(int mode, const DnsHandle* h, const Args& a) {
  const bool two = h->d == 2;
  if (h->order == 4) return two ? launch_mode<4, true>(mode, a, h->stream) : launch_mode<4, false>(mode, a, h->stream);
  return two ? launch_mode<2, true>(mode, a, h->stream) : launch_mode<2, false>(mode, a, h->stream);
}

// Resident warps of the time-stepping kernel on the whole GPU (occupancy of
// its instantiation times the SM count); 152 * 16 if the device cannot be asked.
template <int ORDER, bool TWO_D>
long long resident_warps_of(int mode) {
  int dev = 0, sms = 0, blocks = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) {
    if (mode == kMpeaFF)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, dns_kernel<ORDER, TWO_D, kMpeaFF>, 32 * kWarps, 0);
    else
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, dns_kernel<ORDER, TWO_D, kMpea64>, 32 * kWarps, 0);
  }
  if (e != cudaSuccess || sms <= 0 || blocks <= 0) {
    cudaGetLastError();
    return 152LL * 16;
  }
  return (long long)sms * blocks * kWarps;
}

// Rows per work item: as few chunks as keep every resident warp of the
// time-stepping kernel busy in one wave (each chunk re-reads 2R halo rows, so
// long chunks are cheaper), at least 8 rows.
void plan_work(DnsHandle* h) {
  const int R = h->order == 4 ? 3 : 1;
  const int W = 32 - 2 * R;
  Args& a = h->base;
  a.n0 = h->n0;
  a.n1 = h->n1;
  a.G = h->G;
  a.strips = (h->n1 + W - 1) / W;
  if (h->d == 1) {
    a.chunk = 1;
    a.chunks = 1;
  } else {
    const int mode = h->precision == HMM_FP64_PLAIN ? kMpea64 : kMpeaFF;
    const long long target = h->order == 4 ? resident_warps_of<4, true>(mode) : resident_warps_of<2, true>(mode);
    long long ch = ((long long)h->n0 * a.strips + target - 1) / target;
    ch = std::max<long long>(8, std::min<long long>(ch, h->n0));
    a.chunk = (int)ch;
    a.chunks = (h->n0 + a.chunk - 1) / a.chunk;
  }
  a.items = a.strips * a.chunks;
}

// ------------------------------------------------------------ tables
// Copies face coefficients (fast-axis faces, then slow-axis faces; G each) to
// the device in FP64 and FP32.
hmm_status upload_faces(DnsHandle* h, const std::vector<double>& f64) {
  std::vector<float> f32(f64.size());
  for (size_t i = 0; i < f64.size(); ++i) f32[i] = (float)f64[i];
  if (!h->d_face64) {
    DNS_CUDA(h, cudaMalloc(&h->d_face64, f64.size() * sizeof(double)));
    DNS_CUDA(h, cudaMalloc(&h->d_face32, f32.size() * sizeof(float)));
  }
  DNS_CUDA(h, cudaMemcpy(h->d_face64, f64.data(), f64.size() * sizeof(double), cudaMemcpyHostToDevice));
  DNS_CUDA(h, cudaMemcpy(h->d_face32, f32.data(), f32.size() * sizeof(float), cudaMemcpyHostToDevice));
  Args& a = h->base;
  a.ax64 = h->d_face64;
  a.ay64 = h->d_face64 + h->G;
  a.ax32 = h->d_face32;
  a.ay32 = h->d_face32 + h->G;
  return HMM_OK;
}

// a^eps at every face from the separable terms: per axis the terms' factors
// are tabulated once (amp folded into the fast axis), then a_x(r, i) =
// c0 + sum_t X_t(face i) Y_t(node r) and a_y(r, i) = c0 + sum_t X_t(node i) Y_t(face r).
hmm_status build_faces(DnsHandle* h) {
  const int n0 = h->n0, n1 = h->n1, nt = (int)h->terms.size();
  const int kf = h->d - 1;               // axis index of the fast axis
  std::vector<double> tfx((size_t)nt * n1), tnx((size_t)nt * n1), tfy((size_t)nt * n0, 1.0), tny((size_t)nt * n0, 1.0);
  for (int t = 0; t < nt; ++t) {
    const hmm_coef_term& T = h->terms[t];
    for (int i = 0; i < n1; ++i) {
      tfx[(size_t)t * n1 + i] = T.amp * term_factor(T, kf, (i + 0.5) * h->dx[1], h->p.eps);
      tnx[(size_t)t * n1 + i] = T.amp * term_factor(T, kf, i * h->dx[1], h->p.eps);
    }
    if (h->d == 2)
      for (int r = 0; r < n0; ++r) {
        tfy[(size_t)t * n0 + r] = term_factor(T, 0, (r + 0.5) * h->dx[0], h->p.eps);
        tny[(size_t)t * n0 + r] = term_factor(T, 0, r * h->dx[0], h->p.eps);
      }
  }
  const long long G = h->G;
  std::vector<double> f64((size_t)2 * G, 1.0);
  double amin = 1e300;
  for (int r = 0; r < n0; ++r)
    for (int i = 0; i < n1; ++i) {
      double ax = h->p.c0, ay = h->p.c0;
      for (int t = 0; t < nt; ++t) {
        ax += tfx[(size_t)t * n1 + i] * tny[(size_t)t * n0 + r];
        ay += tnx[(size_t)t * n1 + i] * tfy[(size_t)t * n0 + r];
      }
      const long long g = (long long)r * n1 + i;
      f64[g] = ax;
      if (h->d == 2) f64[G + g] = ay;
      amin = std::min(amin, h->d == 2 ? std::min(ax, ay) : ax);
    }
  // a > 0 at every face (A1)
  if (!(amin > 0)) return fail(h, HMM_ERR_INVALID_ARG, "coefficient a^eps <= 0 at a face (A1)");
  return upload_faces(h, f64);
}

hmm_status pick_dt(DnsHandle* h) {
  if (h->p.dt > 0) {
    h->dt = h->p.dt;
  } else {
    const double s = ab3_stability_limit(h->p.alpha);
    if (!(s > 0)) return fail(h, HMM_ERR_INVALID_ARG, "no finite AB3 stability limit");
    const double lam = h->order == 2 ? 4.0 : (28.0 / 12.0) * (28.0 / 12.0);
    double om = 0;
    for (int k = 0; k < h->d; ++k) {
      const double dxk = h->d == 2 ? h->dx[k] : h->dx[1];
      om += lam / (dxk * dxk);
    }
    om *= h->a_max;
    const double safety = h->p.dt_safety > 0 ? h->p.dt_safety : 0.5;
    h->dt = safety * s / om;
  }
  h->base.half_dt = 0.5 * h->dt;
  return HMM_OK;
}

void free_all(DnsHandle* h) {
  void* ptrs[] = {h->d_face64, h->d_face32, h->d_state[0], h->d_state[1],
                  h->d_hist[0], h->d_hist[1], h->d_hist[2], h->d_m64, h->d_stage, h->d_H, h->d_acc,
                  h->d_host_io, h->d_err};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (h->ev0) cudaEventDestroy(h->ev0);
  if (h->ev1) cudaEventDestroy(h->ev1);
  if (h->ev_in) cudaEventDestroy(h->ev_in);
  if (h->ev_out) cudaEventDestroy(h->ev_out);
  for (auto& row : h->graph)
    for (auto& g : row)
      if (g) cudaGraphExecDestroy(g);
  if (h->stream) cudaStreamDestroy(h->stream);
}

void drop_graphs(DnsHandle* h) {
  for (auto& row : h->graph)
    for (auto& g : row) {
      if (g) cudaGraphExecDestroy(g);
      g = nullptr;
    }
}

DnsHandle* as_handle(void* p) { return reinterpret_cast<DnsHandle*>(p); }

// ------------------------------------------------------------ stepping
hmm_status enqueue_rk4_step(DnsHandle* h, double* M) {
  Args a = h->base;
  const long long G = h->G;
  const int slot = (int)(h->j % 3);
  double* h64 = h->precision == HMM_FP64_PLAIN ? (double*)h->d_hist[slot] : nullptr;
  float* h32 = h->precision == HMM_FP64_PLAIN ? nullptr : (float*)h->d_hist[slot];
  for (int stage = 1; stage <= 4; ++stage) {
    a.m64 = stage == 1 ? M : h->d_stage;
    a.H_out = h->d_H;
    cudaError_t e = launch_stencil(kField, h, a);
    if (e != cudaSuccess) return cuda_fail(h, e, "dns field kernel launch");
    dns_rk4_stage<<<pw_blocks(G), 256, 0, h->stream>>>(stage, G, h->p.alpha, h->dt, M, h->d_stage, h->d_H, h->d_acc,
                                                       stage == 1 ? h64 : nullptr, stage == 1 ? h32 : nullptr);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(h, e, "dns rk4 stage launch");
  }
  return HMM_OK;
}

// Arguments of the time-stepping kernel for step j from state cur (the next
// state goes to the other buffer); returns the kernel mode.
int mpea_args(const DnsHandle* h, Args& a) {
  a = h->base;
  const int nxt = 1 - h->cur;
  a.h1 = h->d_hist[(h->j - 1) % 3];
  a.h2 = h->d_hist[(h->j - 2) % 3];
  a.h_out = h->d_hist[h->j % 3];
  a.err = h->d_err;
  if (h->precision == HMM_FP64_PLAIN) {
    a.m64 = (const double*)h->d_state[h->cur];
    a.m64_out = (double*)h->d_state[nxt];
    return kMpea64;
  }
  a.ff = (const float2*)h->d_state[h->cur];
  a.ff_out = (float2*)h->d_state[nxt];
  return kMpeaFF;
}

hmm_status enqueue_mpea_step(DnsHandle* h) {
  Args a;
  const int mode = mpea_args(h, a);
  cudaError_t e = launch_stencil(mode, h, a);
  if (e != cudaSuccess) return cuda_fail(h, e, "dns mpea kernel launch");
  h->cur = 1 - h->cur;
  return HMM_OK;
}

void set_chunk(DnsHandle* h, int chunk) {
  Args& a = h->base;
  a.chunk = chunk;
  a.chunks = (h->n0 + chunk - 1) / chunk;
  a.items = a.strips * a.chunks;
}

// Autotuner of the work plan, run once at the first time step of the
// time-stepping kernel (when the history exists and the state is real): the
// kernel is timed on this grid for a few chunk lengths (rows per work item) --
// the one-wave plan, half, twice and four times it, at least 8 rows and at most
// n0 -- one warm-up and three timed launches each, writing the next state and
// history slots, which the real step then overwrites. The fastest plan is kept;
// the six-step graphs are captured after it.
hmm_status autotune(DnsHandle* h) {
  h->tuned = true;
  if (h->d == 1) return HMM_OK;
  const int c1 = h->base.chunk;
  std::vector<int> cands;
  for (int c : {c1, std::max(8, c1 / 2), std::min(h->n0, 2 * c1), std::min(h->n0, 4 * c1)})
    if (std::find(cands.begin(), cands.end(), c) == cands.end()) cands.push_back(c);
  int best = c1;
  float best_ms = 1e30f;
  for (int c : cands) {
    set_chunk(h, c);
    Args a;
    const int mode = mpea_args(h, a);
    cudaError_t e = launch_stencil(mode, h, a);
    if (e == cudaSuccess) e = cudaEventRecord(h->ev0, h->stream);
    for (int r = 0; r < 3 && e == cudaSuccess; ++r) e = launch_stencil(mode, h, a);
    if (e == cudaSuccess) e = cudaEventRecord(h->ev1, h->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(h->ev1);
    float ms = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, h->ev0, h->ev1);
    if (e != cudaSuccess) return cuda_fail(h, e, "dns autotune");
    if (ms < best_ms) {
      best_ms = ms;
      best = c;
    }
  }
  set_chunk(h, best);
  DNS_CUDA(h, cudaMemsetAsync(h->d_err, 0, sizeof(int), h->stream));
  return HMM_OK;
}

// Six MPEA steps (the state ping-pong and the three history slots both return
// to where they started) as one CUDA graph, captured on first use for the
// current (cur, j mod 3) and replayed afterwards.
hmm_status launch_six(DnsHandle* h) {
  cudaGraphExec_t& g = h->graph[h->cur][h->j % 3];
  if (!g) {
    const int cur0 = h->cur;
    const long long j0 = h->j;
    DNS_CUDA(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    hmm_status st = HMM_OK;
    for (int k = 0; k < 6 && st == HMM_OK; ++k) {
      st = enqueue_mpea_step(h);
      h->j += 1;
    }
    h->cur = cur0;
    h->j = j0;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(h->stream, &graph);
    if (st != HMM_OK) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&g, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      g = nullptr;
      return cuda_fail(h, e, "cudaGraphInstantiate");
    }
  }
  DNS_CUDA(h, cudaGraphLaunch(g, h->stream));
  h->j += 6;                      // cur is unchanged after an even number of steps
  return HMM_OK;
}

// The current state lives in d_state[cur] (FP64 form always; FF form once the
// start-up is over) or, during the FF form's start-up, in d_m64. The work runs
// on the library's stream, ordered after the caller's stream and before its
// later work by events.
hmm_status run_steps(DnsHandle* h, double* M_dev, int n_steps) {
  const long long G = h->G;
  const size_t bytes64 = (size_t)3 * G * sizeof(double);
  DNS_CUDA(h, cudaEventRecord(h->ev_in, h->user));
  DNS_CUDA(h, cudaStreamWaitEvent(h->stream, h->ev_in, 0));
  DNS_CUDA(h, cudaMemsetAsync(h->d_err, 0, sizeof(int), h->stream));
  DNS_CUDA(h, cudaEventRecord(h->ev0, h->stream));
  const bool ff = h->precision != HMM_FP64_PLAIN;
  double* m64 = ff ? h->d_m64 : (double*)h->d_state[h->cur];
  bool in_m64 = true;
  if (ff && h->j >= 2) {
    dns_split<<<pw_blocks(G), 256, 0, h->stream>>>(G, M_dev, (float2*)h->d_state[h->cur]);
    in_m64 = false;
  } else {
    DNS_CUDA(h, cudaMemcpyAsync(m64, M_dev, bytes64, cudaMemcpyDeviceToDevice, h->stream));
    if (!ff) in_m64 = false;    // FP64: d_state[cur] is m64
  }
  for (int s = 0; s < n_steps;) {
    if (h->j < 2) {
      DNS_TRY(enqueue_rk4_step(h, ff ? h->d_m64 : (double*)h->d_state[h->cur]));
      h->j += 1;
      s += 1;
      continue;
    }
    if (ff && in_m64) {
      dns_split<<<pw_blocks(G), 256, 0, h->stream>>>(G, h->d_m64, (float2*)h->d_state[h->cur]);
      in_m64 = false;
    }
    if (!h->tuned) DNS_TRY(autotune(h));
    if (n_steps - s >= 6) {
      DNS_TRY(launch_six(h));
      s += 6;
    } else {
      DNS_TRY(enqueue_mpea_step(h));
      h->j += 1;
      s += 1;
    }
  }
  if (ff && !in_m64) {
    dns_join<<<pw_blocks(G), 256, 0, h->stream>>>(G, (const float2*)h->d_state[h->cur], M_dev);
  } else {
    const double* src = ff ? h->d_m64 : (const double*)h->d_state[h->cur];
    DNS_CUDA(h, cudaMemcpyAsync(M_dev, src, bytes64, cudaMemcpyDeviceToDevice, h->stream));
  }
  DNS_CUDA(h, cudaGetLastError());
  DNS_CUDA(h, cudaEventRecord(h->ev1, h->stream));
  int err = 0;
  DNS_CUDA(h, cudaMemcpyAsync(&err, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  DNS_CUDA(h, cudaEventRecord(h->ev_out, h->stream));
  DNS_CUDA(h, cudaStreamWaitEvent(h->user, h->ev_out, 0));
  DNS_CUDA(h, cudaStreamSynchronize(h->stream));
  float ms = 0;
  DNS_CUDA(h, cudaEventElapsedTime(&ms, h->ev0, h->ev1));
  h->last_ms = ms;
  if (err) return fail(h, HMM_ERR_NONFINITE, "non-finite value in the direct simulation");
  return HMM_OK;
}

}  // namespace

extern "C" {

hmm_status hmm_dns_init(const hmm_dns_params* params, void* cuda_stream, void** handle_out) {
  if (!params || !handle_out) return fail(nullptr, HMM_ERR_INVALID_ARG, "null params or handle_out");
  *handle_out = nullptr;
  const hmm_dns_params& p = *params;
  if (p.dim < 1 || p.dim > 2) return fail(nullptr, HMM_ERR_INVALID_ARG, "dim must be 1 or 2");
  for (int i = 0; i < 4; ++i)
    if (p.reserved[i] != 0) return fail(nullptr, HMM_ERR_INVALID_ARG, "reserved fields must be zero");
  long long G = 1;
  for (int k = 0; k < p.dim; ++k) {
    if (p.n[k] < 4 || p.n[k] > (1 << 20)) return fail(nullptr, HMM_ERR_INVALID_ARG, "n[k] must be in [4, 2^20]");
    G *= p.n[k];
  }
  if (G > 2147483647LL) return fail(nullptr, HMM_ERR_INVALID_ARG, "too many grid points (G > 2^31 - 1)");
  if (!(p.L > 0)) return fail(nullptr, HMM_ERR_INVALID_ARG, "L must be > 0");
  if (!(p.alpha >= 0 && p.alpha <= 1)) return fail(nullptr, HMM_ERR_INVALID_ARG, "alpha must be in [0, 1]");
  if (!(p.eps > 0)) return fail(nullptr, HMM_ERR_INVALID_ARG, "eps must be > 0");
  if (p.n_terms < 0 || p.n_terms > kMaxTerms) return fail(nullptr, HMM_ERR_INVALID_ARG, "n_terms must be 0..8");
  if (p.n_terms > 0 && !p.terms) return fail(nullptr, HMM_ERR_INVALID_ARG, "terms is NULL");
  const int order = p.stencil_order <= 0 ? 4 : p.stencil_order;
  if (order != 2 && order != 4) return fail(nullptr, HMM_ERR_INVALID_ARG, "stencil_order must be 2 or 4");
  if (p.precision != HMM_FP64_PLAIN && p.precision != HMM_FP32_BATCHED)
    return fail(nullptr, HMM_ERR_INVALID_ARG, "precision must be HMM_FP64_PLAIN or HMM_FP32_BATCHED");
  if (!std::isfinite(p.dt) || !std::isfinite(p.c0)) return fail(nullptr, HMM_ERR_INVALID_ARG, "non-finite dt or c0");
  for (int t = 0; t < p.n_terms; ++t) {
    const hmm_coef_term& T = p.terms[t];
    if (!std::isfinite(T.amp)) return fail(nullptr, HMM_ERR_INVALID_ARG, "non-finite term amplitude");
    for (int k = 0; k < 3; ++k) {
      if (T.kind[k] < 0 || T.kind[k] > 2 || T.scale[k] < 0 || T.scale[k] > 1)
        return fail(nullptr, HMM_ERR_INVALID_ARG, "coefficient term kind/scale out of range");
      if (k >= p.dim && T.kind[k] != 0)
        return fail(nullptr, HMM_ERR_INVALID_ARG, "coefficient factor on an axis beyond dim");
    }
  }
  DnsHandle* h = new DnsHandle();
  h->p = p;
  h->terms.assign(p.terms, p.terms + p.n_terms);
  h->p.terms = nullptr;
  h->user = reinterpret_cast<cudaStream_t>(cuda_stream);
  h->d = p.dim;
  h->order = order;
  h->precision = p.precision;
  h->n0 = p.dim == 2 ? p.n[0] : 1;
  h->n1 = p.dim == 2 ? p.n[1] : p.n[0];
  h->G = G;
  h->dx[0] = p.dim == 2 ? p.L / p.n[0] : 0.0;
  h->dx[1] = p.L / h->n1;
  const double c4 = order == 4 ? 1.0 / 576.0 : 1.0;
  h->base.cx = c4 / (h->dx[1] * h->dx[1]);
  h->base.cy = p.dim == 2 ? c4 / (h->dx[0] * h->dx[0]) : 0.0;
  h->base.alpha = p.alpha;
  h->a_max = p.c0;
  for (const auto& T : h->terms) h->a_max += std::fabs(T.amp);
  auto bail = [&](hmm_status s) {
    g_dns_init_error = h->err;
    free_all(h);
    delete h;
    return s;
  };
  if (!(h->a_max > 0)) { h->err = "coefficient upper bound must be positive"; return bail(HMM_ERR_INVALID_ARG); }
  plan_work(h);
  hmm_status s = build_faces(h);
  if (s != HMM_OK) return bail(s);
  s = pick_dt(h);
  if (s != HMM_OK) return bail(s);
  const size_t st_bytes = h->precision == HMM_FP64_PLAIN ? (size_t)3 * G * sizeof(double) : (size_t)6 * G * sizeof(float);
  const size_t hi_bytes = h->precision == HMM_FP64_PLAIN ? (size_t)3 * G * sizeof(double) : (size_t)3 * G * sizeof(float);
  const size_t b64 = (size_t)3 * G * sizeof(double);
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaMalloc(&h->d_state[i], st_bytes);
  for (int i = 0; i < 3 && e == cudaSuccess; ++i) e = cudaMalloc(&h->d_hist[i], hi_bytes);
  if (e == cudaSuccess && h->precision != HMM_FP64_PLAIN) e = cudaMalloc(&h->d_m64, b64);
  if (e == cudaSuccess) e = cudaMalloc(&h->d_stage, b64);
  if (e == cudaSuccess) e = cudaMalloc(&h->d_H, b64);
  if (e == cudaSuccess) e = cudaMalloc(&h->d_acc, b64);
  if (e == cudaSuccess) e = cudaMalloc(&h->d_err, sizeof(int));
  if (e == cudaSuccess) e = cudaEventCreate(&h->ev0);
  if (e == cudaSuccess) e = cudaEventCreate(&h->ev1);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    cuda_fail(h, e, "hmm_dns_init allocation");
    return bail(e == cudaErrorMemoryAllocation ? HMM_ERR_OUT_OF_MEMORY : HMM_ERR_CUDA);
  }
  *handle_out = h;
  return HMM_OK;
}

hmm_status hmm_dns_set_face_table(void* handle, const double* table_host, long long n_values) {
  DnsHandle* h = as_handle(handle);
  if (!h) return fail(nullptr, HMM_ERR_NOT_INITIALISED, "null handle");
  if (!table_host) return fail(h, HMM_ERR_INVALID_ARG, "null table");
  if (n_values != (long long)h->d * h->G) return fail(h, HMM_ERR_INVALID_ARG, "table length must be dim * G");
  double amax = 0;
  for (long long i = 0; i < n_values; ++i) {
    const double v = table_host[i];
    if (!(v > 0) || !std::isfinite(v)) return fail(h, HMM_ERR_INVALID_ARG, "table values must be positive and finite (A1)");
    amax = std::max(amax, v);
  }
  // library order: fast-axis faces (ax) then slow-axis faces (ay); the table
  // holds block k for axis k, so in 2D block 1 is ax and block 0 is ay
  const long long G = h->G;
  std::vector<double> f64((size_t)2 * G, 1.0);
  if (h->d == 2) {
    std::copy(table_host + G, table_host + 2 * G, f64.begin());
    std::copy(table_host, table_host + G, f64.begin() + G);
  } else {
    std::copy(table_host, table_host + G, f64.begin());
  }
  DNS_CUDA(h, cudaStreamSynchronize(h->stream));
  DNS_TRY(upload_faces(h, f64));
  drop_graphs(h);                 // the graphs hold the old time step
  h->a_max = amax;
  DNS_TRY(pick_dt(h));
  h->j = 0;
  return HMM_OK;
}

hmm_status hmm_dns_step(void* handle, double* M_dev, int n_steps) {
  DnsHandle* h = as_handle(handle);
  if (!h) return fail(nullptr, HMM_ERR_NOT_INITIALISED, "null handle");
  if (!M_dev || n_steps < 0) return fail(h, HMM_ERR_INVALID_ARG, "null M_dev or negative n_steps");
  h->err.clear();
  return run_steps(h, M_dev, n_steps);
}

hmm_status hmm_dns_step_host(void* handle, double* M_host, int n_steps) {
  DnsHandle* h = as_handle(handle);
  if (!h) return fail(nullptr, HMM_ERR_NOT_INITIALISED, "null handle");
  if (!M_host || n_steps < 0) return fail(h, HMM_ERR_INVALID_ARG, "null M_host or negative n_steps");
  h->err.clear();
  const size_t bytes = (size_t)3 * h->G * sizeof(double);
  if (!h->d_host_io) DNS_CUDA(h, cudaMalloc(&h->d_host_io, bytes));
  DNS_CUDA(h, cudaMemcpyAsync(h->d_host_io, M_host, bytes, cudaMemcpyHostToDevice, h->stream));
  DNS_TRY(run_steps(h, h->d_host_io, n_steps));
  DNS_CUDA(h, cudaMemcpyAsync(M_host, h->d_host_io, bytes, cudaMemcpyDeviceToHost, h->stream));
  DNS_CUDA(h, cudaStreamSynchronize(h->stream));
  return HMM_OK;
}

hmm_status hmm_dns_plan(void* handle, int* strips, int* chunk, int* items) {
  DnsHandle* h = as_handle(handle);
  if (!h) return fail(nullptr, HMM_ERR_NOT_INITIALISED, "null handle");
  if (strips) *strips = h->base.strips;
  if (chunk) *chunk = h->base.chunk;
  if (items) *items = h->base.items;
  return HMM_OK;
}

hmm_status hmm_dns_reset(void* handle) {
  DnsHandle* h = as_handle(handle);
  if (!h) return fail(nullptr, HMM_ERR_NOT_INITIALISED, "null handle");
  h->j = 0;
  return HMM_OK;
}

hmm_status hmm_dns_info(void* handle, double* dt, long long* j, double* last_ms) {
  DnsHandle* h = as_handle(handle);
  if (!h) return fail(nullptr, HMM_ERR_NOT_INITIALISED, "null handle");
  if (dt) *dt = h->dt;
  if (j) *j = h->j;
  if (last_ms) *last_ms = h->last_ms;
  return HMM_OK;
}

const char* hmm_dns_last_error(void* handle) {
  DnsHandle* h = as_handle(handle);
  return h ? h->err.c_str() : g_dns_init_error.c_str();
}

void hmm_dns_destroy(void* handle) {
  DnsHandle* h = as_handle(handle);
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  free_all(h);
  delete h;
}

}  // extern "C"

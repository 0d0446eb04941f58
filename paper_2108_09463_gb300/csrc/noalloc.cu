// Allocation-free variant of the batched FP32 micro solve.
//
// Some callers cannot allocate device memory: code running inside a custom
// allocator's callback (where cudaMalloc would re-enter the allocator), or in a
// process whose device memory is fully reserved by another framework. hmm_init allocates
// (box tables, weight tables, per-CTA arenas), so those callers get
// hmm_micro_batch_noalloc instead: it runs the same FP32 micro kernel with every
// buffer it needs carved out of one file-scope device array of fixed size,
// reserved when the library is loaded and held by every GPU that loads it until
// the process exits.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/hmm.h"
#include "hmm_internal.cuh"

namespace hmm {

void set_null_handle_error(const char* msg);
size_t micro_slot_bytes_fp32(int dim, int nmax, int stepper);

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;   // 32 MiB
constexpr int kNoAllocMaxDevices = 64;
constexpr int kNoAllocMaxSteps = 16384;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {

std::mutex g_setup_mutex;
void* g_scratch_addr[kNoAllocMaxDevices] = {};

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Box descriptors of a batch of uniform boxes (one eps, one N), in C order.
__global__ void noalloc_boxes_kernel(BoxDesc* boxes, int P, int dim, int n0, int n1, int n2,
                                     double DX0, double DX1, double DX2, int N, double eps,
                                     double dx, double dt) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  BoxDesc bd;
  const int nm[3] = {n0, n1, n2};
  const double DX[3] = {DX0, DX1, DX2};
  int rem = p;
  for (int k = 2; k >= 0; --k) {
    bd.ci[k] = 0;
    bd.xc[k] = 0.0;
  }
  for (int k = dim - 1; k >= 0; --k) {
    bd.ci[k] = rem % nm[k];
    rem /= nm[k];
  }
  for (int k = 0; k < dim; ++k) bd.xc[k] = bd.ci[k] * DX[k];
  bd.p = p;
  bd.N = N;
  bd.wofs = 0;
  bd.eps = eps;
  bd.dx = dx;
  bd.dt = dt;
  bd.fax = -1;
  boxes[p] = bd;
}

hmm_status noalloc_fail(hmm_status s, const char* msg) {
  set_null_handle_error(msg);
  return s;
}

#define NA_CUDA(call)                                                        \
  do {                                                                       \
    cudaError_t e_ = (call);                                                 \
    if (e_ != cudaSuccess) {                                                 \
      char b_[256];                                                          \
      std::snprintf(b_, sizeof b_, "%s: %s", #call, cudaGetErrorString(e_)); \
      return noalloc_fail(HMM_ERR_CUDA, b_);                                 \
    }                                                                        \
  } while (0)

// The device address of the scratch array on the current device (looked up once
// per device; the lookup is the only set-up and must not run inside a capture).
hmm_status scratch_address(int dev, unsigned char** out) {
  if (dev < 0 || dev >= kNoAllocMaxDevices) return noalloc_fail(HMM_ERR_INVALID_ARG, "device index too large");
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void* ptr = nullptr;
    NA_CUDA(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
    g_scratch_addr[dev] = ptr;
  }
  *out = static_cast<unsigned char*>(g_scratch_addr[dev]);
  return HMM_OK;
}

}  // namespace
}  // namespace hmm

using namespace hmm;

extern "C" hmm_status hmm_micro_batch_noalloc(const hmm_params* params, const double* M_dev,
                                             double* Havg_dev, void* cuda_stream) {
  if (!params || !M_dev || !Havg_dev) return noalloc_fail(HMM_ERR_INVALID_ARG, "null argument");
  {
    // The call copies host data in, reads the error word back and synchronises its
    // stream, so a stream that is being captured is refused before anything is
    // enqueued (the capture stays valid).
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    NA_CUDA(cudaStreamIsCapturing(static_cast<cudaStream_t>(cuda_stream), &cap));
    if (cap != cudaStreamCaptureStatusNone)
      return noalloc_fail(HMM_ERR_INVALID_ARG,
                          "the allocation-free entry point cannot run on a stream that is being captured");
  }
  hmm_params p = *params;
  char msg[256];
  if (p.dim < 1 || p.dim > 3) return noalloc_fail(HMM_ERR_INVALID_ARG, "dim must be 1, 2 or 3");
  if (p.precision != HMM_FP32_BATCHED)
    return noalloc_fail(HMM_ERR_INVALID_ARG, "the allocation-free entry point runs the FP32 form only");
  if (p.eps_field || p.box_n_field)
    return noalloc_fail(HMM_ERR_INVALID_ARG, "the allocation-free entry point needs uniform eps and N");
  if (p.tile_rows != 0 && p.tile_rows != 2 && p.tile_rows != 4)
    return noalloc_fail(HMM_ERR_INVALID_ARG, "tile_rows must be 0, 2 or 4");
  if (p.macro_stepper != HMM_MPEA && p.macro_stepper != HMM_MPE)
    return noalloc_fail(HMM_ERR_INVALID_ARG, "macro_stepper must be 0 (MPEA) or 1 (MPE)");
  if (p.model != HMM_FIELD_MODEL) return noalloc_fail(HMM_ERR_INVALID_ARG, "the allocation-free batch runs the field model");
  if (p.micro_stepper < HMM_HEUNP || p.micro_stepper > HMM_MICRO_MPEA)
    return noalloc_fail(HMM_ERR_INVALID_ARG, "micro_stepper must be 0 (HeunP), 1 (RK4P), 2 (MPE) or 3 (MPEA)");
  if (p.kernel_variant != 0 && p.kernel_variant != 1)
    return noalloc_fail(HMM_ERR_INVALID_ARG, "the allocation-free entry point runs the generic kernel");
  if (!(p.L > 0)) p.L = 1.0;
  if (p.px <= 0) p.px = 3;
  if (p.qx <= 0) p.qx = 7;
  if (p.pt <= 0) p.pt = 3;
  if (p.qt <= 0) p.qt = 7;
  if (p.interp_order <= 0) p.interp_order = 4;
  if (p.stencil_order <= 0) p.stencil_order = 4;
  if (!(p.dt_safety > 0)) p.dt_safety = 0.8;
  if ((p.interp_order != 2 && p.interp_order != 4) || (p.stencil_order != 2 && p.stencil_order != 4))
    return noalloc_fail(HMM_ERR_INVALID_ARG, "interp_order and stencil_order must be 2 or 4");
  if (!(p.alpha > 0 && p.alpha <= 1) || !(p.alpha_micro > 0 && p.alpha_micro <= 4))
    return noalloc_fail(HMM_ERR_INVALID_ARG, "alpha must be in (0, 1] and alpha_micro in (0, 4]");
  if (p.n_terms < 0 || p.n_terms > kMaxTerms || (p.n_terms > 0 && !p.terms))
    return noalloc_fail(HMM_ERR_INVALID_ARG, "n_terms must be 0..8 with a terms array");
  if (!(p.eps > 0) || !(p.pts_per_eps > 0))
    return noalloc_fail(HMM_ERR_INVALID_ARG, "eps and pts_per_eps must be > 0");
  if (p.px > host::kMaxKernelP || p.pt > host::kMaxKernelP || p.qx > 12 || p.qt > 12)
    return noalloc_fail(HMM_ERR_INVALID_ARG, "kernel parameters must satisfy p <= 6, q <= 12");
  if (p.micro_steps < 1 || p.micro_steps > kNoAllocMaxSteps) {
    std::snprintf(msg, sizeof msg, "micro_steps must be 1..%d for the allocation-free entry point",
                  kNoAllocMaxSteps);
    return noalloc_fail(HMM_ERR_INVALID_ARG, msg);
  }
  const int R = p.stencil_order == 2 ? 1 : 3, k = p.interp_order / 2;
  const int nlim = p.dim == 1 ? 1024 : (p.dim == 2 ? 256 : 64);
  const int N = p.box_n;
  if (N < 2 * R + 2 || N > nlim) return noalloc_fail(HMM_ERR_INVALID_ARG, "box_n out of range");
  long long P = 1;
  double DX[3] = {0, 0, 0};
  int nm[3] = {1, 1, 1};
  for (int a = 0; a < p.dim; ++a) {
    if (p.n_macro[a] < 2 * k + 1) return noalloc_fail(HMM_ERR_INVALID_ARG, "n_macro must be >= interp_order + 1");
    nm[a] = p.n_macro[a];
    DX[a] = p.L / p.n_macro[a];
    P *= p.n_macro[a];
  }
  if (P > (1LL << 24)) return noalloc_fail(HMM_ERR_INVALID_ARG, "too many macro points");
  double a_max = p.c0;
  for (int t = 0; t < p.n_terms; ++t) {
    a_max += std::fabs(p.terms[t].amp);
    for (int a = 0; a < 3; ++a)
      if (p.terms[t].kind[a] < 0 || p.terms[t].kind[a] > 2 || p.terms[t].scale[a] < 0 ||
          p.terms[t].scale[a] > 1 || (a >= p.dim && p.terms[t].kind[a] != 0))
        return noalloc_fail(HMM_ERR_INVALID_ARG, "coefficient term kind/scale out of range");
  }
  if (!(a_max > 0)) return noalloc_fail(HMM_ERR_INVALID_ARG, "coefficient upper bound must be positive");

  // Kernels, micro grid and time step: the same host rules as hmm_init.
  double cK[host::kMaxKernelP + 1], cK0[host::kMaxKernelP + 1];
  if (!host::kernel_coeffs(p.px, p.qx, false, cK) || !host::kernel_coeffs(p.pt, p.qt, true, cK0))
    return noalloc_fail(HMM_ERR_INVALID_ARG, "kernel moment system overflowed");
  const double dx = p.eps / p.pts_per_eps;
  const double mup = (N - 1) * dx / 2.0;
  const double mu = p.mu_over_eps > 0 ? p.mu_over_eps * p.eps : 0.8 * mup;
  const double dt = host::micro_dt(p.dt_safety, p.alpha_micro, a_max, p.dim, p.stencil_order, dx, p.micro_stepper);
  if (!(dt > 0)) return noalloc_fail(HMM_ERR_INVALID_ARG, "micro time step is not positive");
  const int M = p.micro_steps;

  // Scratch layout: [queue, error] | boxes | W64 | W32 | w64 | w32 | per-CTA arenas.
  const size_t o_boxes = 256;
  const size_t o_W64 = o_boxes + align256(sizeof(BoxDesc) * (size_t)P);
  const size_t o_W32 = o_W64 + align256(sizeof(double) * N);
  const size_t o_w64 = o_W32 + align256(sizeof(float) * N);
  const size_t o_w32 = o_w64 + align256(sizeof(double) * (M + 1));
  const size_t o_arena = o_w32 + align256(sizeof(float) * (M + 1));
  const size_t slot = micro_slot_bytes_fp32(p.dim, N, p.micro_stepper);
  if (o_arena + slot > kNoAllocScratchBytes) {
    std::snprintf(msg, sizeof msg,
                  "problem needs %zu bytes of scratch for one box; the allocation-free maximum is %zu",
                  o_arena + slot, kNoAllocScratchBytes);
    return noalloc_fail(HMM_ERR_INVALID_ARG, msg);
  }
  const int nslots = (int)((kNoAllocScratchBytes - o_arena) / slot);

  int dev = 0, nsm = 0;
  NA_CUDA(cudaGetDevice(&dev));
  NA_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  unsigned char* base = nullptr;
  hmm_status st = scratch_address(dev, &base);
  if (st != HMM_OK) return st;
  cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);

  // Weight tables, written through a small host buffer in chunks.
  constexpr int kChunk = 512;
  double hb[kChunk];
  float hf[kChunk];
  {
    double s = 0.0;
    for (int j = 0; j < N; ++j) s += host::eval_kernel(cK, p.px, p.qx, ((j - (N - 1) / 2.0) * dx) / mu);
    if (!(s != 0)) return noalloc_fail(HMM_ERR_INVALID_ARG, "spatial weights vanish (mu too small)");
    for (int j0 = 0; j0 < N; j0 += kChunk) {
      const int n = N - j0 < kChunk ? N - j0 : kChunk;
      for (int j = 0; j < n; ++j) {
        hb[j] = host::eval_kernel(cK, p.px, p.qx, (((j0 + j) - (N - 1) / 2.0) * dx) / mu) / s;
        hf[j] = (float)hb[j];
      }
      for (int j = 0; j < n; ++j) {
        const int jj = j0 + j;
        if ((jj < R || jj >= N - R) && hb[j] != 0.0)
          return noalloc_fail(HMM_ERR_INVALID_ARG, "averaging box [-mu, mu] reaches the Dirichlet ring");
      }
      NA_CUDA(cudaMemcpyAsync(base + o_W64 + sizeof(double) * j0, hb, sizeof(double) * n, cudaMemcpyHostToDevice, stream));
      NA_CUDA(cudaMemcpyAsync(base + o_W32 + sizeof(float) * j0, hf, sizeof(float) * n, cudaMemcpyHostToDevice, stream));
    }
    double ws = 0.0;
    for (int n = 0; n <= M; ++n) ws += host::eval_kernel0(cK0, p.pt, p.qt, (double)n / (double)M);
    if (!(ws != 0)) return noalloc_fail(HMM_ERR_INVALID_ARG, "time weights vanish");
    for (int n0 = 0; n0 <= M; n0 += kChunk) {
      const int n = M + 1 - n0 < kChunk ? M + 1 - n0 : kChunk;
      for (int j = 0; j < n; ++j) {
        hb[j] = host::eval_kernel0(cK0, p.pt, p.qt, (double)(n0 + j) / (double)M) / ws;
        hf[j] = (float)hb[j];
      }
      NA_CUDA(cudaMemcpyAsync(base + o_w64 + sizeof(double) * n0, hb, sizeof(double) * n, cudaMemcpyHostToDevice, stream));
      NA_CUDA(cudaMemcpyAsync(base + o_w32 + sizeof(float) * n0, hf, sizeof(float) * n, cudaMemcpyHostToDevice, stream));
    }
  }

  // Box descriptors on the device; queue and error word cleared.
  BoxDesc* boxes = reinterpret_cast<BoxDesc*>(base + o_boxes);
  noalloc_boxes_kernel<<<(int)((P + 255) / 256), 256, 0, stream>>>(boxes, (int)P, p.dim, nm[0], nm[1], nm[2],
                                                                    DX[0], DX[1], DX[2], N, p.eps, dx, dt);
  NA_CUDA(cudaGetLastError());
  NA_CUDA(cudaMemsetAsync(base, 0, 256, stream));

  MicroArgs a{};
  a.boxes = boxes;
  a.n_boxes = (int)P;
  a.queue = reinterpret_cast<int*>(base);
  a.err = reinterpret_cast<int*>(base) + 1;
  a.M = M_dev;
  a.Havg = Havg_dev;
  a.P = (int)P;
  for (int i = 0; i < 3; ++i) {
    a.nmac[i] = nm[i];
    a.DX[i] = DX[i];
  }
  a.interp_k = k;
  a.msteps = M;
  a.stepper = p.micro_stepper;
  a.alpha_micro = p.alpha_micro;
  a.W64 = reinterpret_cast<const double*>(base + o_W64);
  a.W32 = reinterpret_cast<const float*>(base + o_W32);
  a.w64 = reinterpret_cast<const double*>(base + o_w64);
  a.w32 = reinterpret_cast<const float*>(base + o_w32);
  a.om32 = nullptr;   // used by the shared-memory-resident 2D kernel only
  a.c0 = p.c0;
  a.n_terms = p.n_terms;
  for (int t = 0; t < p.n_terms; ++t) {
    a.terms[t].amp = p.terms[t].amp;
    for (int i = 0; i < 3; ++i) {
      a.terms[t].kind[i] = p.terms[t].kind[i];
      a.terms[t].scale[i] = p.terms[t].scale[i];
      a.terms[t].omega[i] = p.terms[t].omega[i];
      a.terms[t].phase[i] = p.terms[t].phase[i];
    }
  }
  a.arena = reinterpret_cast<char*>(base + o_arena);
  a.slot_bytes = slot;
  a.nmax = N;

  const int block = 256;
  const size_t smem = micro_smem_bytes(p.dim, N, k, p.n_terms);
  int per_sm = 0;
  NA_CUDA(prepare_micro_fp32(p.dim, R, block, smem, &per_sm));
  if (per_sm < 1) return noalloc_fail(HMM_ERR_INVALID_ARG, "micro kernel does not fit on an SM");
  long long grid = (long long)per_sm * nsm;
  if (grid > nslots) grid = nslots;
  if (grid > P) grid = P;
  NA_CUDA(launch_micro_fp32(a, p.dim, R, (int)grid, block, smem, stream));

  int err = 0;
  NA_CUDA(cudaMemcpyAsync(&err, base + sizeof(int), sizeof(int), cudaMemcpyDeviceToHost, stream));
  NA_CUDA(cudaStreamSynchronize(stream));
  if (err & kErrCoefNonPositive) return noalloc_fail(HMM_ERR_INVALID_ARG, "coefficient a^eps <= 0 at a micro face (A1)");
  if (err) return noalloc_fail(HMM_ERR_NONFINITE, "non-finite value in the micro solve");
  set_null_handle_error("");   // hmm_last_error(NULL) describes failures only
  return HMM_OK;
}

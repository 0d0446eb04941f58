// Kernels of the direct simulation resolving eps (include/hmm_dns.h).
//
// One warp owns a strip of W = 32 - 2R consecutive nodes of the fast axis
// (R = 1 for order 2, 3 for order 4) and marches down a chunk of rows of the
// slow axis. Lane l holds the node x_l = X0 - R + l of the current row (lanes
// 0..R-1 and 32-R..31 are the strip's halo, taken modulo n with the periodic
// wrap). Along the fast axis the staggered differences take their neighbours
// from the other lanes by warp shuffles; along the slow axis each lane keeps
// its own column's last R+1 rows and the last R+1 face fluxes in registers, so
// a node's y-divergence is complete R rows after it was loaded. No barrier
// wider than the warp is needed.
//
// Rows arrive through a per-warp ring of shared-memory slots that cp.async
// fills two rows ahead of the row being consumed: the state row, the two face
// coefficients that row brings into use, and (time stepping) the history of
// the row it completes. Each lane copies and reads only its own elements.
//
// Face fluxes F_f = a_f * G_f with the raw differences
//   order 4: G_f = (u_{f-1} - u_{f+2}) + 27 (u_{f+1} - u_f),   H += c ((F_{x-2} - F_{x+1}) + 27 (F_x - F_{x-1}))
//   order 2: G_f = u_{f+1} - u_f,                               H += c (F_x - F_{x-1})
// (face f between nodes f and f+1), c = 1/(24 dx)^2 or 1/dx^2 per axis. The
// coefficient a^eps at the faces is a table of G values per axis (built by the
// host from the separable terms, or given by the caller).
//
// In the float-float form (FF) a node is (hi, lo) per component, one float2;
// each difference is taken on hi and lo together with packed FP32x2
// arithmetic and then summed, so that it keeps FP32 accuracy relative to its
// own size instead of to |m|.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

namespace hmm_dns {

constexpr int kWarps = 4;           // warps per block (one work item each)
constexpr int kErrNonFinite = 1;

enum Mode { kField = 0, kMpea64 = 1, kMpeaFF = 2 };

struct Args {
  int n0, n1;            // slow-axis rows (1 for d = 1) and fast-axis columns
  long long G;           // n0 * n1
  int strips, chunk, chunks, items;
  double cx, cy;         // stencil scale along the fast and the slow axis
  // face coefficients: faces along the fast axis (between x and x+1) and along
  // the slow axis (between rows y and y+1), G each, FP64 and FP32 copies
  const double* ax64; const double* ay64;
  const float* ax32; const float* ay32;
  double alpha, half_dt;
  // state
  const double* m64; double* m64_out;                 // kField / kMpea64: 3 x G
  const float2* ff; float2* ff_out;                   // kMpeaFF: 3 x G (hi, lo) pairs
  const void* h1; const void* h2; void* h_out;        // history (double or float, 3 x G)
  double* H_out;                                      // kField: 3 x G
  int* err;
};

template <bool FF> struct Node;
template <> struct Node<false> { double v[3]; };
template <> struct Node<true> { float2 v[3]; };       // (hi, lo)

template <typename T>
__device__ __forceinline__ T shfl_up(T v, int d) { return __shfl_up_sync(0xffffffffu, v, d); }
template <typename T>
__device__ __forceinline__ T shfl_dn(T v, int d) { return __shfl_down_sync(0xffffffffu, v, d); }
__device__ __forceinline__ float2 shfl_up(float2 v, int d) { return make_float2(shfl_up(v.x, d), shfl_up(v.y, d)); }
__device__ __forceinline__ float2 shfl_dn(float2 v, int d) { return make_float2(shfl_dn(v.x, d), shfl_dn(v.y, d)); }

template <bool FF>
__device__ __forceinline__ Node<FF> node_shfl_up(const Node<FF>& a, int d) {
  Node<FF> r;
#pragma unroll
  for (int c = 0; c < 3; ++c) r.v[c] = shfl_up(a.v[c], d);
  return r;
}

template <bool FF>
__device__ __forceinline__ Node<FF> node_shfl_dn(const Node<FF>& a, int d) {
  Node<FF> r;
#pragma unroll
  for (int c = 0; c < 3; ++c) r.v[c] = shfl_dn(a.v[c], d);
  return r;
}

__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }

// Raw face difference of component c: order 4 from (u_{f-1}, u_f, u_{f+1}, u_{f+2}),
// order 2 from (u_f, u_{f+1}) passed as (b, c1).
template <int ORDER, bool FF>
__device__ __forceinline__ auto face_diff(const Node<FF>& a, const Node<FF>& b, const Node<FF>& c1,
                                          const Node<FF>& d, int c) {
  if constexpr (FF) {
    if constexpr (ORDER == 4) {
      const float2 g = __ffma2_rn(make_float2(27.f, 27.f), sub2(c1.v[c], b.v[c]), sub2(a.v[c], d.v[c]));
      return g.x + g.y;
    } else {
      const float2 g = sub2(c1.v[c], b.v[c]);
      return g.x + g.y;
    }
  } else {
    if constexpr (ORDER == 4) return (a.v[c] - d.v[c]) + 27.0 * (c1.v[c] - b.v[c]);
    else return c1.v[c] - b.v[c];
  }
}

template <bool FF>
__device__ __forceinline__ Node<FF> load_node(const Args& A, long long idx) {
  Node<FF> r;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if constexpr (FF) r.v[c] = __ldg(A.ff + c * A.G + idx);
    else r.v[c] = __ldg(A.m64 + c * A.G + idx);
  }
  return r;
}

// Asynchronous global -> shared copies (cp.async, cached in L1 and L2) and
// their group bookkeeping. Each lane copies and later reads only its own
// elements, so the group waits are the only synchronisation needed.
__device__ __forceinline__ void cp_async(void* smem, const void* gmem, int bytes) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  if (bytes == 8) asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(gmem) : "memory");
  else asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// x-part of H at the lane's node (raw, unscaled) from the row's nodes `u`,
// the divergence of the face fluxes; valid on lanes R..31-R.
template <int ORDER, bool FF, typename R_>
__device__ __forceinline__ void x_part(const Node<FF>& u, R_ ax, R_ out[3]) {
  Node<FF> um1, up1, up2;
  if constexpr (ORDER == 4) {
    um1 = node_shfl_up<FF>(u, 1);
    up1 = node_shfl_dn<FF>(u, 1);
    up2 = node_shfl_dn<FF>(u, 2);
  } else {
    up1 = node_shfl_dn<FF>(u, 1);
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    R_ F = ax * face_diff<ORDER, FF>(um1, u, up1, up2, c);
    if constexpr (ORDER == 4) {
      R_ Fm2 = shfl_up(F, 2), Fm1 = shfl_up(F, 1), Fp1 = shfl_dn(F, 1);
      out[c] = (Fm2 - Fp1) + R_(27) * (F - Fm1);
    } else {
      R_ Fm1 = shfl_up(F, 1);
      out[c] = F - Fm1;
    }
  }
}

template <int ORDER, bool TWO_D, int MODE>
__global__ void __launch_bounds__(32 * kWarps, (MODE == kMpeaFF) ? 7 : 4) dns_kernel(Args A) {
  constexpr bool FF = (MODE == kMpeaFF);
  using R_ = typename std::conditional<FF, float, double>::type;
  using S_ = typename std::conditional<FF, float2, double>::type;   // state element
  constexpr int RR = (ORDER == 4) ? 3 : 1;
  constexpr int W = 32 - 2 * RR;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int item = blockIdx.x * kWarps + wib;
  if (item >= A.items) return;                      // whole warp leaves together
  const int strip = item % A.strips;
  const int chunk = item / A.strips;
  const int n0 = A.n0, n1 = A.n1;
  int xl = strip * W - RR + lane;                   // lane's node on the fast axis
  const bool out_lane = lane >= RR && lane < 32 - RR && xl < n1;
  xl = (xl % n1 + n1) % n1;
  const int r0 = TWO_D ? chunk * A.chunk : 0;
  const int r1 = TWO_D ? min(r0 + A.chunk, n0) : 1;
  const S_* state = FF ? reinterpret_cast<const S_*>(A.ff) : reinterpret_cast<const S_*>(A.m64);
  const R_* AX = FF ? reinterpret_cast<const R_*>(A.ax32) : reinterpret_cast<const R_*>(A.ax64);
  const R_* AY = FF ? reinterpret_cast<const R_*>(A.ay32) : reinterpret_cast<const R_*>(A.ay64);

  // Rolling state of the own column: rows q-R..q and the last R+1 y-face fluxes
  // (order 4: faces q-5..q-2, order 2: faces q-2..q-1), oldest first.
  Node<FF> win[RR + 1];
  R_ fq[RR + 1][3];
#pragma unroll
  for (int k = 0; k <= RR; ++k) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      fq[k][c] = R_(0);
      if constexpr (FF) win[k].v[c] = make_float2(0.f, 0.f);
      else win[k].v[c] = 0.0;
    }
  }
  // q in [r0 - R, r1 + R) and n0 >= 4 > R: one add or subtract wraps it
  auto wrap = [&](int q) { return q < 0 ? q + n0 : (q >= n0 ? q - n0 : q); };
  // The ring: DEPTH slots per warp; the slot of state row q also holds a_y of
  // the face row q brings into use (q-2 for order 4, q-1 for order 2), and a_x
  // and the history of the row q completes, q - R, when that row is an output.
  constexpr int DEPTH = 3;
  constexpr int HD = (MODE == kField) ? 1 : DEPTH;
  constexpr int WK = TWO_D ? kWarps : 1;
  __shared__ S_ s_st[WK][TWO_D ? DEPTH : 1][3][32];
  __shared__ R_ s_a[WK][TWO_D ? DEPTH : 1][2][32];
  __shared__ R_ s_h[WK][TWO_D ? HD : 1][2][3][32];
  const int q_first = r0 - RR, q_last = TWO_D ? r1 - 1 + RR : 0;
  // Rows are issued in increasing order q = q_first, q_first + 1, ...: their
  // wrapped row and face row advance by one add and a compare per row, and the
  // ring slot of the row being consumed rotates.
  int irow = TWO_D ? wrap(q_first) : 0;
  int ifrow = TWO_D ? wrap(ORDER == 4 ? q_first - 2 : q_first - 1) : 0;
  int cslot = DEPTH - 1;                             // slot of the row last consumed
  auto issue = [&](int q, int sl) {
    if (q <= q_last) {
      const long long idx = (long long)irow * n1 + xl;
#pragma unroll
      for (int c = 0; c < 3; ++c) cp_async(&s_st[wib][sl][c][lane], state + c * A.G + idx, 8);
      if (q >= r0) cp_async(&s_a[wib][sl][1][lane], AY + (long long)ifrow * n1 + xl, (int)sizeof(R_));
      const int pr = q - RR;
      if (pr >= r0 && pr < r1) {
        const long long gi = (long long)pr * n1 + xl;
        cp_async(&s_a[wib][sl][0][lane], AX + gi, (int)sizeof(R_));
        if constexpr (MODE != kField) {
          const R_* H1 = reinterpret_cast<const R_*>(A.h1);
          const R_* H2 = reinterpret_cast<const R_*>(A.h2);
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            cp_async(&s_h[wib][sl % HD][0][c][lane], H1 + c * A.G + gi, (int)sizeof(R_));
            cp_async(&s_h[wib][sl % HD][1][c][lane], H2 + c * A.G + gi, (int)sizeof(R_));
          }
        }
      }
    }
    cp_async_commit();      // one group per row, empty past the last row
    irow = irow + 1 == n0 ? 0 : irow + 1;
    ifrow = ifrow + 1 == n0 ? 0 : ifrow + 1;
  };
  auto push_row = [&](int q) {
#pragma unroll
    for (int k = 0; k < RR; ++k) win[k] = win[k + 1];
    if constexpr (TWO_D) {
      cslot = cslot == DEPTH - 1 ? 0 : cslot + 1;    // row q's slot
      cp_async_wait<DEPTH - 2>();                    // row q's group is complete
#pragma unroll
      for (int c = 0; c < 3; ++c) win[RR].v[c] = s_st[wib][cslot][c][lane];
      issue(q + DEPTH - 1, cslot == 0 ? DEPTH - 1 : cslot - 1);   // into the slot row q - 1 used
    } else {
      win[RR] = load_node<FF>(A, xl);
    }
  };
  // y-face flux from the full window: order 4 the face between rows q-2 and q-1
  // (rows q-3..q), order 2 the face between rows q-1 and q
  auto push_face = [&](int q) {
    const R_ ay = s_a[wib][cslot][1][lane];
#pragma unroll
    for (int k = 0; k < RR; ++k)
#pragma unroll
      for (int c = 0; c < 3; ++c) fq[k][c] = fq[k + 1][c];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      if constexpr (ORDER == 4) fq[RR][c] = ay * face_diff<4, FF>(win[0], win[1], win[2], win[3], c);
      else fq[RR][c] = ay * face_diff<2, FF>(win[0], win[0], win[1], win[1], c);
    }
  };
  // H at the lane's node of row p (node values u), then the point's update.
  auto emit = [&](int p, const Node<FF>& u) {
    const long long gi = (long long)p * n1 + xl;
    const long long G = A.G;
    R_ ax, hp1[3], hp2[3];                           // a_x, h^{j-1}, h^{j-2}
    if constexpr (TWO_D) {
      const int sl = cslot;                          // arrived with state row p + R
      ax = s_a[wib][sl][0][lane];
      if constexpr (MODE != kField) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          hp1[c] = s_h[wib][sl % HD][0][c][lane];
          hp2[c] = s_h[wib][sl % HD][1][c][lane];
        }
      }
    } else {
      ax = __ldg(AX + gi);
      if constexpr (MODE != kField) {
        const R_* H1 = reinterpret_cast<const R_*>(A.h1);
        const R_* H2 = reinterpret_cast<const R_*>(A.h2);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          hp1[c] = __ldg(H1 + c * G + gi);
          hp2[c] = __ldg(H2 + c * G + gi);
        }
      }
    }
    R_ H[3];
    x_part<ORDER, FF, R_>(u, ax, H);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      R_ hy = R_(0);
      if constexpr (TWO_D) {
        if constexpr (ORDER == 4) hy = (fq[0][c] - fq[3][c]) + R_(27) * (fq[2][c] - fq[1][c]);
        else hy = fq[1][c] - fq[0][c];
      }
      H[c] = R_(A.cx) * H[c] + R_(A.cy) * hy;
    }
    if (!out_lane) return;
    if constexpr (MODE == kField) {
#pragma unroll
      for (int c = 0; c < 3; ++c) A.H_out[c * G + gi] = H[c];
    } else {
      R_ m[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        if constexpr (FF) m[c] = u.v[c].x;
        else m[c] = u.v[c];
      }
      const R_ al = R_(A.alpha);
      // h^j = H + alpha m x H (eq. h_term)
      R_ h[3];
      h[0] = H[0] + al * (m[1] * H[2] - m[2] * H[1]);
      h[1] = H[1] + al * (m[2] * H[0] - m[0] * H[2]);
      h[2] = H[2] + al * (m[0] * H[1] - m[1] * H[0]);
      R_* HO = reinterpret_cast<R_*>(A.h_out);
      const R_ c23 = R_(23.0 / 12.0), c16 = R_(16.0 / 12.0), c5 = R_(5.0 / 12.0);
      R_ w[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        R_ hh = (c23 * h[c] - c16 * hp1[c]) + c5 * hp2[c];
        w[c] = R_(A.half_dt) * hh;
        HO[c * G + gi] = h[c];
      }
      // midpoint update (eq. mpe_update) in closed form
      R_ a0 = w[1] * m[2] - w[2] * m[1];
      R_ a1 = w[2] * m[0] - w[0] * m[2];
      R_ a2 = w[0] * m[1] - w[1] * m[0];
      R_ b0 = w[1] * a2 - w[2] * a1;
      R_ b1 = w[2] * a0 - w[0] * a2;
      R_ b2 = w[0] * a1 - w[1] * a0;
      R_ f;
      if constexpr (FF) f = __fdividef(2.f, 1.f + (w[0] * w[0] + w[1] * w[1] + w[2] * w[2]));   // 2 ulp
      else f = 2.0 / (1.0 + (w[0] * w[0] + w[1] * w[1] + w[2] * w[2]));
      R_ dl[3] = {f * (a0 + b0), f * (a1 + b1), f * (a2 + b2)};
      bool bad = false;
      if constexpr (FF) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          float s, e;
          two_sum(u.v[c].x, dl[c], s, e);
          float lo = u.v[c].y + e;
          float hi = s + lo;
          lo = lo - (hi - s);
          A.ff_out[c * G + gi] = make_float2(hi, lo);
          bad |= !isfinite(hi);
        }
      } else {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          double v = u.v[c] + dl[c];
          A.m64_out[c * G + gi] = v;
          bad |= !isfinite(v);
        }
      }
      if (bad) atomicOr(A.err, kErrNonFinite);
    }
  };

  if constexpr (!TWO_D) {
    push_row(0);
    emit(0, win[RR]);
    (void)q_first;
    (void)q_last;
  } else {
    // rows r0-R..r0-1 fill the window; rows r0..r0+R-1 also push their faces;
    // from row r0+R on each new row completes row p = q - R (p in [r0, r1))
#pragma unroll
    for (int k = 0; k < DEPTH - 1; ++k) issue(q_first + k, k);
    for (int q = r0 - RR; q < r0; ++q) push_row(q);
    for (int q = r0; q < r0 + RR; ++q) {
      push_row(q);
      push_face(q);
    }
    for (int q = r0 + RR; q < r1 + RR; ++q) {
      push_row(q);
      push_face(q);
      emit(q - RR, win[0]);
    }
  }
}

}  // namespace hmm_dns

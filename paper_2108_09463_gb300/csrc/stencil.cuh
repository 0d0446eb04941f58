// Staggered conservative stencil H = div(a grad m) and the Landau-Lifshitz
// right-hand side, shared by the FP64 and FP32 micro kernels.
//
// Along axis k, with faces j+1/2 between nodes j and j+1:
//   order 2 (R = 1): G_{j+1/2} = m_{j+1} - m_j,           H_i += F_{i+1/2} - F_{i-1/2}
//   order 4 (R = 3): G_{j+1/2} = m_{j-1} - 27 m_j + 27 m_{j+1} - m_{j+2},
//                    H_i += F_{i-3/2} - 27 F_{i-1/2} + 27 F_{i+1/2} - F_{i+3/2}
// with F = a_f G and the factor 1/dx^2 (order 2) or 1/(24 dx)^2 (order 4)
// applied once at the end ("cs").
#pragma once
#include "micro_common.cuh"

namespace hmm {

template <int R, typename T>
__device__ __forceinline__ T axis_div(const T* __restrict__ m, const T* __restrict__ a, int idx,
                                      int s) {
  if (R == 1) {
    const T m_1 = m[idx - s], m0 = m[idx], m1 = m[idx + s];
    return a[idx] * (m1 - m0) - a[idx - s] * (m0 - m_1);
  } else {
    const T m_3 = m[idx - 3 * s], m_2 = m[idx - 2 * s], m_1 = m[idx - s], m0 = m[idx];
    const T m1 = m[idx + s], m2 = m[idx + 2 * s], m3 = m[idx + 3 * s];
    const T g_2 = (m_3 - m0) + T(27) * (m_1 - m_2);   // face i-3/2
    const T g_1 = (m_2 - m1) + T(27) * (m0 - m_1);    // face i-1/2
    const T g0 = (m_1 - m2) + T(27) * (m1 - m0);      // face i+1/2
    const T g1 = (m0 - m3) + T(27) * (m2 - m1);       // face i+3/2
    const T F_2 = a[idx - 2 * s] * g_2, F_1 = a[idx - s] * g_1;
    const T F0 = a[idx] * g0, F1 = a[idx + s] * g1;
    return (F_2 - F1) + T(27) * (F0 - F_1);
  }
}

// H at node idx for the 3 components (SoA planes of stride cap).
template <int D, int R, typename T>
__device__ __forceinline__ void stencil_H(const T* __restrict__ m, const T* __restrict__ af,
                                          size_t cap, const Strides<D>& st, int idx, T cs, T* H) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const T* mc = m + c * cap;
    T acc = axis_div<R, T>(mc, af, idx, st.s[0]);
#pragma unroll
    for (int k = 1; k < D; ++k) acc += axis_div<R, T>(mc, af + k * cap, idx, st.s[k]);
    H[c] = acc * cs;
  }
}

// Flux model sites: the faces along axis k that touch an interior node, faces
// j_k + 1/2 with j_k = R-1 .. N-R-1, at interior nodes along the other axes;
// t in [0, (N-2R+1)(N-2R)^(D-1)). Returns the index of the face's lower node and
// its per-axis node coordinates in j.
template <int D, int R>
__device__ __forceinline__ int flux_site(int t, int N, int k, int* j) {
  const int Ni = N - 2 * R, Nk = Ni + 1;
  int rem = t, idx = 0;
#pragma unroll
  for (int ax = D - 1; ax >= 0; --ax) {
    const int n = ax == k ? Nk : Ni;
    const int q = rem % n;
    rem /= n;
    j[ax] = ax == k ? q + R - 1 : q + R;
  }
#pragma unroll
  for (int ax = 0; ax < D; ++ax) idx = idx * N + j[ax];
  return idx;
}

// The face flux a_f D_s m along axis k (stride s) at the face between node idx
// and idx + s, times 1/(24 dx) (order 4) or 1/dx (order 2) ("cf"), 3 components.
template <int R, typename T>
__device__ __forceinline__ void face_flux(const T* __restrict__ m, const T* __restrict__ ak, size_t cap, int idx,
                                          int s, T cf, T* F) {
  const T a = ak[idx] * cf;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const T* mc = m + c * cap;
    T g;
    if (R == 1) g = mc[idx + s] - mc[idx];
    else g = (mc[idx - s] - mc[idx + 2 * s]) + T(27) * (mc[idx + s] - mc[idx]);
    F[c] = a * g;
  }
}

// f = -m x H - alpha m x (m x H)   (Section 3.1)
template <typename T>
__device__ __forceinline__ void ll_rhs(const T* m, const T* H, T alpha, T* f) {
  const T p0 = m[1] * H[2] - m[2] * H[1];
  const T p1 = m[2] * H[0] - m[0] * H[2];
  const T p2 = m[0] * H[1] - m[1] * H[0];
  const T d0 = m[1] * p2 - m[2] * p1;
  const T d1 = m[2] * p0 - m[0] * p2;
  const T d2 = m[0] * p1 - m[1] * p0;
  f[0] = -p0 - alpha * d0;
  f[1] = -p1 - alpha * d1;
  f[2] = -p2 - alpha * d2;
}

}  // namespace hmm

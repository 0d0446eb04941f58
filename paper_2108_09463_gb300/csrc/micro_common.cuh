// Device helpers shared by the FP64 and FP32 micro-batch kernels.
//
// One CTA solves one micro problem at a time and pulls the next box from an
// atomic work queue (boxes are sorted longest first). Per box:
//   1. per-axis Lagrange weights of the micro nodes (Section 4.1, eq. Q_k),
//   2. the (2k+1)^d macro neighbourhood with periodic wrap,
//   3. m_init = P/|P| at every node, contracting one axis after the other,
//   4. per-axis 1D tables of the coefficient factors, then a^eps at every face.
#pragma once
#include "hmm_internal.cuh"

namespace hmm {

// Node-array strides for a box with N nodes per axis, last axis fastest.
template <int D>
struct Strides {
  int s[3];
  __device__ explicit Strides(int N) {
    s[D - 1] = 1;
    if (D > 1) s[D - 2] = N;
    if (D > 2) s[0] = N * N;
  }
};

template <int D>
__device__ __forceinline__ int ipow(int n) {
  return D == 1 ? n : (D == 2 ? n * n : n * n * n);
}

// Linear node index of the t-th interior node (interior = [R, N-R)^D).
template <int D, int R>
__device__ __forceinline__ int interior_node(int t, int N) {
  const int Ni = N - 2 * R;
  if (D == 1) return t + R;
  if (D == 2) {
    const int i0 = t / Ni, i1 = t - i0 * Ni;
    return (i0 + R) * N + (i1 + R);
  }
  const int i0 = t / (Ni * Ni);
  const int rem = t - i0 * Ni * Ni;
  const int i1 = rem / Ni, i2 = rem - i1 * Ni;
  return ((i0 + R) * N + (i1 + R)) * N + (i2 + R);
}

template <int D>
__device__ __forceinline__ void node_coords(int idx, int N, int* j) {
  if (D == 1) { j[0] = idx; return; }
  if (D == 2) { j[0] = idx / N; j[1] = idx - j[0] * N; return; }
  j[0] = idx / (N * N);
  const int rem = idx - j[0] * N * N;
  j[1] = rem / N;
  j[2] = rem - j[1] * N;
}

// Fetch the next box index for this CTA (all threads get the same value).
__device__ __forceinline__ int next_box(int* queue, int* s_slot) {
  __syncthreads();
  if (threadIdx.x == 0) *s_slot = atomicAdd(queue, 1);
  __syncthreads();
  return *s_slot;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum of three doubles; result valid in thread 0. scratch >= 3*32 doubles.
__device__ __forceinline__ void block_sum3(double& x, double& y, double& z, double* scratch) {
  x = warp_sum(x);
  y = warp_sum(y);
  z = warp_sum(z);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) {
    scratch[wid] = x;
    scratch[32 + wid] = y;
    scratch[64 + wid] = z;
  }
  __syncthreads();
  if (wid == 0) {
    x = lane < nw ? scratch[lane] : 0.0;
    y = lane < nw ? scratch[32 + lane] : 0.0;
    z = lane < nw ? scratch[64 + lane] : 0.0;
    x = warp_sum(x);
    y = warp_sum(y);
    z = warp_sum(z);
  }
}

// Shared-memory layout for the per-box set-up tables (doubles).
struct SetupSmem {
  double* lag;    // [D][N][2k+1]   Lagrange weights of node j along each axis
  double* neigh;  // [3][(2k+1)^D]  macro neighbourhood
  double* part;   // [3][(2k+1)^(D-1)][N] neighbourhood contracted along the last axis
  double* ctab;   // [n_terms][D][2N-1] coefficient factors at node and half-node positions
  double* red;    // [96] reduction scratch
};

__host__ __device__ inline size_t setup_smem_doubles(int D, int nmax, int k, int n_terms) {
  const int w = 2 * k + 1;
  int wd = 1, wd1 = 1;
  for (int i = 0; i < D; ++i) wd *= w;
  for (int i = 0; i < D - 1; ++i) wd1 *= w;
  return (size_t)D * nmax * w + 3 * wd + 3 * (size_t)wd1 * nmax +
         (size_t)(n_terms > 0 ? n_terms : 1) * D * (2 * nmax - 1) + 96;
}

__device__ inline SetupSmem carve_setup(double* base, int D, int nmax, int k, int n_terms) {
  const int w = 2 * k + 1;
  int wd = 1, wd1 = 1;
  for (int i = 0; i < D; ++i) wd *= w;
  for (int i = 0; i < D - 1; ++i) wd1 *= w;
  SetupSmem s;
  s.lag = base;
  s.neigh = s.lag + (size_t)D * nmax * w;
  s.part = s.neigh + 3 * wd;
  s.ctab = s.part + 3 * (size_t)wd1 * nmax;
  s.red = s.ctab + (size_t)(n_terms > 0 ? n_terms : 1) * D * (2 * nmax - 1);
  return s;
}

// Coordinates of micro node j (half = 1: of the face j+1/2): (j + half/2 - (N-1)/2) dx.
__device__ __forceinline__ double node_offset(int j2, int N, double dx) {
  // j2 is twice the node position (2j or 2j+1); (j2 - (N-1))/2 is exact.
  return __dmul_rn(0.5 * (double)(j2 - (N - 1)), dx);
}

// Set-up part 1: Lagrange weights, neighbourhood, contraction, coefficient tables.
template <int D>
__device__ void box_setup_tables(const MicroArgs& a, const BoxDesc& bd, const SetupSmem& sm) {
  const int N = bd.N, k = a.interp_k, w = 2 * k + 1;
  const int tid = threadIdx.x, nt = blockDim.x;
  // Lagrange basis l_a(s), s = xi_j / DX, nodes -k..k (Section 4.1); a flux box
  // centred at x_i + (DX_k/2) e_k evaluates the same interpolant at s + 1/2 on axis k.
  for (int e = tid; e < D * N; e += nt) {
    const int ax = e / N, j = e - ax * N;
    const double s = node_offset(2 * j, N, bd.dx) / a.DX[ax] + (ax == bd.fax ? 0.5 : 0.0);
    for (int ia = 0; ia < w; ++ia) {
      double v = 1.0;
      for (int ib = 0; ib < w; ++ib)
        if (ib != ia) v *= (s - (double)(ib - k)) / (double)(ia - ib);
      sm.lag[(size_t)e * w + ia] = v;
    }
  }
  // Macro neighbourhood M_{i+a}, periodic wrap.
  int wd = 1;
  for (int i = 0; i < D; ++i) wd *= w;
  for (int e = tid; e < 3 * wd; e += nt) {
    const int c = e / wd;
    int r = e - c * wd;
    int lin = 0;
    int off[3] = {0, 0, 0};
    for (int ax = D - 1; ax >= 0; --ax) {
      off[ax] = r % w;
      r /= w;
    }
    for (int ax = 0; ax < D; ++ax) {
      int ii = bd.ci[ax] + off[ax] - k;
      ii %= a.nmac[ax];
      if (ii < 0) ii += a.nmac[ax];
      lin = lin * a.nmac[ax] + ii;
    }
    sm.neigh[e] = a.M[(size_t)c * a.P + lin];
  }
  // Coefficient factor tables at node (even) and half-node (odd) positions.
  const int nh = 2 * N - 1;
  for (int e = tid; e < a.n_terms * D * nh; e += nt) {
    const int t = e / (D * nh);
    const int rem = e - t * D * nh;
    const int ax = rem / nh, j2 = rem - ax * nh;
    const TermDev& T = a.terms[t];
    double g = 1.0;
    if (T.kind[ax] != 0) {
      const double x = __dadd_rn(bd.xc[ax], node_offset(j2, N, bd.dx));
      const double s = T.scale[ax] == 0 ? x / bd.eps : x;
      const double th = __dadd_rn(__dmul_rn(__dmul_rn(__dmul_rn(2.0, kPi), T.omega[ax]), s), T.phase[ax]);
      g = T.kind[ax] == 1 ? sin(th) : cos(th);
    }
    sm.ctab[e] = g;
  }
  __syncthreads();
  // Contract the neighbourhood along the last axis: part[c][a'][j] = sum_b l_b(j) M[c][a'][b].
  int wd1 = wd / w;
  const double* lagL = sm.lag + (size_t)(D - 1) * N * w;
  for (int e = tid; e < 3 * wd1 * N; e += nt) {
    const int j = e % N;
    const int cb = e / N;  // c * wd1 + a'
    double acc = 0.0;
    for (int b = 0; b < w; ++b) acc += lagL[j * w + b] * sm.neigh[(size_t)cb * w + b];
    sm.part[e] = acc;
  }
  __syncthreads();
}

// P_[2k] at node idx (the remaining axes contracted from the partial sums).
template <int D>
__device__ __forceinline__ void interp_P(const MicroArgs& a, const SetupSmem& sm, int N, int idx,
                                         double* P) {
  const int w = 2 * a.interp_k + 1;
  int j[3];
  node_coords<D>(idx, N, j);
  int wd1 = 1;
  for (int i = 0; i < D - 1; ++i) wd1 *= w;
  const int jl = j[D - 1];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const double* pc = sm.part + (size_t)c * wd1 * N;
    double acc;
    if (D == 1) {
      acc = pc[jl];
    } else if (D == 2) {
      const double* l0 = sm.lag + (size_t)j[0] * w;
      acc = 0.0;
      for (int a0 = 0; a0 < w; ++a0) acc += l0[a0] * pc[(size_t)a0 * N + jl];
    } else {
      const double* l0 = sm.lag + (size_t)j[0] * w;
      const double* l1 = sm.lag + ((size_t)N + j[1]) * w;
      acc = 0.0;
      for (int a0 = 0; a0 < w; ++a0) {
        double inner = 0.0;
        for (int a1 = 0; a1 < w; ++a1) inner += l1[a1] * pc[((size_t)a0 * w + a1) * N + jl];
        acc += l0[a0] * inner;
      }
    }
    P[c] = acc;
  }
}

// a^eps at the face between node idx and its +1 neighbour along axis k.
template <int D>
__device__ __forceinline__ double face_coef(const MicroArgs& a, const SetupSmem& sm, int N, int idx,
                                            int k) {
  int j[3];
  node_coords<D>(idx, N, j);
  const int nh = 2 * N - 1;
  double out = a.c0;
  for (int t = 0; t < a.n_terms; ++t) {
    double v = a.terms[t].amp;
#pragma unroll
    for (int ax = 0; ax < D; ++ax) {
      const int j2 = 2 * j[ax] + (ax == k ? 1 : 0);
      v = __dmul_rn(v, sm.ctab[((size_t)t * D + ax) * nh + j2]);
    }
    out = __dadd_rn(out, v);
  }
  return out;
}

// a^eps at the face between node idx of box bd and its +1 neighbour along axis k:
// from the caller's table when one is set (macro point bd.p's block, d sub-blocks of
// N^d values), else from the separable terms.
template <int D>
__device__ __forceinline__ double face_value(const MicroArgs& a, const BoxDesc& bd, const SetupSmem& sm, int N,
                                             int idx, int k) {
  if (a.faces) return a.faces[a.face_off[bd.p] + (long long)k * ipow<D>(N) + idx];
  return face_coef<D>(a, sm, N, idx, k);
}

}  // namespace hmm

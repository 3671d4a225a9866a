// Patch sweep and matrix-free operator kernels, templated on dimension and
// degree, for one scalar type GMG_T (this header is included once per type by
// patch_f64.cu / patch_f32.cu, each with its own __constant__ tables).
//
// All level operators are written for unit-width cells: on a level with
// h = 1/n, A = h^{d-2} A_ref and A_j^{-1} = h^{2-d} A_ref,j^{-1}, so the
// coefficient tables do not depend on the level.
//
// Patch local_update (Sec. 3.1; Algorithm 4 runs it for every patch of one
// colour per launch):
//   gather    closure bar u_j ((2k+1)^d nodes) into shared memory
//   evaluate  r = h^{2-d} b_j - [A_ref bar u_j]_interior by sum factorisation
//             over the patch: the patch operator is a sum of tensor products
//             of the two-cell 1D matrices M_p, K_p (interior rows x closure
//             columns, banded: a row touches one cell, or two at the vertex)
//   solve     d = (T x .. x T) diag(1/sum lambda) (T x .. x T)^T r
//             (fast diagonalisation, App. A.3)
//   scatter   u_interior += omega d  (same-colour interiors are disjoint)
#pragma once
#include <cuda_runtime.h>

#include "kernels.h"

#ifndef GMG_T
#error "define GMG_T before including patch_kernels.cuh"
#endif

namespace gmg {
namespace GMG_NS {

using T = GMG_T;

__host__ __device__ constexpr int cmax(int a, int b) { return a > b ? a : b; }
// compact per-degree offsets of the coefficient tables (degree k = 1..8)
__host__ __device__ constexpr int off_patch(int k) { return k <= 1 ? 0 : off_patch(k - 1) + (2 * k - 3) * (2 * k - 1); }
__host__ __device__ constexpr int off_t(int k) { return k <= 1 ? 0 : off_t(k - 1) + (2 * k - 3) * (2 * k - 3); }
__host__ __device__ constexpr int off_cell(int k) { return k <= 1 ? 0 : off_cell(k - 1) + k * k; }
constexpr int kPatchTotal = off_patch(9);
constexpr int kTTotal = off_t(9);
constexpr int kCellTotal = off_cell(9);

// two-cell patch matrices, rows = interior closure rows 1..2k-1, cols 0..2k
__constant__ T c_Mp[kPatchTotal];
__constant__ T c_Kp[kPatchTotal];
// fast-diagonalisation eigenvectors T[i][j] (row = node, column = mode)
__constant__ T c_T[kTTotal];
// unit-cell 1D mass and stiffness ((k+1)^2)
__constant__ T c_Mc[kCellTotal];
__constant__ T c_Kc[kCellTotal];

// band of closure row c (1..2k-1) of the two-cell patch matrices
__host__ __device__ constexpr int band_lo(int c, int K) { return c > K ? K : 0; }
__host__ __device__ constexpr int band_hi(int c, int K) { return c < K ? K : 2 * K; }

template <int DIM, int K>
struct PatchDims {
  static constexpr int C = 2 * K + 1;
  static constexpr int M = 2 * K - 1;
  static constexpr int NCLO = DIM == 3 ? C * C * C : C * C;
  static constexpr int NINT = DIM == 3 ? M * M * M : M * M;
  // buffer A: closure, then (3D) the stage-y results, (2D) r and the FD work
  static constexpr int SA = DIM == 3 ? cmax(C * C * C, 2 * C * M * M) : C * C;
  // buffer B: stage-z (3D) / stage-y (2D) results, then (3D) r and FD work
  static constexpr int SB = DIM == 3 ? cmax(2 * C * C * M, M * M * M) : 2 * C * M;
  static constexpr int SMEM_BYTES = (SA + SB) * (int)sizeof(T);
};

// acc + sign * sum_j E[i][j] x[j] over the band of closure row i+1 of a
// two-cell patch table E (compile-time offset); i = 0..M-1
template <int K, bool NEG = false>
__device__ __forceinline__ T patch_row(const T* E, int i, const T (&x)[2 * K + 1], T acc = T(0)) {
  constexpr int C = 2 * K + 1;
#pragma unroll
  for (int j = 0; j < C; ++j) {
    if (j >= band_lo(i + 1, K) && j <= band_hi(i + 1, K))
      acc = fma(NEG ? -E[i * C + j] : E[i * C + j], x[j], acc);
  }
  return acc;
}

// FD transform along one axis, in place on a line of M = 2K-1 values at
// stride s, using the mirror symmetry of the eigenvectors: modes 0..K-1 are
// even (T[M-1-j][i] = T[j][i]), modes K..M-1 odd (T[M-1-j][i] = -T[j][i]).
// forward (TRANSPOSE = true): y_i = sum_j T[j][i] x_j
// backward:                   x_j = sum_i T[j][i] y_i
template <int K, bool TRANSPOSE>
__device__ __forceinline__ void fd_line(T* base, int s) {
  constexpr int M = 2 * K - 1, c = K - 1;
  const T* Tm = c_T + off_t(K);
  if (TRANSPOSE) {
    T sv[K], dv[K > 1 ? K - 1 : 1];
#pragma unroll
    for (int j = 0; j < c; ++j) {
      T a = base[j * s], b = base[(M - 1 - j) * s];
      sv[j] = a + b;
      dv[j] = a - b;
    }
    sv[c] = base[c * s];
#pragma unroll
    for (int i = 0; i < K; ++i) {  // even modes
      T acc = T(0);
#pragma unroll
      for (int j = 0; j <= c; ++j) acc = fma(Tm[j * M + i], sv[j], acc);
      base[i * s] = acc;
    }
#pragma unroll
    for (int i = K; i < M; ++i) {  // odd modes
      T acc = T(0);
#pragma unroll
      for (int j = 0; j < c; ++j) acc = fma(Tm[j * M + i], dv[j], acc);
      base[i * s] = acc;
    }
  } else {
    T y[M];
#pragma unroll
    for (int i = 0; i < M; ++i) y[i] = base[i * s];
#pragma unroll
    for (int j = 0; j < c; ++j) {
      T e = T(0), o = T(0);
#pragma unroll
      for (int i = 0; i < K; ++i) e = fma(Tm[j * M + i], y[i], e);
#pragma unroll
      for (int i = K; i < M; ++i) o = fma(Tm[j * M + i], y[i], o);
      base[j * s] = e + o;
      base[(M - 1 - j) * s] = e - o;
    }
    T e = T(0);
#pragma unroll
    for (int i = 0; i < K; ++i) e = fma(Tm[c * M + i], y[i], e);
    base[c * s] = e;
  }
}

// Apply the FD transform along every axis of the M^DIM blocks of PPC patches
// (block q at R + q * stride).
template <int DIM, int K, bool TRANSPOSE, int NT, int PPC>
__device__ __forceinline__ void fd_all_axes(T* R, int stride, const bool* valid) {
  constexpr int M = 2 * K - 1;
  constexpr int L = DIM == 3 ? M * M : M;
#pragma unroll
  for (int axis = 0; axis < DIM; ++axis) {
    for (int idx = threadIdx.x; idx < PPC * L; idx += NT) {
      const int q = idx / L, l = idx % L;
      if (!valid[q]) continue;
      T* Rq = R + q * stride;
      if (DIM == 2) {
        if (axis == 0) fd_line<K, TRANSPOSE>(Rq + l * M, 1);
        else fd_line<K, TRANSPOSE>(Rq + l, M);
      } else {
        if (axis == 0) fd_line<K, TRANSPOSE>(Rq + l * M, 1);
        else if (axis == 1) fd_line<K, TRANSPOSE>(Rq + (l % M) + (l / M) * M * M, M);
        else fd_line<K, TRANSPOSE>(Rq + l, M * M);
      }
    }
    __syncthreads();
  }
}

// One colour of the sweep: each CTA takes PPC consecutive patches of the
// colour; every stage distributes the lines of all its patches over the
// threads, so partial warps are rare.
template <int DIM, int K, int NT, int PPC>
__global__ void __launch_bounds__(NT) patch_colour_kernel(T* __restrict__ u, const T* __restrict__ b,
                                                          const T* __restrict__ dinv, PatchLaunch pl) {
  using D = PatchDims<DIM, K>;
  constexpr int C = D::C, M = D::M;
  constexpr int STRIDE = D::SA + D::SB;  // elements of shared memory per patch
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* const S = reinterpret_cast<T*>(smem_raw);
  __shared__ long long s_origin[PPC];
  __shared__ bool s_valid[PPC];
  const T* Mp = c_Mp + off_patch(K);
  const T* Kp = c_Kp + off_patch(K);
  const long long py = pl.g.py, pz = pl.g.pz;
  const T sb = (T)pl.sb;
  const T om = (T)pl.omega;
  const int ngroups = (pl.n_patches + PPC - 1) / PPC;

  for (int grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
    if (threadIdx.x < PPC) {
      const int pid = grp * PPC + threadIdx.x;
      const bool ok = pid < pl.n_patches;
      int i0 = 0, i1 = 0, i2 = 0;
      if (ok) {
        i0 = pid % pl.count[0];
        const int rest = pid / pl.count[0];
        i1 = rest % pl.count[1];
        i2 = DIM == 3 ? rest / pl.count[1] : 0;
      }
      const long long o0 = (long long)(pl.first[0] + 2 * i0 - 1) * K;
      const long long o1 = (long long)(pl.first[1] + 2 * i1 - 1) * K;
      const long long o2 = DIM == 3 ? (long long)(pl.first[2] + 2 * i2 - 1) * K : 0;
      s_origin[threadIdx.x] = o0 + py * o1 + pz * o2;
      s_valid[threadIdx.x] = ok;
    }
    __syncthreads();

    // ---- gather the closures (eq. "gather") ----
    for (int idx = threadIdx.x; idx < PPC * D::NCLO; idx += NT) {
      const int q = idx / D::NCLO, t = idx % D::NCLO;
      if (!s_valid[q]) continue;
      const int x = t % C, y = (t / C) % C, z = DIM == 3 ? t / (C * C) : 0;
      S[q * STRIDE + t] = u[s_origin[q] + x + py * y + pz * z];
    }
    __syncthreads();

    if (DIM == 3) {
      // ---- stage z: P = Mp_z u, Q = Kp_z u   (dims x:C, y:C, z:M, in B) ----
      for (int idx = threadIdx.x; idx < PPC * C * C; idx += NT) {
        const int q = idx / (C * C), l = idx % (C * C);
        if (!s_valid[q]) continue;
        const T* A = S + q * STRIDE;
        T* B = S + q * STRIDE + D::SA;
        T x[C];
#pragma unroll
        for (int j = 0; j < C; ++j) x[j] = A[l + j * C * C];
#pragma unroll
        for (int i = 0; i < M; ++i) {
          B[l + i * C * C] = patch_row<K>(Mp, i, x);
          B[C * C * M + l + i * C * C] = patch_row<K>(Kp, i, x);
        }
      }
      __syncthreads();
      // ---- stage y: A1 = Mp_y P, A2 = Kp_y P + Mp_y Q   (dims x:C, y:M, z:M, in A) ----
      for (int idx = threadIdx.x; idx < PPC * C * M; idx += NT) {
        const int q = idx / (C * M), l = idx % (C * M);
        if (!s_valid[q]) continue;
        T* A = S + q * STRIDE;
        const T* B = S + q * STRIDE + D::SA;
        const int x0 = l % C, z = l / C;
        T p[C], r[C];
#pragma unroll
        for (int j = 0; j < C; ++j) {
          p[j] = B[x0 + j * C + z * C * C];
          r[j] = B[C * C * M + x0 + j * C + z * C * C];
        }
#pragma unroll
        for (int i = 0; i < M; ++i) {
          A[x0 + i * C + z * C * M] = patch_row<K>(Mp, i, p);
          A[C * M * M + x0 + i * C + z * C * M] = patch_row<K>(Mp, i, r, patch_row<K>(Kp, i, p));
        }
      }
      __syncthreads();
      // ---- stage x: r = sb b - (Kp_x A1 + Mp_x A2)   (dims M^3, into B) ----
      for (int idx = threadIdx.x; idx < PPC * M * M; idx += NT) {
        const int q = idx / (M * M), l = idx % (M * M);
        if (!s_valid[q]) continue;
        const T* A = S + q * STRIDE;
        T* B = S + q * STRIDE + D::SA;
        const int y = l % M, z = l / M;
        T a1[C], a2[C];
#pragma unroll
        for (int j = 0; j < C; ++j) {
          a1[j] = A[j + C * (y + M * z)];
          a2[j] = A[C * M * M + j + C * (y + M * z)];
        }
        const long long row = s_origin[q] + 1 + py * (y + 1) + pz * (z + 1);
#pragma unroll
        for (int i = 0; i < M; ++i) {
          T acc = sb * b[row + i];
          acc = patch_row<K, true>(Kp, i, a1, acc);
          B[i + M * l] = patch_row<K, true>(Mp, i, a2, acc);
        }
      }
      __syncthreads();
    } else {
      // ---- stage y: P = Mp_y u, Q = Kp_y u   (dims x:C, y:M, into B) ----
      for (int idx = threadIdx.x; idx < PPC * C; idx += NT) {
        const int q = idx / C, l = idx % C;
        if (!s_valid[q]) continue;
        const T* A = S + q * STRIDE;
        T* B = S + q * STRIDE + D::SA;
        T x[C];
#pragma unroll
        for (int j = 0; j < C; ++j) x[j] = A[l + j * C];
#pragma unroll
        for (int i = 0; i < M; ++i) {
          B[l + i * C] = patch_row<K>(Mp, i, x);
          B[C * M + l + i * C] = patch_row<K>(Kp, i, x);
        }
      }
      __syncthreads();
      // ---- stage x: r = sb b - (Kp_x P + Mp_x Q)   (dims M^2, into A: the
      // closure is consumed) ----
      for (int idx = threadIdx.x; idx < PPC * M; idx += NT) {
        const int q = idx / M, l = idx % M;
        if (!s_valid[q]) continue;
        T* A = S + q * STRIDE;
        const T* B = S + q * STRIDE + D::SA;
        T p[C], r[C];
#pragma unroll
        for (int j = 0; j < C; ++j) {
          p[j] = B[j + C * l];
          r[j] = B[C * M + j + C * l];
        }
        const long long row = s_origin[q] + 1 + py * (l + 1);
#pragma unroll
        for (int i = 0; i < M; ++i) {
          T acc = sb * b[row + i];
          acc = patch_row<K, true>(Kp, i, p, acc);
          A[i + M * l] = patch_row<K, true>(Mp, i, r, acc);
        }
      }
      __syncthreads();
    }

    // ---- local solve by fast diagonalisation, in place ----
    T* R0 = DIM == 3 ? S + D::SA : S;  // r of patch 0 (3D: buffer B, 2D: buffer A)
    fd_all_axes<DIM, K, true, NT, PPC>(R0, STRIDE, s_valid);
    for (int idx = threadIdx.x; idx < PPC * D::NINT; idx += NT) {
      const int q = idx / D::NINT, t = idx % D::NINT;
      if (s_valid[q]) R0[q * STRIDE + t] *= dinv[t];
    }
    __syncthreads();
    fd_all_axes<DIM, K, false, NT, PPC>(R0, STRIDE, s_valid);

    // ---- scatter (eq. "scatter"): u_interior += omega d ----
    for (int idx = threadIdx.x; idx < PPC * D::NINT; idx += NT) {
      const int q = idx / D::NINT, t = idx % D::NINT;
      if (!s_valid[q]) continue;
      const int x = t % M, y = (t / M) % M;
      long long g = s_origin[q] + (x + 1) + py * (y + 1);
      if (DIM == 3) g += pz * (t / (M * M) + 1);
      u[g] = fma(om, R0[q * STRIDE + t], u[g]);
    }
    __syncthreads();  // shared buffers and s_origin are reused by the next group
  }
}

// ---------------------------------------------------------------------------
// Matrix-free level operator on a tile of BC cells per direction.
// Global 1D matrix row for node i = c K + p: p > 0 -> cell c row p;
// p == 0 (vertex) -> cell c-1 row K plus cell c row 0.
// Tile inputs: nodes [(c0-1)K, (c0+BC)K] (EI per direction, zero outside the
// lattice); outputs: nodes [c0 K, (c0+BC) K) (EO per direction).
template <int K, int EI>
__device__ __forceinline__ T cell_row(const T* E, int o, const T (&x)[EI]) {
  const int p = o % K;
  T acc = T(0);
  if (p == 0) {
#pragma unroll
    for (int q = 0; q <= K; ++q) acc = fma(E[K * (K + 1) + q], x[o + q], acc);
#pragma unroll
    for (int q = 0; q <= K; ++q) acc = fma(E[q], x[o + K + q], acc);
  } else {
#pragma unroll
    for (int q = 0; q <= K; ++q) acc = fma(E[p * (K + 1) + q], x[o - p + K + q], acc);
  }
  return acc;
}

template <int DIM, int K, int BC>
struct ApplyDims {
  static constexpr int EI = (BC + 1) * K + 1;
  static constexpr int EO = BC * K;
  static constexpr int SA = DIM == 3 ? cmax(EI * EI * EI, 2 * EI * EO * EO) : EI * EI;
  static constexpr int SB = DIM == 3 ? 2 * EI * EI * EO : 2 * EI * EO;
  static constexpr int SMEM_BYTES = (SA + SB) * (int)sizeof(T);
};

template <int DIM, int K, int BC, int NT>
__global__ void __launch_bounds__(NT) apply_kernel(const T* __restrict__ xin, T* __restrict__ y,
                                                   const T* __restrict__ bvec, ApplyLaunch al) {
  using D = ApplyDims<DIM, K, BC>;
  constexpr int EI = D::EI, EO = D::EO;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* A = reinterpret_cast<T*>(smem_raw);
  T* B = A + D::SA;
  const T* Mc = c_Mc + off_cell(K);
  const T* Kc = c_Kc + off_cell(K);
  const int N = al.g.N, n = al.g.n;
  const long long py = al.g.py, pz = al.g.pz;
  const int tiles = (n + BC - 1) / BC;
  const int ntile = DIM == 3 ? tiles * tiles * tiles : tiles * tiles;
  const T alpha = (T)al.alpha, beta = (T)al.beta;

  for (int tid = blockIdx.x; tid < ntile; tid += gridDim.x) {
    const int t0 = tid % tiles, t1 = (tid / tiles) % tiles, t2 = DIM == 3 ? tid / (tiles * tiles) : 0;
    const int g0 = (t0 * BC - 1) * K, g1 = (t1 * BC - 1) * K, g2 = DIM == 3 ? (t2 * BC - 1) * K : 0;
    // gather the tile with zero fill outside the lattice
    const int nin = DIM == 3 ? EI * EI * EI : EI * EI;
    for (int t = threadIdx.x; t < nin; t += NT) {
      int x = t % EI, yy = (t / EI) % EI, z = DIM == 3 ? t / (EI * EI) : 0;
      int gx = g0 + x, gy = g1 + yy, gz = g2 + z;
      bool ok = gx >= 0 && gx < N && gy >= 0 && gy < N && (DIM == 2 || (gz >= 0 && gz < N));
      A[t] = ok ? xin[gx + py * gy + pz * gz] : T(0);
    }
    __syncthreads();
    if (DIM == 3) {
      // stage z: P = M_z x, Q = K_z x   (x:EI, y:EI, z:EO)
      for (int l = threadIdx.x; l < EI * EI; l += NT) {
        T v[EI];
#pragma unroll
        for (int j = 0; j < EI; ++j) v[j] = A[l + j * EI * EI];
#pragma unroll
        for (int o = 0; o < EO; ++o) {
          B[l + o * EI * EI] = cell_row<K, EI>(Mc, o, v);
          B[EI * EI * EO + l + o * EI * EI] = cell_row<K, EI>(Kc, o, v);
        }
      }
      __syncthreads();
      // stage y: A1 = M_y P, A2 = K_y P + M_y Q   (x:EI, y:EO, z:EO)
      for (int l = threadIdx.x; l < EI * EO; l += NT) {
        int x0 = l % EI, z = l / EI;
        T p[EI], q[EI];
#pragma unroll
        for (int j = 0; j < EI; ++j) {
          p[j] = B[x0 + j * EI + z * EI * EI];
          q[j] = B[EI * EI * EO + x0 + j * EI + z * EI * EI];
        }
#pragma unroll
        for (int o = 0; o < EO; ++o) {
          A[x0 + o * EI + z * EI * EO] = cell_row<K, EI>(Mc, o, p);
          A[EI * EO * EO + x0 + o * EI + z * EI * EO] = cell_row<K, EI>(Kc, o, p) + cell_row<K, EI>(Mc, o, q);
        }
      }
      __syncthreads();
      // stage x and write: y = alpha (K_x A1 + M_x A2) + beta b on owned interior nodes
      for (int l = threadIdx.x; l < EO * EO; l += NT) {
        int yy = l % EO, z = l / EO;
        int gy = g1 + K + yy, gz = g2 + K + z;
        if (gy <= 0 || gy >= N - 1 || gz <= 0 || gz >= N - 1) continue;
        T a1[EI], a2[EI];
#pragma unroll
        for (int j = 0; j < EI; ++j) {
          a1[j] = A[j + EI * (yy + EO * z)];
          a2[j] = A[EI * EO * EO + j + EI * (yy + EO * z)];
        }
        const long long row = py * gy + pz * gz;
#pragma unroll
        for (int o = 0; o < EO; ++o) {
          int gx = g0 + K + o;
          if (gx <= 0 || gx >= N - 1) continue;
          T v = alpha * (cell_row<K, EI>(Kc, o, a1) + cell_row<K, EI>(Mc, o, a2));
          if (bvec) v += beta * bvec[row + gx];
          y[row + gx] = v;
        }
      }
    } else {
      // stage y: P = M_y x, Q = K_y x   (x:EI, y:EO)
      for (int l = threadIdx.x; l < EI; l += NT) {
        T v[EI];
#pragma unroll
        for (int j = 0; j < EI; ++j) v[j] = A[l + j * EI];
#pragma unroll
        for (int o = 0; o < EO; ++o) {
          B[l + o * EI] = cell_row<K, EI>(Mc, o, v);
          B[EI * EO + l + o * EI] = cell_row<K, EI>(Kc, o, v);
        }
      }
      __syncthreads();
      for (int l = threadIdx.x; l < EO; l += NT) {
        int gy = g1 + K + l;
        if (gy <= 0 || gy >= N - 1) continue;
        T p[EI], q[EI];
#pragma unroll
        for (int j = 0; j < EI; ++j) {
          p[j] = B[j + EI * l];
          q[j] = B[EI * EO + j + EI * l];
        }
        const long long row = py * gy;
#pragma unroll
        for (int o = 0; o < EO; ++o) {
          int gx = g0 + K + o;
          if (gx <= 0 || gx >= N - 1) continue;
          T v = alpha * (cell_row<K, EI>(Kc, o, p) + cell_row<K, EI>(Mc, o, q));
          if (bvec) v += beta * bvec[row + gx];
          y[row + gx] = v;
        }
      }
    }
    __syncthreads();
  }
}

}  // namespace GMG_NS
}  // namespace gmg

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
#include <cuda.h>
#include <cuda_runtime.h>

#include "../../include/gmg.h"
#include "async.cuh"
#include "df_arith.cuh"
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
// the eigenvectors c_T split into float pairs hi + lo (double-float FD
// transforms of FP64 problems; unused by FP32 problems)
__constant__ float c_Thi[kTTotal];
__constant__ float c_Tlo[kTTotal];
// the two-cell patch matrices split the same way (double-float residual and
// face terms of FP64 problems)
__constant__ float c_Mphi[kPatchTotal];
__constant__ float c_Mplo[kPatchTotal];
__constant__ float c_Kphi[kPatchTotal];
__constant__ float c_Kplo[kPatchTotal];
// and the unit-cell matrices (double-float three-pass operator)
__constant__ float c_Mchi[kCellTotal];
__constant__ float c_Mclo[kCellTotal];
__constant__ float c_Kchi[kCellTotal];
__constant__ float c_Kclo[kCellTotal];

// band of closure row c (1..2k-1) of the two-cell patch matrices
__host__ __device__ constexpr int band_lo(int c, int K) { return c > K ? K : 0; }
__host__ __device__ constexpr int band_hi(int c, int K) { return c < K ? K : 2 * K; }


// acc + sign * sum_j E[i][j] x[j] over the band of closure row i+1 of the
// two-cell patch matrix E = M_p (KIND 0) or K_p (KIND 1); i = 0..M-1.  The
// __constant__ tables are indexed directly with compile-time offsets so that
// every coefficient is an immediate constant-bank operand.
template <int K, int KIND, bool NEG = false>
__device__ __forceinline__ T patch_row(int i, const T (&x)[2 * K + 1], T acc = T(0)) {
  constexpr int C = 2 * K + 1;
#pragma unroll
  for (int j = 0; j < C; ++j) {
    if (j >= band_lo(i + 1, K) && j <= band_hi(i + 1, K)) {
      const T e = KIND == 0 ? c_Mp[off_patch(K) + i * C + j] : c_Kp[off_patch(K) + i * C + j];
      acc = fma(NEG ? -e : e, x[j], acc);
    }
  }
  return acc;
}

// The same row restricted to the two end columns 0 and 2K of the closure
// (a closure line whose other entries are taken as zero).
template <int K, int KIND>
__device__ __forceinline__ T patch_row_ends(int i, T x0, T xc) {
  constexpr int C = 2 * K + 1;
  T acc = T(0);
  if (band_lo(i + 1, K) == 0)
    acc = (KIND == 0 ? c_Mp[off_patch(K) + i * C] : c_Kp[off_patch(K) + i * C]) * x0;
  if (band_hi(i + 1, K) == 2 * K)
    acc = fma(KIND == 0 ? c_Mp[off_patch(K) + i * C + C - 1] : c_Kp[off_patch(K) + i * C + C - 1], xc, acc);
  return acc;
}

// FD transforms of one line of M = 2K-1 values held in registers, using the
// mirror symmetry of the eigenvectors: modes 0..K-1 are even
// (T[M-1-j][i] = T[j][i]), modes K..M-1 odd (T[M-1-j][i] = -T[j][i]).
// forward: y_i = sum_j T[j][i] x_j;   backward: x_j = sum_i T[j][i] y_i
template <int K>
__device__ __forceinline__ void fd_forward(const T (&x)[2 * K - 1], T (&y)[2 * K - 1]) {
  constexpr int M = 2 * K - 1, c = K - 1;
    T sv[K], dv[K > 1 ? K - 1 : 1];
#pragma unroll
  for (int j = 0; j < c; ++j) {
    sv[j] = x[j] + x[M - 1 - j];
    dv[j] = x[j] - x[M - 1 - j];
  }
  sv[c] = x[c];
#pragma unroll
  for (int i = 0; i < K; ++i) {
    T acc = T(0);
#pragma unroll
    for (int j = 0; j <= c; ++j) acc = fma(c_T[off_t(K) + j * M + i], sv[j], acc);
    y[i] = acc;
  }
#pragma unroll
  for (int i = K; i < M; ++i) {
    T acc = T(0);
#pragma unroll
    for (int j = 0; j < c; ++j) acc = fma(c_T[off_t(K) + j * M + i], dv[j], acc);
    y[i] = acc;
  }
}

template <int K>
__device__ __forceinline__ void fd_backward(const T (&y)[2 * K - 1], T (&x)[2 * K - 1]) {
  constexpr int M = 2 * K - 1, c = K - 1;
  #pragma unroll
  for (int j = 0; j < c; ++j) {
    T e = T(0), o = T(0);
#pragma unroll
    for (int i = 0; i < K; ++i) e = fma(c_T[off_t(K) + j * M + i], y[i], e);
#pragma unroll
    for (int i = K; i < M; ++i) o = fma(c_T[off_t(K) + j * M + i], y[i], o);
    x[j] = e + o;
    x[M - 1 - j] = e - o;
  }
  T e = T(0);
#pragma unroll
  for (int i = 0; i < K; ++i) e = fma(c_T[off_t(K) + c * M + i], y[i], e);
  x[c] = e;
}

// FD transform of a shared-memory line in place (stride s); with SCALE the
// result is multiplied elementwise by d[0], d[ds], ... (the diagonal).
template <int K, bool FORWARD, bool SCALE = false>
__device__ __forceinline__ void fd_smem_line(T* base, int s, const T* __restrict__ d = nullptr,
                                             int ds = 0) {
  constexpr int M = 2 * K - 1;
  T in[M], out[M];
#pragma unroll
  for (int j = 0; j < M; ++j) in[j] = base[j * s];
  if (FORWARD) fd_forward<K>(in, out);
  else fd_backward<K>(in, out);
#pragma unroll
  for (int j = 0; j < M; ++j) base[j * s] = SCALE ? out[j] * __ldg(d + j * ds) : out[j];
}

// The innermost transform pair of the FD solve on one shared-memory line
// (stride s) in registers: forward transform, times the diagonal d[0], d[ds],
// ..., backward transform.
template <int K>
__device__ __forceinline__ void fd_smem_line_solve(T* base, int s, const T* __restrict__ d, int ds) {
  constexpr int M = 2 * K - 1;
  T v[M], w[M];
#pragma unroll
  for (int j = 0; j < M; ++j) v[j] = base[j * s];
  fd_forward<K>(v, w);
#pragma unroll
  for (int j = 0; j < M; ++j) w[j] *= __ldg(d + j * ds);
  fd_backward<K>(w, v);
#pragma unroll
  for (int j = 0; j < M; ++j) base[j * s] = v[j];
}

// the FD transforms of fd_forward / fd_backward in double-float arithmetic
// (same mirror-symmetric even/odd splitting, eigenvectors from c_Thi/c_Tlo)
template <int K>
__device__ __forceinline__ void fd_forward_df(const dfv (&x)[2 * K - 1], dfv (&y)[2 * K - 1]) {
  constexpr int M = 2 * K - 1, c = K - 1;
  dfv sv[K], dv[K > 1 ? K - 1 : 1];
#pragma unroll
  for (int j = 0; j < c; ++j) {
    sv[j] = df_add(x[j], x[M - 1 - j]);
    dv[j] = df_add(x[j], df_neg(x[M - 1 - j]));
  }
  sv[c] = x[c];
#pragma unroll
  for (int i = 0; i < K; ++i) {
    df_acc acc = df_acc_first(c_Thi[off_t(K) + i], c_Tlo[off_t(K) + i], sv[0]);
#pragma unroll
    for (int j = 1; j <= c; ++j) df_acc_add(acc, c_Thi[off_t(K) + j * M + i], c_Tlo[off_t(K) + j * M + i], sv[j]);
    y[i] = df_acc_value(acc);
  }
#pragma unroll
  for (int i = K; i < M; ++i) {
    df_acc acc = df_acc_first(c_Thi[off_t(K) + i], c_Tlo[off_t(K) + i], dv[0]);
#pragma unroll
    for (int j = 1; j < c; ++j) df_acc_add(acc, c_Thi[off_t(K) + j * M + i], c_Tlo[off_t(K) + j * M + i], dv[j]);
    y[i] = df_acc_value(acc);
  }
}

template <int K>
__device__ __forceinline__ void fd_backward_df(const dfv (&y)[2 * K - 1], dfv (&x)[2 * K - 1]) {
  constexpr int M = 2 * K - 1, c = K - 1;
#pragma unroll
  for (int j = 0; j < c; ++j) {
    df_acc e = df_acc_first(c_Thi[off_t(K) + j * M], c_Tlo[off_t(K) + j * M], y[0]);
#pragma unroll
    for (int i = 1; i < K; ++i) df_acc_add(e, c_Thi[off_t(K) + j * M + i], c_Tlo[off_t(K) + j * M + i], y[i]);
    df_acc o = df_acc_first(c_Thi[off_t(K) + j * M + K], c_Tlo[off_t(K) + j * M + K], y[K]);
#pragma unroll
    for (int i = K + 1; i < M; ++i) df_acc_add(o, c_Thi[off_t(K) + j * M + i], c_Tlo[off_t(K) + j * M + i], y[i]);
    const dfv ev = df_acc_value(e), ov = df_acc_value(o);
    x[j] = df_add(ev, ov);
    x[M - 1 - j] = df_add(ev, df_neg(ov));
  }
  df_acc e = df_acc_first(c_Thi[off_t(K) + c * M], c_Tlo[off_t(K) + c * M], y[0]);
#pragma unroll
  for (int i = 1; i < K; ++i) df_acc_add(e, c_Thi[off_t(K) + c * M + i], c_Tlo[off_t(K) + c * M + i], y[i]);
  x[c] = df_acc_value(e);
}

// entry (i, j) of the two-cell patch matrix M_p (KIND 0) or K_p (KIND 1) as
// a float pair, negated with NEG
template <int K, int KIND, bool NEG = false>
__device__ __forceinline__ void patch_entry_df(int i, int j, float& hi, float& lo) {
  constexpr int C = 2 * K + 1;
  const int o = off_patch(K) + i * C + j;
  hi = KIND == 0 ? c_Mphi[o] : c_Kphi[o];
  lo = KIND == 0 ? c_Mplo[o] : c_Kplo[o];
  if (NEG) {
    hi = -hi;
    lo = -lo;
  }
}

// acc += (or -= with NEG) sum_j E[i][j] x[j] over the band of closure row
// i+1 of E = M_p (KIND 0) or K_p (KIND 1), double-float (Dot2)
template <int K, int KIND, bool NEG = false>
__device__ __forceinline__ void patch_row_df(int i, const dfv (&x)[2 * K + 1], df_acc& acc) {
  constexpr int C = 2 * K + 1;
#pragma unroll
  for (int j = 0; j < C; ++j) {
    if (j >= band_lo(i + 1, K) && j <= band_hi(i + 1, K)) {
      float h, l;
      patch_entry_df<K, KIND, NEG>(i, j, h, l);
      df_acc_add(acc, h, l, x[j]);
    }
  }
}

// the same over the interior columns 1..2K-1 (x[a] at closure column a + 1)
template <int K, int KIND>
__device__ __forceinline__ void patch_row_int_df(int i, const dfv (&x)[2 * K - 1], df_acc& acc) {
  constexpr int M = 2 * K - 1;
#pragma unroll
  for (int a = 0; a < M; ++a) {
    if (a + 1 >= band_lo(i + 1, K) && a + 1 <= band_hi(i + 1, K)) {
      float h, l;
      patch_entry_df<K, KIND>(i, a + 1, h, l);
      df_acc_add(acc, h, l, x[a]);
    }
  }
}

// double-float FD transform of a shared-memory line (pairs, stride s) in place
template <int K, bool FORWARD>
__device__ __forceinline__ void fd_smem_line_df(float2* base, int s) {
  constexpr int M = 2 * K - 1;
  dfv in[M], out[M];
#pragma unroll
  for (int j = 0; j < M; ++j) {
    const float2 v = base[j * s];
    in[j] = {v.x, v.y};
  }
  if (FORWARD) fd_forward_df<K>(in, out);
  else fd_backward_df<K>(in, out);
#pragma unroll
  for (int j = 0; j < M; ++j) base[j * s] = make_float2(out[j].hi, out[j].lo);
}

// the innermost transform pair in double-float: forward, times the diagonal
// d[0], d[ds], ... (float pairs), backward
template <int K>
__device__ __forceinline__ void fd_smem_line_solve_df(float2* base, int s, const float2* __restrict__ d, int ds) {
  constexpr int M = 2 * K - 1;
  dfv v[M], w[M];
#pragma unroll
  for (int j = 0; j < M; ++j) {
    const float2 a = base[j * s];
    v[j] = {a.x, a.y};
  }
  fd_forward_df<K>(v, w);
#pragma unroll
  for (int j = 0; j < M; ++j) {
    const float2 dj = __ldg(d + j * ds);
    w[j] = df_mul(w[j], {dj.x, dj.y});
  }
  fd_backward_df<K>(w, v);
#pragma unroll
  for (int j = 0; j < M; ++j) base[j * s] = make_float2(v[j].hi, v[j].lo);
}

// Asynchronous global -> shared copy of one element (cp.async, cached in L1),
// and the group commit / wait of the copies issued by this thread.
__device__ __forceinline__ void async_copy(T* smem_dst, const T* gmem_src) {
  const unsigned dst = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(dst), "l"(gmem_src), "n"(sizeof(T)));
}
__device__ __forceinline__ void async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// Shared-memory plan of the sweep kernel, per patch (elements):
//   IN  (NBUF copies): closure of u, then interior of b, rows of XU / XB
//       elements ([z][y][x]); with the TMA gather (TMA = true) a row is the
//       TMA box width: C (resp. M + 1) plus the alignment shift, rounded up to
//       16 bytes, and each box starts on 128 bytes
//   WA  3D: stage-y results A1, A2;  2D: stage-y results P, Q
//   WB  3D: stage-z results P, Q, then r and the FD work;  2D: r and FD work
// Stage x always reads WA and writes WB.
template <int DIM, int K, bool TMA = false>
struct SweepSmem {
  static constexpr int C = 2 * K + 1, M = 2 * K - 1;
  static constexpr int A = 16 / (int)sizeof(T);  // elements per 16 bytes
  static constexpr int XU = TMA ? (C + A - 1 + A - 1) / A * A : C;
  static constexpr int XB = TMA ? XU : M;
  static constexpr int R128 = 128 / (int)sizeof(T);
  static constexpr int rnd(int n) { return TMA ? (n + R128 - 1) / R128 * R128 : n; }
  static constexpr int NCLO = rnd(DIM == 3 ? C * C * XU : C * XU);
  static constexpr int NBIN = rnd(DIM == 3 ? M * M * XB : M * XB);
  static constexpr int NINT = DIM == 3 ? M * M * M : M * M;
  static constexpr int IN = NCLO + NBIN;
  static constexpr int WA = DIM == 3 ? 2 * C * M * M : 2 * C * M;
  static constexpr int WB = DIM == 3 ? cmax(2 * C * C * M, M * M * M) : M * M;
  static constexpr int per_patch(int nbuf) { return nbuf * IN + WA + WB; }
  // TMA box bytes of the closure of u and of the interior rows of b
  static constexpr int BOX_U = (DIM == 3 ? C * C * XU : C * XU) * (int)sizeof(T);
  static constexpr int BOX_B = (DIM == 3 ? M * M * XB : M * XB) * (int)sizeof(T);
};

// Tensor maps of the u and b vectors of each table entry (TMA gather).
template <int ME>
struct TmaMaps {
  CUtensorMap u[ME], b[ME];
};
template <>
struct TmaMaps<0> {};

// One colour of the sweep.  Persistent CTAs walk groups of PPC consecutive
// patches of the colour.  With NBUF = 2, while a group is computed the next
// group's closure of u and interior of b stream into the other input buffer,
// so global-memory latency overlaps the contractions; NBUF = 1 is used when
// two buffers do not fit in shared memory.  The gather is either one TMA box
// per patch and vector (ME > 0: tiled cp.async.bulk.tensor loads issued by one
// thread, completing on the buffer's mbarrier; the box starts at the closure
// origin rounded down to 16 bytes and the shift is kept per patch) or one
// cp.async per element (ME = 0).  Stages (3D; 2D drops the z stages):
//   z: P,Q | y: A1,A2 | x: r + forward FD along x | forward FD y |
//   forward FD z, times the FD diagonal, backward FD z (one z line per
//   thread) | backward FD y | backward FD x + scatter (u_new = u_old +
//   omega d, u_old from the buffer)
// Same-colour patches never write each other's closure, so the buffered
// closure values are the values the gather (eq. "gather") reads.
template <int DIM, int K, int NT, int PPC, int NBUF, int ME>
__global__ void __launch_bounds__(NT) patch_colour_kernel(const __grid_constant__ PatchTable tab,
                                                          const T* __restrict__ dinv,
                                                          const __grid_constant__ TmaMaps<ME> maps,
                                                          int* __restrict__ err) {
  constexpr bool TMA = ME > 0;
  // FP64, 3D: the local solver is exact (fast diagonalisation of the
  // constant-coefficient patch), so the updated interior A_j^{-1} (b_j -
  // bar A_j bar u_j) + u_j equals A_j^{-1} (b_j - bar A_j bar u_j^0), bar u_j^0
  // the closure with its interior set to zero: the residual is evaluated
  // with a zero interior and the scatter writes omega d + (1 - omega) u_j.
  // (FP32 keeps the correction form: recomputing the interior would cost
  // a factor cond(A_j) in single precision.)
  constexpr bool EXACT = sizeof(T) == 8 && DIM == 3;
  // FP64: the arithmetic runs in double-float on the FP32 pipe (the work
  // buffers hold float pairs; the FD diagonal's pairs follow it in dinv)
  constexpr bool DF = sizeof(T) == 8;
  using Z = SweepSmem<DIM, K, TMA>;
  constexpr int C = Z::C, M = Z::M, XU = Z::XU, XB = Z::XB;
  constexpr int LINES = DIM == 3 ? M * M : M;  // interior lines per axis
  extern __shared__ __align__(128) unsigned char smem_raw[];
  // TMA boxes start on 128 bytes: the launch adds 128 bytes of slack
  T* const IN0 = reinterpret_cast<T*>(TMA ? smem_raw + ((128 - (async::smem_u32(smem_raw) & 127)) & 127)
                                          : smem_raw);  // [NBUF][PPC][IN]
  T* const WA = IN0 + NBUF * PPC * Z::IN;              // [PPC][WA]
  T* const WB = WA + PPC * Z::WA;                      // [PPC][WB]
  float2* const WA2 = reinterpret_cast<float2*>(WA);   // DF views (same element size)
  float2* const WB2 = reinterpret_cast<float2*>(WB);
  const float2* const dinv_df = reinterpret_cast<const float2*>(dinv + Z::NINT);
  auto ldf = [](const float2 v) -> dfv { return {v.x, v.y}; };
  auto stf = [](const dfv v) -> float2 { return make_float2(v.hi, v.lo); };
  __shared__ long long s_origin[2][PPC];
  __shared__ int s_coord[2][PPC][3];   // closure origin (lattice coordinates), TMA gather
  __shared__ int s_nvalid[2];
  __shared__ int s_entry[2];
  __shared__ __align__(8) uint64_t s_bar[2];
  uint32_t phase = 0;  // bit s: parity of the next phase of s_bar[s]
  bool wait_ok = true;
  const T om = (T)tab.omega;
  const int mode = tab.mode;
  const int ngroups = tab.total_groups;
  if (TMA && threadIdx.x == 0) {
    async::mbar_init(&s_bar[0], 1);
    async::mbar_init(&s_bar[1], 1);
  }
  if (TMA) __syncthreads();
  // element offsets inside a patch's buffers: closure of u at (x, y, z)
  // (closure coordinates), interior of b at (x, y, z) (interior coordinates)
  auto uo = [](int x, int y, int z) { return DIM == 3 ? (z * C + y) * XU + x : y * XU + x; };
  auto bo = [](int x, int y, int z) { return DIM == 3 ? (z * M + y) * XB + x : y * XB + x; };
  // shift of the patch's closure inside its TMA box (0 without TMA)
  auto ushift = [&](int slot, int q) { return TMA ? s_coord[slot][q][0] % Z::A : 0; };

  // table entry and patch origins of a group (threads 0..PPC-1); callers
  // follow with a barrier
  auto set_origins = [&](int grp, int slot) {
    int lo = 0, hi = tab.n - 1;  // last entry with group_begin <= grp
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (tab.e[mid].group_begin <= grp) lo = mid;
      else hi = mid - 1;
    }
    const PatchEntry& e = tab.e[lo];
    const int g = grp - e.group_begin;
    const int nv = min(PPC, e.n_patches - g * PPC);
    if (threadIdx.x == 0) {
      s_nvalid[slot] = nv;
      s_entry[slot] = lo;
    }
    if (threadIdx.x < nv) {
      int pid = g * PPC + threadIdx.x;
      if (e.plist) pid = e.plist[pid];
      const int i0 = pid % e.count[0];
      const int rest = pid / e.count[0];
      const int i1 = rest % e.count[1];
      const int i2 = DIM == 3 ? rest / e.count[1] : 0;
      const long long o0 = (long long)(e.first[0] + 2 * i0 - 1) * K;
      const long long o1 = (long long)(e.first[1] + 2 * i1 - 1) * K;
      const long long o2 = DIM == 3 ? (long long)(e.first[2] + 2 * i2 - 1) * K : 0;
      s_origin[slot][threadIdx.x] = o0 + e.py * o1 + e.pz * o2;
      s_coord[slot][threadIdx.x][0] = (int)o0;
      s_coord[slot][threadIdx.x][1] = (int)o1;
      s_coord[slot][threadIdx.x][2] = (int)o2;
    }
  };
  // issue the copies of the group whose origins are in `slot` into input
  // buffer `slot`, then commit them as one group
  auto prefetch = [&](int slot) {
    const int nv = s_nvalid[slot];
    if constexpr (TMA) {
      if (threadIdx.x == 0) {
        const int ent = s_entry[slot];
        T* dst0 = IN0 + slot * PPC * Z::IN;
        async::mbar_arrive_expect_tx(&s_bar[slot], (uint32_t)(nv * ((mode == 0 ? Z::BOX_U : 0) + Z::BOX_B)));
        for (int q = 0; q < nv; ++q) {
          const int x0 = s_coord[slot][q][0], xa = x0 - x0 % Z::A;
          const int y0 = s_coord[slot][q][1], z0 = s_coord[slot][q][2];
          T* dst = dst0 + q * Z::IN;
          if (DIM == 3) {
            if (mode == 0) async::tma_load_3d(dst, &maps.u[ent], xa, y0, z0, &s_bar[slot]);
            async::tma_load_3d(dst + Z::NCLO, &maps.b[ent], xa, y0 + 1, z0 + 1, &s_bar[slot]);
          } else {
            if (mode == 0) async::tma_load_2d(dst, &maps.u[ent], xa, y0, &s_bar[slot]);
            async::tma_load_2d(dst + Z::NCLO, &maps.b[ent], xa, y0 + 1, &s_bar[slot]);
          }
        }
      }
      return;
    }
    const PatchEntry& e = tab.e[s_entry[slot]];
    const T* __restrict__ u = static_cast<const T*>(e.u);
    const T* __restrict__ b = static_cast<const T*>(e.b);
    const long long py = e.py, pz = e.pz;
    T* dst0 = IN0 + slot * PPC * Z::IN;
    // the solve-only mode needs no closure: only the residual's interior
    for (int idx = threadIdx.x; idx < (mode == 0 ? nv * Z::NCLO : 0); idx += NT) {  // closure of u
      const int q = idx / Z::NCLO, t = idx % Z::NCLO;
      const int x = t % C, row = t / C;
      const long long g = s_origin[slot][q] + x + py * (row % C) + (DIM == 3 ? pz * (row / C) : 0);
      async_copy(dst0 + q * Z::IN + t, u + g);
    }
    for (int idx = threadIdx.x; idx < nv * Z::NINT; idx += NT) {  // interior of b
      const int q = idx / Z::NINT, t = idx % Z::NINT;
      const int x = t % M, row = t / M;
      const long long g = s_origin[slot][q] + 1 + x + py * (row % M + 1) +
                          (DIM == 3 ? pz * (row / M + 1) : 0);
      async_copy(dst0 + q * Z::IN + Z::NCLO + t, b + g);
    }
    async_commit();
  };

  // wait for the gather of `slot`: the TMA phase (bounded; an expired wait
  // is recorded and the kernel carries on, so it always terminates) or this
  // thread's cp.async groups (all but `pending` newest)
  auto wait_gather = [&](int slot, int pending) {
    if constexpr (TMA) {
      if (wait_ok && !async::mbar_wait(&s_bar[slot], (phase >> slot) & 1u)) wait_ok = false;
      phase ^= 1u << slot;
    } else {
      if (pending) async_wait<1>();
      else async_wait<0>();
    }
  };
  int grp = blockIdx.x;
  if (NBUF == 2 && grp < ngroups) {
    set_origins(grp, 0);
    __syncthreads();
    prefetch(0);
  }
  for (int it = 0; grp < ngroups; grp += gridDim.x, ++it) {
    const int cur = NBUF == 2 ? (it & 1) : 0;
    if (NBUF == 1) {
      set_origins(grp, 0);
      __syncthreads();
      prefetch(0);
      wait_gather(0, 0);
    } else if (grp + (int)gridDim.x < ngroups) {
      set_origins(grp + gridDim.x, cur ^ 1);
      __syncthreads();
      prefetch(cur ^ 1);
      wait_gather(cur, 1);  // the current group's copies are done
    } else {
      wait_gather(cur, 0);
    }
    __syncthreads();  // ... and everybody's
    const int nvalid = s_nvalid[cur];
    const T* IN = IN0 + cur * PPC * Z::IN;
    const PatchEntry& ec = tab.e[s_entry[cur]];
    T* __restrict__ u = static_cast<T*>(ec.u);
    const long long py = ec.py, pz = ec.pz;
    const T sb = (T)ec.sb;

    if (mode != 0) {
      // solve only: nothing to evaluate, the buffer holds the residual
    } else if (DIM == 3) {
      // ---- stage z: P = Mp_z u, Q = Kp_z u   (dims x:C, y:C, z:M, in WB) ----
      if constexpr (EXACT) {
        // the patch interior is taken as zero (see the scatter): a line with
        // (x, y) inside the patch has only its two end values left.  Lines
        // are enumerated interior ones first, patches interleaved, so that a
        // warp runs one kind of line.
        constexpr int CI = C - 2;
        for (int idx = threadIdx.x; idx < nvalid * C * C; idx += NT) {
          const int q = idx % nvalid, lp = idx / nvalid;
          int x, y;
          if (lp < CI * CI) {
            x = 1 + lp % CI;
            y = 1 + lp / CI;
          } else {
            const int e = lp - CI * CI;
            if (e < C) { x = e; y = 0; }
            else if (e < 2 * C) { x = e - C; y = C - 1; }
            else { x = ((e - 2 * C) & 1) ? C - 1 : 0; y = 1 + (e - 2 * C) / 2; }
          }
          const int l = x + C * y;
          const T* U = IN + q * Z::IN + ushift(cur, q) + uo(x, y, 0);
          T* B = WB + q * Z::WB;
          if constexpr (DF) {
            float2* B2 = WB2 + q * Z::WB;
            if (lp < CI * CI) {
              const dfv u0 = df_from_double(U[0]), uc = df_from_double(U[(C - 1) * C * XU]);
#pragma unroll
              for (int i = 0; i < M; ++i) {
                df_acc a = {0.f, 0.f}, b = {0.f, 0.f};
                float h, lo;
                if (band_lo(i + 1, K) == 0) {
                  patch_entry_df<K, 0>(i, 0, h, lo);
                  df_acc_add(a, h, lo, u0);
                  patch_entry_df<K, 1>(i, 0, h, lo);
                  df_acc_add(b, h, lo, u0);
                }
                if (band_hi(i + 1, K) == 2 * K) {
                  patch_entry_df<K, 0>(i, C - 1, h, lo);
                  df_acc_add(a, h, lo, uc);
                  patch_entry_df<K, 1>(i, C - 1, h, lo);
                  df_acc_add(b, h, lo, uc);
                }
                B2[l + i * C * C] = stf(df_acc_value(a));
                B2[C * C * M + l + i * C * C] = stf(df_acc_value(b));
              }
            } else {
              dfv xv[C];
#pragma unroll
              for (int j = 0; j < C; ++j) xv[j] = df_from_double(U[j * C * XU]);
#pragma unroll
              for (int i = 0; i < M; ++i) {
                df_acc a = {0.f, 0.f}, b = {0.f, 0.f};
                patch_row_df<K, 0>(i, xv, a);
                patch_row_df<K, 1>(i, xv, b);
                B2[l + i * C * C] = stf(df_acc_value(a));
                B2[C * C * M + l + i * C * C] = stf(df_acc_value(b));
              }
            }
            continue;
          }
          if (lp < CI * CI) {
            const T u0 = U[0], uc = U[(C - 1) * C * XU];
#pragma unroll
            for (int i = 0; i < M; ++i) {
              B[l + i * C * C] = patch_row_ends<K, 0>(i, u0, uc);
              B[C * C * M + l + i * C * C] = patch_row_ends<K, 1>(i, u0, uc);
            }
          } else {
            T xv[C];
#pragma unroll
            for (int j = 0; j < C; ++j) xv[j] = U[j * C * XU];
#pragma unroll
            for (int i = 0; i < M; ++i) {
              B[l + i * C * C] = patch_row<K, 0>(i, xv);
              B[C * C * M + l + i * C * C] = patch_row<K, 1>(i, xv);
            }
          }
        }
      } else {
        for (int idx = threadIdx.x; idx < nvalid * C * C; idx += NT) {
          const int q = idx / (C * C), l = idx % (C * C);
          const T* U = IN + q * Z::IN + ushift(cur, q) + uo(l % C, l / C, 0);
          T* B = WB + q * Z::WB;
          T x[C];
#pragma unroll
          for (int j = 0; j < C; ++j) x[j] = U[j * C * XU];
#pragma unroll
          for (int i = 0; i < M; ++i) {
            B[l + i * C * C] = patch_row<K, 0>(i, x);
            B[C * C * M + l + i * C * C] = patch_row<K, 1>(i, x);
          }
        }
      }
      __syncthreads();
      // ---- stage y: A1 = Mp_y P, A2 = Kp_y P + Mp_y Q   (dims x:C, y:M, z:M, in WA) ----
      for (int idx = threadIdx.x; idx < nvalid * C * M; idx += NT) {
        const int q = idx / (C * M), l = idx % (C * M);
        T* A = WA + q * Z::WA;
        const T* B = WB + q * Z::WB;
        const int x0 = l % C, z = l / C;
        if constexpr (DF) {
          const float2* B2 = WB2 + q * Z::WB;
          float2* A2 = WA2 + q * Z::WA;
          dfv p[C], r[C];
#pragma unroll
          for (int j = 0; j < C; ++j) {
            p[j] = ldf(B2[x0 + j * C + z * C * C]);
            r[j] = ldf(B2[C * C * M + x0 + j * C + z * C * C]);
          }
#pragma unroll
          for (int i = 0; i < M; ++i) {
            df_acc a = {0.f, 0.f}, b = {0.f, 0.f};
            patch_row_df<K, 0>(i, p, a);
            patch_row_df<K, 1>(i, p, b);
            patch_row_df<K, 0>(i, r, b);
            A2[x0 + i * C + z * C * M] = stf(df_acc_value(a));
            A2[C * M * M + x0 + i * C + z * C * M] = stf(df_acc_value(b));
          }
          continue;
        }
        T p[C], r[C];
#pragma unroll
        for (int j = 0; j < C; ++j) {
          p[j] = B[x0 + j * C + z * C * C];
          r[j] = B[C * C * M + x0 + j * C + z * C * C];
        }
#pragma unroll
        for (int i = 0; i < M; ++i) {
          A[x0 + i * C + z * C * M] = patch_row<K, 0>(i, p);
          A[C * M * M + x0 + i * C + z * C * M] = patch_row<K, 0>(i, r, patch_row<K, 1>(i, p));
        }
      }
      __syncthreads();
    } else {
      // ---- stage y: P = Mp_y u, Q = Kp_y u   (dims x:C, y:M, in WA) ----
      for (int idx = threadIdx.x; idx < nvalid * C; idx += NT) {
        const int q = idx / C, l = idx % C;
        const T* U = IN + q * Z::IN + ushift(cur, q) + l;
        T* A = WA + q * Z::WA;
        if constexpr (DF) {
          float2* A2 = WA2 + q * Z::WA;
          dfv xv[C];
#pragma unroll
          for (int j = 0; j < C; ++j) xv[j] = df_from_double(U[j * XU]);
#pragma unroll
          for (int i = 0; i < M; ++i) {
            df_acc a = {0.f, 0.f}, b = {0.f, 0.f};
            patch_row_df<K, 0>(i, xv, a);
            patch_row_df<K, 1>(i, xv, b);
            A2[l + i * C] = stf(df_acc_value(a));
            A2[C * M + l + i * C] = stf(df_acc_value(b));
          }
          continue;
        }
        T x[C];
#pragma unroll
        for (int j = 0; j < C; ++j) x[j] = U[j * XU];
#pragma unroll
        for (int i = 0; i < M; ++i) {
          A[l + i * C] = patch_row<K, 0>(i, x);
          A[C * M + l + i * C] = patch_row<K, 1>(i, x);
        }
      }
      __syncthreads();
    }

    // ---- stage x: r = sb b - (Kp_x X1 + Mp_x X2) per interior line (X1, X2 =
    // A1, A2 in 3D, P, Q in 2D, both in WA), then the forward FD transform
    // along x in registers; result into WB ----
    for (int idx = threadIdx.x; idx < nvalid * LINES; idx += NT) {
      const int q = idx / LINES, l = idx % LINES;
      constexpr int PLANE = DIM == 3 ? C * M * M : C * M;
      const T* X = WA + q * Z::WA;
      // interior row l of b: x = 0..M-1 at (y, z) = (l % M, l / M) (3D) or y = l (2D)
      const T* Bq = IN + q * Z::IN + Z::NCLO + (TMA ? ushift(cur, q) + 1 : 0) +
                    (DIM == 3 ? bo(0, l % M, l / M) : bo(0, l, 0));
      if constexpr (DF) {
        const float2* X2 = WA2 + q * Z::WA;
        const float sbf = (float)ec.sb;  // h^{2-d}: n in 3D, 1 in 2D, exact in float
        dfv rd[M], yd[M];
        if (mode == 0) {
          dfv a1[C], a2[C];
#pragma unroll
          for (int j = 0; j < C; ++j) {
            a1[j] = ldf(X2[j + C * l]);
            a2[j] = ldf(X2[PLANE + j + C * l]);
          }
#pragma unroll
          for (int i = 0; i < M; ++i) {
            const dfv bb = df_mul(df_from_double(Bq[i]), {sbf, 0.f});
            df_acc acc = {bb.hi, bb.lo};
            patch_row_df<K, 1, true>(i, a1, acc);
            patch_row_df<K, 0, true>(i, a2, acc);
            rd[i] = df_acc_value(acc);
          }
        } else {
#pragma unroll
          for (int i = 0; i < M; ++i) rd[i] = df_mul(df_from_double(Bq[i]), {sbf, 0.f});
        }
        fd_forward_df<K>(rd, yd);
        float2* R2 = WB2 + q * Z::WB + M * l;
#pragma unroll
        for (int i = 0; i < M; ++i) R2[i] = stf(yd[i]);
        continue;
      }
      T r[M], y[M];
      if (mode == 0) {
        T a1[C], a2[C];
#pragma unroll
        for (int j = 0; j < C; ++j) {
          a1[j] = X[j + C * l];
          a2[j] = X[PLANE + j + C * l];
        }
#pragma unroll
        for (int i = 0; i < M; ++i) {
          T acc = sb * Bq[i];
          acc = patch_row<K, 1, true>(i, a1, acc);
          r[i] = patch_row<K, 0, true>(i, a2, acc);
        }
      } else {
#pragma unroll
        for (int i = 0; i < M; ++i) r[i] = sb * Bq[i];
      }
      fd_forward<K>(r, y);
      T* R = WB + q * Z::WB + M * l;
#pragma unroll
      for (int i = 0; i < M; ++i) R[i] = y[i];
    }
    __syncthreads();

    // ---- local solve by fast diagonalisation (App. A.3), in place in WB ----
    if (DIM == 3) {
      for (int idx = threadIdx.x; idx < nvalid * LINES; idx += NT) {  // forward y
        const int q = idx / LINES, l = idx % LINES;
        if constexpr (DF) fd_smem_line_df<K, true>(WB2 + q * Z::WB + (l % M) + (l / M) * M * M, M);
        else fd_smem_line<K, true>(WB + q * Z::WB + (l % M) + (l / M) * M * M, M);
      }
      __syncthreads();
      for (int idx = threadIdx.x; idx < nvalid * LINES; idx += NT) {  // forward z, diagonal, backward z
        const int q = idx / LINES, l = idx % LINES;
        if constexpr (DF) fd_smem_line_solve_df<K>(WB2 + q * Z::WB + l, M * M, dinv_df + l, M * M);
        else fd_smem_line_solve<K>(WB + q * Z::WB + l, M * M, dinv + l, M * M);
      }
      __syncthreads();
      for (int idx = threadIdx.x; idx < nvalid * LINES; idx += NT) {  // backward y
        const int q = idx / LINES, l = idx % LINES;
        if constexpr (DF) fd_smem_line_df<K, false>(WB2 + q * Z::WB + (l % M) + (l / M) * M * M, M);
        else fd_smem_line<K, false>(WB + q * Z::WB + (l % M) + (l / M) * M * M, M);
      }
      __syncthreads();
    } else {
      for (int idx = threadIdx.x; idx < nvalid * LINES; idx += NT) {  // forward y, diagonal, backward y
        const int q = idx / LINES, l = idx % LINES;
        if constexpr (DF) fd_smem_line_solve_df<K>(WB2 + q * Z::WB + l, M, dinv_df + l, M);
        else fd_smem_line_solve<K>(WB + q * Z::WB + l, M, dinv + l, M);
      }
      __syncthreads();
    }

    // ---- backward FD along x and scatter (eq. "scatter") ----
    for (int idx = threadIdx.x; idx < nvalid * LINES; idx += NT) {
      const int q = idx / LINES, l = idx % LINES;
      const T* R = WB + q * Z::WB + M * l;
      // interior line l of the patch: closure row (y+1, z+1), x = 1..M
      const T* U = IN + q * Z::IN + ushift(cur, q) +
                   (DIM == 3 ? uo(1, l % M + 1, l / M + 1) : uo(1, l + 1, 0));
      T d[M];
      if constexpr (DF) {
        const float2* R2 = WB2 + q * Z::WB + M * l;
        dfv yv[M], dd[M];
#pragma unroll
        for (int i = 0; i < M; ++i) yv[i] = ldf(R2[i]);
        fd_backward_df<K>(yv, dd);
#pragma unroll
        for (int i = 0; i < M; ++i) d[i] = df_to_double(dd[i]);
      } else {
        T yv[M];
#pragma unroll
        for (int i = 0; i < M; ++i) yv[i] = R[i];
        fd_backward<K>(yv, d);
      }
      const long long row = s_origin[cur][q] + 1 + py * (l % M + 1) + (DIM == 3 ? pz * (l / M + 1) : 0);
#pragma unroll
      for (int i = 0; i < M; ++i)
        u[row + i] = EXACT && DIM == 3 && mode == 0 ? fma(om, d[i], (T(1) - om) * U[i])
                                                    : fma(om, d[i], mode == 0 ? U[i] : u[row + i]);
    }
    if (TMA) async::fence_proxy_async();  // reads of the buffers before the next TMA writes
    __syncthreads();  // buffers and origins are refilled / reused next iteration
  }
  if (TMA && !wait_ok) atomicExch(err, GMG_ERR_TIMEOUT);
}

// ---------------------------------------------------------------------------
// Matrix-free level operator on a tile of BC cells per direction.
// Global 1D matrix row for node i = c K + p: p > 0 -> cell c row p;
// p == 0 (vertex) -> cell c-1 row K plus cell c row 0.
// Tile inputs: nodes [(c0-1)K, (c0+BC)K] (EI per direction, zero outside the
// lattice); outputs: nodes [c0 K, (c0+BC) K) (EO per direction).
template <int K, int EI, int KIND>
__device__ __forceinline__ T cell_row(int o, const T (&x)[EI]) {
  // KIND 0: unit-cell mass, 1: unit-cell stiffness (direct __constant__ index)
  auto E = [](int i) -> T { return KIND == 0 ? c_Mc[off_cell(K) + i] : c_Kc[off_cell(K) + i]; };
  const int p = o % K;
  T acc = T(0);
  if (p == 0) {
#pragma unroll
    for (int q = 0; q <= K; ++q) acc = fma(E(K * (K + 1) + q), x[o + q], acc);
#pragma unroll
    for (int q = 0; q <= K; ++q) acc = fma(E(q), x[o + K + q], acc);
  } else {
#pragma unroll
    for (int q = 0; q <= K; ++q) acc = fma(E(p * (K + 1) + q), x[o - p + K + q], acc);
  }
  return acc;
}

// Tile of BX x BY (x BZ) cells: inputs E?I = (B? + 1) K + 1 nodes per
// direction (one halo cell below), outputs E?O = B? K.
template <int DIM, int K, int BX, int BY, int BZ>
struct ApplyDims {
  static constexpr int EIX = (BX + 1) * K + 1, EIY = (BY + 1) * K + 1, EIZ = DIM == 3 ? (BZ + 1) * K + 1 : 1;
  static constexpr int EOX = BX * K, EOY = BY * K, EOZ = DIM == 3 ? BZ * K : 1;
  // A: the input tile, later the stage-y results; B: the stage-z results
  static constexpr int SA = DIM == 3 ? cmax(EIX * EIY * EIZ, 2 * EIX * EOY * EOZ) : EIX * EIY;
  static constexpr int SB = DIM == 3 ? 2 * EIX * EIY * EOZ : 2 * EIX * EOY;
  static constexpr int SMEM_BYTES = (SA + SB) * (int)sizeof(T);
};

template <int DIM, int K, int BX, int BY, int BZ, int NT>
__global__ void __launch_bounds__(NT) apply_kernel(const T* __restrict__ xin, T* __restrict__ y,
                                                   const T* __restrict__ bvec, ApplyLaunch al) {
  using D = ApplyDims<DIM, K, BX, BY, BZ>;
  constexpr int EIX = D::EIX, EIY = D::EIY, EIZ = D::EIZ, EOX = D::EOX, EOY = D::EOY, EOZ = D::EOZ;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  T* A = reinterpret_cast<T*>(smem_raw);
  T* B = A + D::SA;
  const int N = al.g.N, n = al.g.n;
  const long long py = al.g.py, pz = al.g.pz;
  const int tx = (n + BX - 1) / BX, ty = (n + BY - 1) / BY, tz = DIM == 3 ? (n + BZ - 1) / BZ : 1;
  const int ntile = tx * ty * tz;
  const T alpha = (T)al.alpha, beta = (T)al.beta;

  for (int tid = blockIdx.x; tid < ntile; tid += gridDim.x) {
    const int t0 = tid % tx, t1 = (tid / tx) % ty, t2 = DIM == 3 ? tid / (tx * ty) : 0;
    const int g0 = (t0 * BX - 1) * K, g1 = (t1 * BY - 1) * K, g2 = DIM == 3 ? (t2 * BZ - 1) * K : 0;
    // gather the tile with zero fill outside the lattice
    const int nin = EIX * EIY * EIZ;
    for (int t = threadIdx.x; t < nin; t += NT) {
      int x = t % EIX, yy = (t / EIX) % EIY, z = DIM == 3 ? t / (EIX * EIY) : 0;
      int gx = g0 + x, gy = g1 + yy, gz = g2 + z;
      bool ok = gx >= 0 && gx < N && gy >= 0 && gy < N && (DIM == 2 || (gz >= 0 && gz < N));
      A[t] = ok ? xin[gx + py * gy + pz * gz] : T(0);
    }
    __syncthreads();
    if (DIM == 3) {
      // stage z: P = M_z x, Q = K_z x   (x:EIX, y:EIY, z:EOZ)
      for (int l = threadIdx.x; l < EIX * EIY; l += NT) {
        T v[EIZ];
#pragma unroll
        for (int j = 0; j < EIZ; ++j) v[j] = A[l + j * EIX * EIY];
#pragma unroll
        for (int o = 0; o < EOZ; ++o) {
          B[l + o * EIX * EIY] = cell_row<K, EIZ, 0>(o, v);
          B[EIX * EIY * EOZ + l + o * EIX * EIY] = cell_row<K, EIZ, 1>(o, v);
        }
      }
      __syncthreads();
      // stage y: A1 = M_y P, A2 = K_y P + M_y Q   (x:EIX, y:EOY, z:EOZ)
      for (int l = threadIdx.x; l < EIX * EOZ; l += NT) {
        int x0 = l % EIX, z = l / EIX;
        T p[EIY], q[EIY];
#pragma unroll
        for (int j = 0; j < EIY; ++j) {
          p[j] = B[x0 + j * EIX + z * EIX * EIY];
          q[j] = B[EIX * EIY * EOZ + x0 + j * EIX + z * EIX * EIY];
        }
#pragma unroll
        for (int o = 0; o < EOY; ++o) {
          A[x0 + o * EIX + z * EIX * EOY] = cell_row<K, EIY, 0>(o, p);
          A[EIX * EOY * EOZ + x0 + o * EIX + z * EIX * EOY] = cell_row<K, EIY, 1>(o, p) + cell_row<K, EIY, 0>(o, q);
        }
      }
      __syncthreads();
      // stage x and write: y = alpha (K_x A1 + M_x A2) + beta b on owned interior nodes
      for (int l = threadIdx.x; l < EOY * EOZ; l += NT) {
        int yy = l % EOY, z = l / EOY;
        int gy = g1 + K + yy, gz = g2 + K + z;
        if (gy <= 0 || gy >= N - 1 || gz <= 0 || gz >= N - 1) continue;
        T a1[EIX], a2[EIX];
#pragma unroll
        for (int j = 0; j < EIX; ++j) {
          a1[j] = A[j + EIX * (yy + EOY * z)];
          a2[j] = A[EIX * EOY * EOZ + j + EIX * (yy + EOY * z)];
        }
        const long long row = py * gy + pz * gz;
#pragma unroll
        for (int o = 0; o < EOX; ++o) {
          int gx = g0 + K + o;
          if (gx <= 0 || gx >= N - 1) continue;
          T v = alpha * (cell_row<K, EIX, 1>(o, a1) + cell_row<K, EIX, 0>(o, a2));
          if (bvec) v += beta * bvec[row + gx];
          y[row + gx] = v;
        }
      }
    } else {
      // stage y: P = M_y x, Q = K_y x   (x:EIX, y:EOY)
      for (int l = threadIdx.x; l < EIX; l += NT) {
        T v[EIY];
#pragma unroll
        for (int j = 0; j < EIY; ++j) v[j] = A[l + j * EIX];
#pragma unroll
        for (int o = 0; o < EOY; ++o) {
          B[l + o * EIX] = cell_row<K, EIY, 0>(o, v);
          B[EIX * EOY + l + o * EIX] = cell_row<K, EIY, 1>(o, v);
        }
      }
      __syncthreads();
      for (int l = threadIdx.x; l < EOY; l += NT) {
        int gy = g1 + K + l;
        if (gy <= 0 || gy >= N - 1) continue;
        T p[EIX], q[EIX];
#pragma unroll
        for (int j = 0; j < EIX; ++j) {
          p[j] = B[j + EIX * l];
          q[j] = B[EIX * EOY + j + EIX * l];
        }
        const long long row = py * gy;
#pragma unroll
        for (int o = 0; o < EOX; ++o) {
          int gx = g0 + K + o;
          if (gx <= 0 || gx >= N - 1) continue;
          T v = alpha * (cell_row<K, EIX, 1>(o, p) + cell_row<K, EIX, 0>(o, q));
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

// Variable-coefficient kernels (-div(a grad u), one coefficient per cell),
// for one scalar type GMG_T; included after patch_kernels.cuh (which gives
// this translation unit its own __constant__ tables and FD helpers) by
// var_f32.cu / var_f64.cu.
//
//  * apply_var_kernel: y += alpha * sum_c a_c A_c x_c, cell by cell by sum
//    factorisation (App. A.1), accumulated with atomics (a node is shared
//    by up to 2^d cells); the caller initialises y.
//  * patch_var_kernel: one colour of the patch smoother (Algorithm 4) whose
//    local residual is evaluated cell by cell with the cell coefficients
//    (Sec. 3.1, eq. "main:4"), and whose local solver is the fast
//    diagonalisation of the constant-coefficient patch scaled by the
//    geometric mean abar of the 2^d cell coefficients, optionally plus a
//    per-patch rank-R correction U diag(s) U^T (reference units); the FD term
//    is damped per patch by theta = min(1, 1.8 abar / max_c a_c)
//    (A_j <= max_c a_c Ahat_j, so the damped FD update's spectrum stays
//    below 1.8), the learned term approximates the rest of the exact inverse:
//        d = (1/abar) [ theta FD_ref(r_ref) + U diag(s) U^T r_ref ],  r_ref = h^{2-d} r.
#pragma once
#include "patch_kernels.cuh"

namespace gmg {
namespace GMG_NS {

// one (K+1)-point 1D cell operator applied to a line: y_i = sum_j E[i][j] x_j
template <int K, int KIND>
__device__ __forceinline__ T cell1d(int i, const T (&x)[K + 1]) {
  T acc = T(0);
#pragma unroll
  for (int j = 0; j <= K; ++j) {
    const T e = KIND == 0 ? c_Mc[off_cell(K) + i * (K + 1) + j] : c_Kc[off_cell(K) + i * (K + 1) + j];
    acc = fma(e, x[j], acc);
  }
  return acc;
}

// Cell operator (unit cell, coefficient 1) on an (K+1)^DIM block in shared
// memory X (x fastest) -> OUT, using P, Q, A1, A2 as scratch; lines of `ncell`
// cells (stride S between cells) are spread over NT threads.  Ends with a
// barrier.
template <int DIM, int K, int NT>
__device__ __forceinline__ void cell_operator(T* X, T* P, T* Q, T* A1, T* A2, T* OUT, int ncell, int S) {
  constexpr int E = K + 1;
  if (DIM == 3) {
    for (int idx = threadIdx.x; idx < ncell * E * E; idx += NT) {  // z: P = M_z x, Q = K_z x
      const int c = idx / (E * E), l = idx % (E * E);
      T v[E];
#pragma unroll
      for (int j = 0; j < E; ++j) v[j] = X[c * S + l + j * E * E];
#pragma unroll
      for (int i = 0; i < E; ++i) {
        P[c * S + l + i * E * E] = cell1d<K, 0>(i, v);
        Q[c * S + l + i * E * E] = cell1d<K, 1>(i, v);
      }
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < ncell * E * E; idx += NT) {  // y: A1 = M_y P, A2 = K_y P + M_y Q
      const int c = idx / (E * E), l = idx % (E * E);
      const int x0 = l % E, z = l / E;
      T p[E], q[E];
#pragma unroll
      for (int j = 0; j < E; ++j) {
        p[j] = P[c * S + x0 + j * E + z * E * E];
        q[j] = Q[c * S + x0 + j * E + z * E * E];
      }
#pragma unroll
      for (int i = 0; i < E; ++i) {
        A1[c * S + x0 + i * E + z * E * E] = cell1d<K, 0>(i, p);
        A2[c * S + x0 + i * E + z * E * E] = cell1d<K, 1>(i, p) + cell1d<K, 0>(i, q);
      }
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < ncell * E * E; idx += NT) {  // x: OUT = K_x A1 + M_x A2
      const int c = idx / (E * E), l = idx % (E * E);
      T a1[E], a2[E];
#pragma unroll
      for (int j = 0; j < E; ++j) {
        a1[j] = A1[c * S + l * E + j];
        a2[j] = A2[c * S + l * E + j];
      }
#pragma unroll
      for (int i = 0; i < E; ++i) OUT[c * S + l * E + i] = cell1d<K, 1>(i, a1) + cell1d<K, 0>(i, a2);
    }
    __syncthreads();
  } else {
    for (int idx = threadIdx.x; idx < ncell * E; idx += NT) {  // y: P = M_y x, Q = K_y x
      const int c = idx / E, l = idx % E;
      T v[E];
#pragma unroll
      for (int j = 0; j < E; ++j) v[j] = X[c * S + l + j * E];
#pragma unroll
      for (int i = 0; i < E; ++i) {
        P[c * S + l + i * E] = cell1d<K, 0>(i, v);
        Q[c * S + l + i * E] = cell1d<K, 1>(i, v);
      }
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < ncell * E; idx += NT) {  // x: OUT = K_x P + M_x Q
      const int c = idx / E, l = idx % E;
      T p[E], q[E];
#pragma unroll
      for (int j = 0; j < E; ++j) {
        p[j] = P[c * S + l * E + j];
        q[j] = Q[c * S + l * E + j];
      }
#pragma unroll
      for (int i = 0; i < E; ++i) OUT[c * S + l * E + i] = cell1d<K, 1>(i, p) + cell1d<K, 0>(i, q);
    }
    __syncthreads();
  }
}

// The same cell operator in double-float arithmetic (FP64 problems): X, P,
// Q, A1, A2, OUT hold float pairs; the unit-cell matrices as float pairs.
template <int K, int KIND>
__device__ __forceinline__ void cell1d_df(int i, const dfv (&x)[K + 1], df_acc& acc) {
#pragma unroll
  for (int j = 0; j <= K; ++j) {
    const int o = off_cell(K) + i * (K + 1) + j;
    df_acc_add(acc, KIND == 0 ? c_Mchi[o] : c_Kchi[o], KIND == 0 ? c_Mclo[o] : c_Kclo[o], x[j]);
  }
}

template <int DIM, int K, int NT>
__device__ __forceinline__ void cell_operator_df(float2* X, float2* P, float2* Q, float2* A1, float2* A2,
                                                 float2* OUT, int ncell, int S) {
  constexpr int E = K + 1;
  auto ld = [](const float2 v) -> dfv { return {v.x, v.y}; };
  auto st = [](const df_acc a) -> float2 {
    const dfv v = df_acc_value(a);
    return make_float2(v.hi, v.lo);
  };
  if (DIM == 3) {
    for (int idx = threadIdx.x; idx < ncell * E * E; idx += NT) {  // z: P = M_z x, Q = K_z x
      const int c = idx / (E * E), l = idx % (E * E);
      dfv v[E];
#pragma unroll
      for (int j = 0; j < E; ++j) v[j] = ld(X[c * S + l + j * E * E]);
#pragma unroll
      for (int i = 0; i < E; ++i) {
        df_acc a = {0.f, 0.f}, b = {0.f, 0.f};
        cell1d_df<K, 0>(i, v, a);
        cell1d_df<K, 1>(i, v, b);
        P[c * S + l + i * E * E] = st(a);
        Q[c * S + l + i * E * E] = st(b);
      }
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < ncell * E * E; idx += NT) {  // y: A1 = M_y P, A2 = K_y P + M_y Q
      const int c = idx / (E * E), l = idx % (E * E);
      const int x0 = l % E, z = l / E;
      dfv p[E], q[E];
#pragma unroll
      for (int j = 0; j < E; ++j) {
        p[j] = ld(P[c * S + x0 + j * E + z * E * E]);
        q[j] = ld(Q[c * S + x0 + j * E + z * E * E]);
      }
#pragma unroll
      for (int i = 0; i < E; ++i) {
        df_acc a = {0.f, 0.f}, b = {0.f, 0.f};
        cell1d_df<K, 0>(i, p, a);
        cell1d_df<K, 1>(i, p, b);
        cell1d_df<K, 0>(i, q, b);
        A1[c * S + x0 + i * E + z * E * E] = st(a);
        A2[c * S + x0 + i * E + z * E * E] = st(b);
      }
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < ncell * E * E; idx += NT) {  // x: OUT = K_x A1 + M_x A2
      const int c = idx / (E * E), l = idx % (E * E);
      dfv a1[E], a2[E];
#pragma unroll
      for (int j = 0; j < E; ++j) {
        a1[j] = ld(A1[c * S + l * E + j]);
        a2[j] = ld(A2[c * S + l * E + j]);
      }
#pragma unroll
      for (int i = 0; i < E; ++i) {
        df_acc a = {0.f, 0.f};
        cell1d_df<K, 1>(i, a1, a);
        cell1d_df<K, 0>(i, a2, a);
        OUT[c * S + l * E + i] = st(a);
      }
    }
    __syncthreads();
  } else {
    for (int idx = threadIdx.x; idx < ncell * E; idx += NT) {  // y: P = M_y x, Q = K_y x
      const int c = idx / E, l = idx % E;
      dfv v[E];
#pragma unroll
      for (int j = 0; j < E; ++j) v[j] = ld(X[c * S + l + j * E]);
#pragma unroll
      for (int i = 0; i < E; ++i) {
        df_acc a = {0.f, 0.f}, b = {0.f, 0.f};
        cell1d_df<K, 0>(i, v, a);
        cell1d_df<K, 1>(i, v, b);
        P[c * S + l + i * E] = st(a);
        Q[c * S + l + i * E] = st(b);
      }
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < ncell * E; idx += NT) {  // x: OUT = K_x P + M_x Q
      const int c = idx / E, l = idx % E;
      dfv p[E], q[E];
#pragma unroll
      for (int j = 0; j < E; ++j) {
        p[j] = ld(P[c * S + l * E + j]);
        q[j] = ld(Q[c * S + l * E + j]);
      }
#pragma unroll
      for (int i = 0; i < E; ++i) {
        df_acc a = {0.f, 0.f};
        cell1d_df<K, 1>(i, p, a);
        cell1d_df<K, 0>(i, q, a);
        OUT[c * S + l * E + i] = st(a);
      }
    }
    __syncthreads();
  }
}

__device__ __forceinline__ void atomic_add(double* a, double v) { atomicAdd(a, v); }
__device__ __forceinline__ void atomic_add(float* a, float v) { atomicAdd(a, v); }

// y += alpha * sum_c a_c A_c x on the interior nodes (cells of unit width).
template <int DIM, int K, int NT, int CPC>
__global__ void __launch_bounds__(NT) apply_var_kernel(const T* __restrict__ x, T* __restrict__ y,
                                                       const T* __restrict__ coef, LevelGeom g, T alpha) {
  constexpr int E = K + 1;
  constexpr int NE = DIM == 3 ? E * E * E : E * E;
  __shared__ T X[CPC * NE], P[CPC * NE], Q[CPC * NE], A1[CPC * NE], A2[CPC * NE];
  __shared__ float2 s_sc[CPC];  // alpha a_c of the CTA's cells as float pairs (FP64 problems)
  const int n = g.n, N = g.N;
  const long long ncell = DIM == 3 ? (long long)n * n * n : (long long)n * n;
  for (long long c0 = (long long)blockIdx.x * CPC; c0 < ncell; c0 += (long long)gridDim.x * CPC) {
    const int nc = (int)(ncell - c0 < CPC ? ncell - c0 : CPC);
    if constexpr (sizeof(T) == 8) {
      if ((int)threadIdx.x < nc) {
        const dfv a = df_from_double(alpha * coef[c0 + threadIdx.x]);
        s_sc[threadIdx.x] = make_float2(a.hi, a.lo);
      }
    }
    for (int idx = threadIdx.x; idx < nc * NE; idx += NT) {
      const long long c = c0 + idx / NE;
      const int t = idx % NE;
      const int cx = (int)(c % n), cy = (int)((c / n) % n), cz = DIM == 3 ? (int)(c / ((long long)n * n)) : 0;
      const int lx = t % E, ly = (t / E) % E, lz = DIM == 3 ? t / (E * E) : 0;
      const long long gi = (long long)(cx * K + lx) + g.py * (cy * K + ly) + (DIM == 3 ? g.pz * (cz * K + lz) : 0);
      if constexpr (sizeof(T) == 8) {
        const dfv v = df_from_double(x[gi]);
        reinterpret_cast<float2*>(X)[idx] = make_float2(v.hi, v.lo);
      } else {
        X[idx] = x[gi];
      }
    }
    __syncthreads();
    if constexpr (sizeof(T) == 8)  // double-float cell operator on float pairs
      cell_operator_df<DIM, K, NT>(reinterpret_cast<float2*>(X), reinterpret_cast<float2*>(P),
                                   reinterpret_cast<float2*>(Q), reinterpret_cast<float2*>(A1),
                                   reinterpret_cast<float2*>(A2), reinterpret_cast<float2*>(X), nc, NE);
    else
      cell_operator<DIM, K, NT>(X, P, Q, A1, A2, X, nc, NE);  // OUT overwrites X per line (own line only)
    for (int idx = threadIdx.x; idx < nc * NE; idx += NT) {
      const long long c = c0 + idx / NE;
      const int t = idx % NE;
      const int cx = (int)(c % n), cy = (int)((c / n) % n), cz = DIM == 3 ? (int)(c / ((long long)n * n)) : 0;
      const int ix = cx * K + t % E, iy = cy * K + (t / E) % E, iz = DIM == 3 ? cz * K + t / (E * E) : 1;
      if (ix <= 0 || ix >= N - 1 || iy <= 0 || iy >= N - 1 || (DIM == 3 && (iz <= 0 || iz >= N - 1))) continue;
      const long long gi = ix + g.py * iy + (DIM == 3 ? g.pz * iz : 0);
      if constexpr (sizeof(T) == 8) {
        const float2 v = reinterpret_cast<const float2*>(X)[idx], a = s_sc[idx / NE];
        atomic_add(y + gi, df_to_double(df_mul({v.x, v.y}, {a.x, a.y})));
      } else {
        atomic_add(y + gi, alpha * coef[c] * X[idx]);
      }
    }
    __syncthreads();
  }
}

// y = beta * b on interior nodes (b may be null: zero); padding untouched
__global__ void init_interior_kernel(T* __restrict__ y, const T* __restrict__ b, T beta, LevelGeom g,
                                     long long n_elems) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n_elems;
       e += (long long)gridDim.x * blockDim.x) {
    const int ix = (int)(e % g.py);
    const int iy = (int)((e / g.py) % g.N);
    const int iz = g.dim == 3 ? (int)(e / g.pz) : 1;
    if (ix <= 0 || ix >= g.N - 1 || iy <= 0 || iy >= g.N - 1 || (g.dim == 3 && (iz <= 0 || iz >= g.N - 1)))
      continue;
    y[e] = b ? beta * b[e] : T(0);
  }
}

// One colour of the variable-coefficient patch smoother: persistent CTAs,
// one patch at a time.  With TMA the closure of u and the interior of b of
// the CTA's next patch arrive by two TMA boxes (as in patch_colour_kernel)
// into the other input slot while the current patch is computed; without it
// they are read element by element into the same layout.
template <int DIM, int K, int NT, bool TMA>
__global__ void __launch_bounds__(NT) patch_var_kernel(T* __restrict__ u, const T* __restrict__ b,
                                                       const T* __restrict__ coef,
                                                       const T* __restrict__ vscale,
                                                       const T* __restrict__ dinv,
                                                       const float* __restrict__ corr, int rank,
                                                       PatchLaunch pl,
                                                       const __grid_constant__ TmaMaps<TMA ? 1 : 0> maps,
                                                       int* __restrict__ err) {
  using Z = SweepSmem<DIM, K, TMA>;
  constexpr int C = 2 * K + 1, M = 2 * K - 1, E = K + 1, XU = Z::XU, XB = Z::XB;
  constexpr int NINT = DIM == 3 ? M * M * M : M * M;
  constexpr int NE = DIM == 3 ? E * E * E : E * E;
  constexpr int NCELL = 1 << DIM;
  // FP64 problems compute in double-float arithmetic on float pairs held in
  // the double-sized work buffers; u, b and the coefficients stay FP64
  constexpr bool DF = sizeof(T) == 8;
  // input slots: closure of u (rows of XU), then interior of b (rows of XB)
  __shared__ __align__(128) T IN[TMA ? 2 : 1][Z::IN];
  __shared__ T R[NINT], RS[NINT];
  __shared__ __align__(8) uint64_t s_bar[2];
  __shared__ int s_shift[2];
  __shared__ T X[NCELL * NE], P[NCELL * NE], Q[NCELL * NE], A1[NCELL * NE], A2[NCELL * NE];
  __shared__ T s_coef[NCELL];
  __shared__ float2 s_coef2[NCELL];
  // the patch's correction block (U then s), prefetched while the residual
  // and the FD solve are computed (rank <= 4)
  __shared__ float s_corr[NINT * 4 + 4];
  __shared__ T s_scale, s_theta;
  __shared__ float s_t[8];
  const long long py = pl.g.py, pz = pl.g.pz;
  const int n = pl.g.n;
  const T sb = (T)pl.sb, om = (T)pl.omega;
  // vertex of patch pid of the colour
  auto vertex = [&](int pid, int& v0, int& v1, int& v2) {
    const int i0 = pid % pl.count[0];
    const int rest = pid / pl.count[0];
    const int i1 = rest % pl.count[1];
    const int i2 = DIM == 3 ? rest / pl.count[1] : 0;
    v0 = pl.first[0] + 2 * i0;
    v1 = pl.first[1] + 2 * i1;
    v2 = DIM == 3 ? pl.first[2] + 2 * i2 : 1;
  };
  auto uo = [](int x, int y, int z) { return DIM == 3 ? (z * C + y) * XU + x : y * XU + x; };
  auto bo = [](int x, int y, int z) { return DIM == 3 ? (z * M + y) * XB + x : y * XB + x; };
  // TMA boxes of patch pid into slot (one thread)
  auto issue = [&](int pid, int slot) {
    if constexpr (TMA) {
      int v0, v1, v2;
      vertex(pid, v0, v1, v2);
      const int x0 = (v0 - 1) * K, y0 = (v1 - 1) * K, z0 = DIM == 3 ? (v2 - 1) * K : 0;
      const int xa = x0 - x0 % Z::A;
      s_shift[slot] = x0 - xa;
      async::mbar_arrive_expect_tx(&s_bar[slot], (uint32_t)(Z::BOX_U + Z::BOX_B));
      if (DIM == 3) {
        async::tma_load_3d(IN[slot], &maps.u[0], xa, y0, z0, &s_bar[slot]);
        async::tma_load_3d(IN[slot] + Z::NCLO, &maps.b[0], xa, y0 + 1, z0 + 1, &s_bar[slot]);
      } else {
        async::tma_load_2d(IN[slot], &maps.u[0], xa, y0, &s_bar[slot]);
        async::tma_load_2d(IN[slot] + Z::NCLO, &maps.b[0], xa, y0 + 1, &s_bar[slot]);
      }
    }
  };
  uint32_t phase = 0;
  bool wait_ok = true;
  if (TMA && threadIdx.x == 0) {
    async::mbar_init(&s_bar[0], 1);
    async::mbar_init(&s_bar[1], 1);
    if ((int)blockIdx.x < pl.n_patches) issue(blockIdx.x, 0);
  }
  if (TMA) __syncthreads();  // barriers initialised before anyone waits on them
  int it = 0;
  for (int pid = blockIdx.x; pid < pl.n_patches; pid += gridDim.x, ++it) {
    const int cur = TMA ? (it & 1) : 0;
    int v0, v1, v2;
    vertex(pid, v0, v1, v2);
    const long long origin = (long long)(v0 - 1) * K + py * ((v1 - 1) * K) + (DIM == 3 ? pz * ((v2 - 1) * K) : 0);
    if (TMA && threadIdx.x == 0 && pid + (int)gridDim.x < pl.n_patches) issue(pid + gridDim.x, cur ^ 1);
    if (corr) {
      const int vid = (v0 - 1) + (n - 1) * ((v1 - 1) + (DIM == 3 ? (n - 1) * (v2 - 1) : 0));
      const float* Up = corr + (long long)vid * (NINT * rank + rank);
      for (int i = threadIdx.x; i < NINT * rank + rank; i += NT)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(async::smem_u32(s_corr + i)), "l"(Up + i)
                     : "memory");
      asm volatile("cp.async.commit_group;\n" ::: "memory");
    }
    if constexpr (!TMA) {  // element-wise gather into the slot layout (XU = C, XB = M)
      for (int t = threadIdx.x; t < (DIM == 3 ? C * C * C : C * C); t += NT) {
        const int x = t % C, y = (t / C) % C, z = DIM == 3 ? t / (C * C) : 0;
        IN[0][t] = u[origin + x + py * y + pz * z];
      }
      for (int t = threadIdx.x; t < NINT; t += NT) {
        const int x = t % M, y = (t / M) % M, z = DIM == 3 ? t / (M * M) : 0;
        IN[0][Z::NCLO + t] = b[origin + 1 + x + py * (y + 1) + (DIM == 3 ? pz * (z + 1) : 0)];
      }
    } else {
      if (wait_ok && !async::mbar_wait(&s_bar[cur], (phase >> cur) & 1u)) wait_ok = false;
      phase ^= 1u << cur;
    }
    if (threadIdx.x < NCELL) {
      const int o0 = threadIdx.x & 1, o1 = (threadIdx.x >> 1) & 1, o2 = (threadIdx.x >> 2) & 1;
      const long long c = (long long)(v0 - 1 + o0) + (long long)n * ((v1 - 1 + o1) + (DIM == 3 ? (long long)n * (v2 - 1 + o2) : 0));
      s_coef[threadIdx.x] = coef[c];
      if constexpr (DF) {
        const dfv a = df_from_double(coef[c]);
        s_coef2[threadIdx.x] = make_float2(a.hi, a.lo);
      }
    }
    __syncthreads();
    const T* const U = IN[cur] + (TMA ? s_shift[cur] : 0);                   // closure (x, y, z)
    const T* const Bv = IN[cur] + Z::NCLO + (TMA ? s_shift[cur] + 1 : 0);   // interior of b
    if (threadIdx.x == 0) {  // the scatter's scale: omega / abar, times theta without the correction
      const int vid = (v0 - 1) + (n - 1) * ((v1 - 1) + (DIM == 3 ? (n - 1) * (v2 - 1) : 0));
      const T abar = vscale[2 * (long long)vid], theta = vscale[2 * (long long)vid + 1];
      s_theta = theta;
      s_scale = corr ? om / abar : om * theta / abar;
    }
    // ---- local residual: the 2^d cell operators of the patch at once, then
    // R = sum_c a_c [A_c u_c]_interior node by node (cells in ascending order) ----
    for (int t = threadIdx.x; t < NCELL * NE; t += NT) {
      const int c = t / NE, l = t % NE;
      const int o0 = c & 1, o1 = (c >> 1) & 1, o2 = (c >> 2) & 1;
      const int x = l % E, y = (l / E) % E, z = DIM == 3 ? l / (E * E) : 0;
      const T v = U[uo(o0 * K + x, o1 * K + y, DIM == 3 ? o2 * K + z : 0)];
      if constexpr (DF) {
        const dfv d = df_from_double(v);
        reinterpret_cast<float2*>(X)[t] = make_float2(d.hi, d.lo);
      } else {
        X[t] = v;
      }
    }
    __syncthreads();
    float2* const R2 = reinterpret_cast<float2*>(R);
    float2* const RS2 = reinterpret_cast<float2*>(RS);
    if constexpr (DF) {
      float2* const X2 = reinterpret_cast<float2*>(X);
      cell_operator_df<DIM, K, NT>(X2, reinterpret_cast<float2*>(P), reinterpret_cast<float2*>(Q),
                                   reinterpret_cast<float2*>(A1), reinterpret_cast<float2*>(A2), X2, NCELL, NE);
      // R = sum_c a_c [A_c u_c]_interior, then r_ref = h^{2-d} b - R
      const float sbf = (float)pl.sb;  // an integer power of the cell count, exact in float
      for (int t = threadIdx.x; t < NINT; t += NT) {
        const int x = t % M + 1, y = (t / M) % M + 1, z = DIM == 3 ? t / (M * M) + 1 : 0;
        df_acc acc = {0.f, 0.f};
#pragma unroll
        for (int c = 0; c < NCELL; ++c) {
          const int lx = x - (c & 1) * K, ly = y - ((c >> 1) & 1) * K, lz = DIM == 3 ? z - ((c >> 2) & 1) * K : 0;
          if (lx < 0 || lx > K || ly < 0 || ly > K || lz < 0 || lz > K) continue;
          const float2 xv = X2[c * NE + lx + E * ly + (DIM == 3 ? E * E * lz : 0)];
          df_acc_add(acc, s_coef2[c].x, s_coef2[c].y, {xv.x, xv.y});
        }
        const dfv bv = df_from_double(Bv[bo(t % M, (t / M) % M, DIM == 3 ? t / (M * M) : 0)]);
        const dfv r = df_add(df_mul(bv, {sbf, 0.f}), df_neg(df_acc_value(acc)));
        R2[t] = make_float2(r.hi, r.lo);
        RS2[t] = R2[t];
      }
      __syncthreads();
    } else {
    cell_operator<DIM, K, NT>(X, P, Q, A1, A2, X, NCELL, NE);
    for (int t = threadIdx.x; t < NINT; t += NT) {
      const int x = t % M + 1, y = (t / M) % M + 1, z = DIM == 3 ? t / (M * M) + 1 : 0;  // closure coords
      T acc = T(0);
#pragma unroll
      for (int c = 0; c < NCELL; ++c) {
        const int lx = x - (c & 1) * K, ly = y - ((c >> 1) & 1) * K, lz = DIM == 3 ? z - ((c >> 2) & 1) * K : 0;
        if (lx < 0 || lx > K || ly < 0 || ly > K || lz < 0 || lz > K) continue;
        acc += s_coef[c] * X[c * NE + lx + E * ly + (DIM == 3 ? E * E * lz : 0)];
      }
      R[t] = acc;
    }
    __syncthreads();
    // ---- reference residual r_ref = h^{2-d} b - R ----
    for (int t = threadIdx.x; t < NINT; t += NT) {
      const T r = sb * Bv[bo(t % M, (t / M) % M, DIM == 3 ? t / (M * M) : 0)] - R[t];
      RS[t] = r;
      R[t] = r;
    }
    __syncthreads();
    }
    // ---- fast diagonalisation of the constant-coefficient patch ----
    if constexpr (DF) {
      for (int a = 0; a < DIM; ++a) {
        for (int l = threadIdx.x; l < (DIM == 3 ? M * M : M); l += NT) {
          if (a == 0) fd_smem_line_df<K, true>(R2 + l * M, 1);
          else if (a == 1) fd_smem_line_df<K, true>(R2 + (l % M) + (DIM == 3 ? (l / M) * M * M : 0), M);
          else fd_smem_line_df<K, true>(R2 + l, M * M);
        }
        __syncthreads();
      }
      const float2* const d2 = reinterpret_cast<const float2*>(dinv + NINT);  // the diagonal as float pairs
      for (int t = threadIdx.x; t < NINT; t += NT) {
        const float2 a = R2[t], d = __ldg(d2 + t);
        const dfv v = df_mul({a.x, a.y}, {d.x, d.y});
        R2[t] = make_float2(v.hi, v.lo);
      }
      __syncthreads();
      for (int a = 0; a < DIM; ++a) {
        for (int l = threadIdx.x; l < (DIM == 3 ? M * M : M); l += NT) {
          if (a == 0) fd_smem_line_df<K, false>(R2 + l * M, 1);
          else if (a == 1) fd_smem_line_df<K, false>(R2 + (l % M) + (DIM == 3 ? (l / M) * M * M : 0), M);
          else fd_smem_line_df<K, false>(R2 + l, M * M);
        }
        __syncthreads();
      }
    } else {
    for (int a = 0; a < DIM; ++a) {
      for (int l = threadIdx.x; l < (DIM == 3 ? M * M : M); l += NT) {
        if (a == 0) fd_smem_line<K, true>(R + l * M, 1);
        else if (a == 1) fd_smem_line<K, true>(R + (l % M) + (DIM == 3 ? (l / M) * M * M : 0), M);
        else fd_smem_line<K, true>(R + l, M * M);
      }
      __syncthreads();
    }
    for (int t = threadIdx.x; t < NINT; t += NT) R[t] *= dinv[t];
    __syncthreads();
    for (int a = 0; a < DIM; ++a) {
      for (int l = threadIdx.x; l < (DIM == 3 ? M * M : M); l += NT) {
        if (a == 0) fd_smem_line<K, false>(R + l * M, 1);
        else if (a == 1) fd_smem_line<K, false>(R + (l % M) + (DIM == 3 ? (l / M) * M * M : 0), M);
        else fd_smem_line<K, false>(R + l, M * M);
      }
      __syncthreads();
    }
    }
    // ---- learned rank-R correction U diag(s) U^T r_ref (block prefetched) ----
    if (corr) {
      asm volatile("cp.async.wait_group 0;\n" ::: "memory");
      __syncthreads();
      const float* Up = s_corr;
      const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
      for (int q = warp; q < rank; q += NT / 32) {
        float acc = 0.f;
        for (int i = lane; i < NINT; i += 32) acc += Up[i * rank + q] * (DF ? RS2[i].x : (float)RS[i]);
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) s_t[q] = acc * Up[NINT * rank + q];
      }
      __syncthreads();
      for (int i = threadIdx.x; i < NINT; i += NT) {
        float acc = 0.f;
        for (int q = 0; q < rank; ++q) acc += Up[i * rank + q] * s_t[q];
        if constexpr (DF) {
          const float2 a = R2[i];
          const dfv v = df_add(df_mul({a.x, a.y}, df_from_double(s_theta)), {acc, 0.f});
          R2[i] = make_float2(v.hi, v.lo);
        } else {
          R[i] = fma(s_theta, R[i], (T)acc);
        }
      }
      __syncthreads();
    }
    // ---- scatter: u += omega d / abar ----
    const T scale = s_scale;
    for (int t = threadIdx.x; t < NINT; t += NT) {
      const int x = t % M, y = (t / M) % M, z = DIM == 3 ? t / (M * M) : 0;
      const long long gi = origin + 1 + x + py * (y + 1) + (DIM == 3 ? pz * (z + 1) : 0);
      if constexpr (DF) {
        const float2 a = R2[t];
        u[gi] = fma(scale, df_to_double({a.x, a.y}), u[gi]);
      } else {
        u[gi] = fma(scale, R[t], u[gi]);
      }
    }
    if (TMA) async::fence_proxy_async();  // slot reads before the next TMA writes into it
    __syncthreads();
  }
  if (TMA && !wait_ok) atomicExch(err, GMG_ERR_TIMEOUT);
}

}  // namespace GMG_NS
}  // namespace gmg

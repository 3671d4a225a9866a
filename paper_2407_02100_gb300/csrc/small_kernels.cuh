// Coarse-level sweep of FP64 problems (double-float arithmetic, one output
// per thread).
//
// On the coarse levels of a V-cycle a colour holds a few hundred patches or
// fewer: one CTA per patch, and the colour step lasts as long as one patch
// takes.  The line kernels (closure and shared-face forms) give a thread a
// whole line of a stage, 2(2k-1) outputs accumulated in double-float one
// after the other, so a single patch takes about 20 us per colour step at
// k = 4 however few patches there are.  This kernel computes the same colour
// step (Algorithm 4: local residual by sum factorisation on the closure,
// fast-diagonalisation solve, u += omega d) with one thread per output of a
// stage (its line read from shared memory), so each stage is a short chain
// of one output's terms and the patch goes through in a few microseconds.
// Every stage reads one shared-memory array and writes another.
//
// Included by patch_f64.cu and patch_f32.cu after patch_kernels.cuh; only
// FP64 problems launch it.
#pragma once

namespace gmg {
namespace GMG_NS {

template <int DIM, int K>
struct WideSmem {
  static constexpr int C = 2 * K + 1, M = 2 * K - 1;
  static constexpr int NINT = DIM == 3 ? M * M * M : M * M;
  // X: the closure of u, then (3D) the stage-y results A1, A2, then FD work;
  // Y: the stage-z results P, Q (3D) or stage-y results (2D), then the
  // residual and FD work
  static constexpr int X = DIM == 3 ? cmax(C * C * C, 2 * C * M * M) : cmax(C * C, M * M);
  static constexpr int Y = DIM == 3 ? cmax(2 * C * C * M, NINT) : cmax(2 * C * M, NINT);
  // the patch matrices M_p, K_p (M x C) and the eigenvectors T (M x M) as
  // float pairs, copied from __constant__ memory once per CTA: a stage's
  // output index varies across the CTA, and shared-memory pairs take one
  // load where constant memory would take two serialised ones
  static constexpr int TAB = 2 * M * C + M * M;
  static constexpr int BYTES = (X + Y + TAB) * (int)sizeof(float2);
  // outputs of the largest stage
  static constexpr int ITEMS = DIM == 3 ? C * C * M : C * M;
};

// threads per CTA: the largest stage in PASSES passes (128 to 1024 threads)
template <int DIM, int K, int PASSES>
constexpr int wide_threads() {
  constexpr int items = WideSmem<DIM, K>::ITEMS;
  constexpr int t = (items + PASSES - 1) / PASSES;
  return t <= 128 ? 128 : t >= 1024 ? 1024 : (t + 31) / 32 * 32;
}

// acc += sum over the band of closure row i + 1 of E (M_p or K_p, pairs in
// shared memory, rows of C) of E[i][j] x[j * s]: rows left of the patch
// centre couple to closure columns 0..k, rows right of it to k..2k, the
// centre row to all 2k + 1
template <int K>
__device__ __forceinline__ void wide_row(df_acc& acc, int i, const float2* E, const float2* x, int s) {
  constexpr int C = 2 * K + 1;
  const int j0 = i + 1 > K ? K : 0;
  const float2* const e = E + i * C;
#pragma unroll
  for (int q = 0; q <= K; ++q) {
    const int j = j0 + q;
    const float2 v = x[j * s], c = e[j];
    df_acc_add(acc, c.x, c.y, {v.x, v.y});
  }
  if (i + 1 == K) {  // the centre row also reaches the right cell
#pragma unroll
    for (int j = K + 1; j < C; ++j) {
      const float2 v = x[j * s], c = e[j];
      df_acc_add(acc, c.x, c.y, {v.x, v.y});
    }
  }
}

// output i of the FD transform of the line x (M values, stride s), T the
// eigenvector pairs in shared memory: forward sum_j T[j][i] x_j, backward
// sum_j T[i][j] x_j
template <int K, bool FORWARD>
__device__ __forceinline__ dfv wide_fd(int i, const float2* T, const float2* x, int s) {
  constexpr int M = 2 * K - 1;
  df_acc acc = {0.f, 0.f};
#pragma unroll
  for (int j = 0; j < M; ++j) {
    const float2 v = x[j * s], c = T[FORWARD ? j * M + i : i * M + j];
    df_acc_add(acc, c.x, c.y, {v.x, v.y});
  }
  return df_acc_value(acc);
}

template <int DIM, int K, int NT>
__global__ void __launch_bounds__(NT) patch_wide_df_kernel(const PatchLaunch pl, double* __restrict__ u,
                                                           const double* __restrict__ b,
                                                           const double* __restrict__ dinv) {
  using Z = WideSmem<DIM, K>;
  constexpr int C = Z::C, M = Z::M, NINT = Z::NINT;
  extern __shared__ __align__(16) float2 wide_smem[];
  float2* const X = wide_smem;
  float2* const Y = wide_smem + Z::X;
  float2* const Mp = Y + Z::Y;   // M x C pairs
  float2* const Kp = Mp + M * C;  // M x C pairs
  float2* const Tt = Kp + M * C;  // M x M pairs
  const float2* const dd = reinterpret_cast<const float2*>(dinv + NINT);  // the diagonal as float pairs
  const long long py = pl.g.py, pz = pl.g.pz;
  const int pid = blockIdx.x;
  const int i0 = pid % pl.count[0], rest = pid / pl.count[0];
  const int i1 = rest % pl.count[1], i2 = DIM == 3 ? rest / pl.count[1] : 0;
  const long long origin = (long long)(pl.first[0] + 2 * i0 - 1) * K + py * ((pl.first[1] + 2 * i1 - 1) * K) +
                           (DIM == 3 ? pz * ((pl.first[2] + 2 * i2 - 1) * K) : 0);
  auto st = [](const dfv a) -> float2 { return make_float2(a.hi, a.lo); };
  for (int t = threadIdx.x; t < M * C; t += NT) {
    Mp[t] = make_float2(c_Mphi[off_patch(K) + t], c_Mplo[off_patch(K) + t]);
    Kp[t] = make_float2(c_Kphi[off_patch(K) + t], c_Kplo[off_patch(K) + t]);
  }
  for (int t = threadIdx.x; t < M * M; t += NT) Tt[t] = make_float2(c_Thi[off_t(K) + t], c_Tlo[off_t(K) + t]);
  // ---- gather the closure of u as float pairs ([z][y][x]) ----
  for (int t = threadIdx.x; t < (DIM == 3 ? C * C * C : C * C); t += NT) {
    const int x = t % C, y = (t / C) % C, z = DIM == 3 ? t / (C * C) : 0;
    X[t] = st(df_from_double(u[origin + x + py * y + pz * z]));
  }
  __syncthreads();
  if (DIM == 3) {
    // ---- stage z: P = Mp_z u, Q = Kp_z u;  Y = P, Q [z][y][x], z interior ----
    for (int t = threadIdx.x; t < C * C * M; t += NT) {
      const int l = t % (C * C), i = t / (C * C);
      df_acc p = {0.f, 0.f}, q = {0.f, 0.f};
      wide_row<K>(p, i, Mp, X + l, C * C);
      wide_row<K>(q, i, Kp, X + l, C * C);
      Y[l + i * C * C] = st(df_acc_value(p));
      Y[C * C * M + l + i * C * C] = st(df_acc_value(q));
    }
    __syncthreads();
    // ---- stage y: A1 = Mp_y P, A2 = Kp_y P + Mp_y Q;  X = A1, A2 [z][y][x], y, z interior ----
    for (int t = threadIdx.x; t < C * M * M; t += NT) {
      const int x = t % C, z = (t / C) % M, i = t / (C * M);
      const int src = x + z * C * C;
      df_acc a1 = {0.f, 0.f}, a2 = {0.f, 0.f};
      wide_row<K>(a1, i, Mp, Y + src, C);
      wide_row<K>(a2, i, Kp, Y + src, C);
      wide_row<K>(a2, i, Mp, Y + C * C * M + src, C);
      X[x + i * C + z * C * M] = st(df_acc_value(a1));
      X[C * M * M + x + i * C + z * C * M] = st(df_acc_value(a2));
    }
    __syncthreads();
  } else {
    // ---- stage y: P = Mp_y u, Q = Kp_y u;  Y = P, Q [y][x], y interior ----
    for (int t = threadIdx.x; t < C * M; t += NT) {
      const int l = t % C, i = t / C;
      df_acc p = {0.f, 0.f}, q = {0.f, 0.f};
      wide_row<K>(p, i, Mp, X + l, C);
      wide_row<K>(q, i, Kp, X + l, C);
      Y[l + i * C] = st(df_acc_value(p));
      Y[C * M + l + i * C] = st(df_acc_value(q));
    }
    __syncthreads();
  }
  // ---- stage x: r = h^{2-d} b - (Kp_x X1 + Mp_x X2), interior [z][y][x] ----
  // (3D: from X into Y; 2D: from Y into X)
  {
    const float2* const S1 = DIM == 3 ? X : Y;
    float2* const R = DIM == 3 ? Y : X;
    constexpr int PLANE = DIM == 3 ? C * M * M : C * M;
    const float sbf = (float)pl.sb;  // h^{2-d}: the cell count in 3D, 1 in 2D, exact in float
    for (int t = threadIdx.x; t < NINT; t += NT) {
      const int i = t % M, l = t / M;  // x, and the line (y, z)
      const long long row = origin + 1 + py * ((DIM == 3 ? l % M : l) + 1) + (DIM == 3 ? pz * (l / M + 1) : 0);
      const dfv bb = df_mul(df_from_double(b[row + i]), {sbf, 0.f});
      df_acc acc = {0.f, 0.f};
      wide_row<K>(acc, i, Kp, S1 + C * l, 1);
      wide_row<K>(acc, i, Mp, S1 + PLANE + C * l, 1);
      R[t] = st(df_add(bb, df_neg(df_acc_value(acc))));
    }
  }
  __syncthreads();
  // ---- fast diagonalisation, one output per thread, ping-pong between the
  // two regions: forward x, y (, z), times the diagonal, backward ----
  float2* A = DIM == 3 ? Y : X;  // holds the residual
  float2* B = DIM == 3 ? X : Y;
  auto pass = [&](int axis, bool forward, bool scale) {
    for (int t = threadIdx.x; t < NINT; t += NT) {
      const int x = t % M, y = (t / M) % M, z = DIM == 3 ? t / (M * M) : 0;
      const int i = axis == 0 ? x : axis == 1 ? y : z;                      // output index on the line
      const int s = axis == 0 ? 1 : axis == 1 ? M : M * M;                   // line stride
      const float2* line = A + t - i * s;
      dfv v = forward ? wide_fd<K, true>(i, Tt, line, s) : wide_fd<K, false>(i, Tt, line, s);
      if (scale) {
        const float2 d = __ldg(dd + t);
        v = df_mul(v, {d.x, d.y});
      }
      B[t] = st(v);
    }
    __syncthreads();
    float2* const tmp = A;
    A = B;
    B = tmp;
  };
  pass(0, true, false);
  if (DIM == 3) {
    pass(1, true, false);
    pass(2, true, true);
    pass(2, false, false);
    pass(1, false, false);
  } else {
    pass(1, true, true);
    pass(1, false, false);
  }
  pass(0, false, false);
  // ---- scatter: u += omega d on the patch interior ----
  const double om = pl.omega;
  for (int t = threadIdx.x; t < NINT; t += NT) {
    const int x = t % M, y = (t / M) % M, z = DIM == 3 ? t / (M * M) : 0;
    const long long gi = origin + 1 + x + py * (y + 1) + (DIM == 3 ? pz * (z + 1) : 0);
    const float2 d = A[t];
    u[gi] = fma(om, df_to_double({d.x, d.y}), u[gi]);
  }
}

template <int DIM, int K, int NT>
static int wide_launch(const PatchLaunch& pl, T* u, const T* b, const T* dinv, cudaStream_t s) {
  using Z = WideSmem<DIM, K>;
  auto kern = patch_wide_df_kernel<DIM, K, NT>;
  static PerDevice<bool> ready_dev;
  bool* const ready = ready_dev.get();
  if (!ready) return GMG_ERR_CUDA;
  if (!*ready) {
    if (prepare(kern, Z::BYTES) != GMG_OK) return GMG_ERR_CUDA;
    *ready = true;
  }
  kern<<<pl.n_patches, NT, Z::BYTES, s>>>(pl, u, b, dinv);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? GMG_OK : GMG_ERR_CUDA;
}

template <int DIM, int K>
static int wide_impl(const PatchLaunch& pl, T* u, const T* b, const T* dinv, cudaStream_t s) {
  if constexpr (sizeof(T) != 8) {
    return GMG_ERR_UNSUPPORTED;
  } else {
    if (pl.n_patches <= 0) return GMG_OK;
    // fewer patches than SMs: each CTA has an SM to itself, so give it the
    // largest stage in one pass; otherwise two passes, for more resident CTAs
    if (pl.n_patches <= sm_count()) return wide_launch<DIM, K, wide_threads<DIM, K, 1>()>(pl, u, b, dinv, s);
    return wide_launch<DIM, K, wide_threads<DIM, K, 2>()>(pl, u, b, dinv, s);
  }
}

}  // namespace GMG_NS

template <>
int launch_patch_small<GMG_T>(const PatchLaunch& pl, GMG_T* u, const GMG_T* b, const GMG_T* dinv,
                              cudaStream_t s) {
  if (pl.mode != 0 || pl.plist) return GMG_ERR_UNSUPPORTED;
  GMG_DISPATCH(GMG_NS::wide_impl, pl.g.dim, pl.g.k, pl, u, b, dinv, s)
}

}  // namespace gmg

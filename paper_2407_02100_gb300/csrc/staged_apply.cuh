// Halo-free FP64 form of the 3D level operator: three passes over the
// level, one per axis, each a 1D contraction with the global 1D matrices
// (unit-cell mass M and stiffness K assembled along one axis), through two
// pairs of workspace vectors:
//   pass z: P = M_z u,  Q = K_z u
//   pass y: A1 = M_y P, A2 = K_y P + M_y Q
//   pass x: y = alpha (K_x A1 + M_x A2) + beta b     (interior nodes)
// which is A = K (x) M (x) M + M (x) K (x) M + M (x) M (x) K by sum
// factorisation (Sec. 2, App. A.1 with the cell integrals summed into
// global rows).  The tile kernel recomputes a halo of up to K + 1 nodes per
// direction in its first two stages; here every output row is evaluated
// once, for ten passes of level vectors through HBM.  Included by
// patch_f64.cu after patch_kernels.cuh (T = double).
#pragma once

namespace gmg {
namespace GMG_NS {

// One thread evaluates the K global rows of nodes c K .. c K + K - 1 along
// AX (cell c of that axis) at one position of the other two axes, from the
// 2K + 1 inputs c K - K .. c K + K of each input vector (zero outside the
// lattice).  Row c K (a vertex) is row K of cell c - 1 plus row 0 of cell c;
// row c K + p (0 < p < K) is row p of cell c.
//   AX 2: positions all (x, y), rows z interior;  in0 = u -> out0 = M in0, out1 = K in0
//   AX 1: positions all x, z interior, rows y interior;
//         in0 = P, in1 = Q -> out0 = M P, out1 = K P + M Q
//   AX 0: positions y, z interior, rows x interior;
//         in0 = A1, in1 = A2 -> out0 = alpha (K A1 + M A2) + beta b
template <int K, int AX>
__global__ void __launch_bounds__(128) axis_pass_kernel(const T* __restrict__ in0, const T* __restrict__ in1,
                                                        T* __restrict__ out0, T* __restrict__ out1,
                                                        const T* __restrict__ bvec, const LevelGeom g, T alpha,
                                                        T beta) {
  constexpr int W = 2 * K + 1;
  const int N = g.N, n = g.n;
  const long long py = g.py, pz = g.pz;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int x, y, z, c;
  long long stride;
  if (AX == 2) {
    if (t >= (long long)N * N * n) return;
    x = (int)(t % N);
    const long long r = t / N;
    y = (int)(r % N);
    c = (int)(r / N);
    z = 0;
    stride = pz;
  } else if (AX == 1) {
    if (t >= (long long)N * (N - 2) * n) return;
    x = (int)(t % N);
    const long long r = t / N;
    z = 1 + (int)(r % (N - 2));
    c = (int)(r / (N - 2));
    y = 0;
    stride = py;
  } else {
    if (t >= (long long)n * (N - 2) * (N - 2)) return;
    c = (int)(t % n);
    const long long r = t / n;
    y = 1 + (int)(r % (N - 2));
    z = 1 + (int)(r / (N - 2));
    x = 0;
    stride = 1;
  }
  // element offset of node c K - K of the thread's line
  const long long base = x + py * y + pz * z + stride * ((long long)c * K - K);
  auto E = [](int kind, int r, int q) -> T {
    return kind == 0 ? c_Mc[off_cell(K) + r * (K + 1) + q] : c_Kc[off_cell(K) + r * (K + 1) + q];
  };
  T a[W], b[AX == 2 ? 1 : W];
#pragma unroll
  for (int w = 0; w < W; ++w) {
    const int node = c * K - K + w;
    const bool ok = node >= 0 && node < N;
    a[w] = ok ? in0[base + stride * w] : T(0);
    if constexpr (AX != 2) b[w] = ok ? in1[base + stride * w] : T(0);
  }
  // global row p of the segment, matrix kind, applied to the window v
  auto row = [&](int p, int kind, const T (&v)[W], T acc) -> T {
    if (p == 0) {
#pragma unroll
      for (int q = 0; q <= K; ++q) acc = fma(E(kind, K, q), v[q], acc);
    }
#pragma unroll
    for (int q = 0; q <= K; ++q) acc = fma(E(kind, p, q), v[K + q], acc);
    return acc;
  };
#pragma unroll
  for (int p = 0; p < K; ++p) {
    const int node = c * K + p;
    if (node < 1 || node > N - 2) continue;
    const long long o = base + stride * (K + p);
    if constexpr (AX == 2) {
      out0[o] = row(p, 0, a, T(0));
      out1[o] = row(p, 1, a, T(0));
    } else if constexpr (AX == 1) {
      out0[o] = row(p, 0, a, T(0));
      out1[o] = row(p, 0, b, row(p, 1, a, T(0)));
    } else {
      T v = alpha * row(p, 0, b, row(p, 1, a, T(0)));
      if (bvec) v = fma(beta, bvec[o], v);
      out0[o] = v;
    }
  }
}

// The same three passes in double-float arithmetic (FP64 problems; GB300
// runs FP64 at about 1/74 of its FP32 rate): the workspace vectors hold
// float pairs (hi, lo) in the 8 bytes of a double, the rows accumulate in
// Dot2 form with the float-pair cell matrices, and the x pass forms
// alpha (K A1 + M A2) + beta b in FP64 from the pair's value (two FP64
// operations per node).
template <int K, int AX>
__global__ void __launch_bounds__(128) axis_pass_df_kernel(const void* __restrict__ in0v,
                                                           const float2* __restrict__ in1,
                                                           float2* __restrict__ out0, float2* __restrict__ out1,
                                                           double* __restrict__ yout, const double* __restrict__ bvec,
                                                           const LevelGeom g, double alpha, double beta) {
  constexpr int W = 2 * K + 1;
  const int N = g.N, n = g.n;
  const long long py = g.py, pz = g.pz;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int x, y, z, c;
  long long stride;
  if (AX == 2) {
    if (t >= (long long)N * N * n) return;
    x = (int)(t % N);
    const long long r = t / N;
    y = (int)(r % N);
    c = (int)(r / N);
    z = 0;
    stride = pz;
  } else if (AX == 1) {
    if (t >= (long long)N * (N - 2) * n) return;
    x = (int)(t % N);
    const long long r = t / N;
    z = 1 + (int)(r % (N - 2));
    c = (int)(r / (N - 2));
    y = 0;
    stride = py;
  } else {
    if (t >= (long long)n * (N - 2) * (N - 2)) return;
    c = (int)(t % n);
    const long long r = t / n;
    y = 1 + (int)(r % (N - 2));
    z = 1 + (int)(r / (N - 2));
    x = 0;
    stride = 1;
  }
  const long long base = x + py * y + pz * z + stride * ((long long)c * K - K);
  dfv a[W], b[AX == 2 ? 1 : W];
#pragma unroll
  for (int w = 0; w < W; ++w) {
    const int node = c * K - K + w;
    const bool ok = node >= 0 && node < N;
    if constexpr (AX == 2) {
      a[w] = ok ? df_from_double(static_cast<const double*>(in0v)[base + stride * w]) : dfv{0.f, 0.f};
    } else {
      const float2 va = ok ? static_cast<const float2*>(in0v)[base + stride * w] : make_float2(0.f, 0.f);
      const float2 vb = ok ? in1[base + stride * w] : make_float2(0.f, 0.f);
      a[w] = {va.x, va.y};
      b[w] = {vb.x, vb.y};
    }
  }
  // acc += global row p of the cell matrix `kind` applied to the window v
  auto row = [&](int p, int kind, const dfv (&v)[W], df_acc& acc) {
    auto eh = [&](int r, int q) { return kind == 0 ? c_Mchi[off_cell(K) + r * (K + 1) + q] : c_Kchi[off_cell(K) + r * (K + 1) + q]; };
    auto el = [&](int r, int q) { return kind == 0 ? c_Mclo[off_cell(K) + r * (K + 1) + q] : c_Kclo[off_cell(K) + r * (K + 1) + q]; };
    if (p == 0) {
#pragma unroll
      for (int q = 0; q <= K; ++q) df_acc_add(acc, eh(K, q), el(K, q), v[q]);
    }
#pragma unroll
    for (int q = 0; q <= K; ++q) df_acc_add(acc, eh(p, q), el(p, q), v[K + q]);
  };
#pragma unroll
  for (int p = 0; p < K; ++p) {
    const int node = c * K + p;
    if (node < 1 || node > N - 2) continue;
    const long long o = base + stride * (K + p);
    df_acc r0 = {0.f, 0.f}, r1 = {0.f, 0.f};
    if constexpr (AX == 2) {
      row(p, 0, a, r0);
      row(p, 1, a, r1);
      const dfv v0 = df_acc_value(r0), v1 = df_acc_value(r1);
      out0[o] = make_float2(v0.hi, v0.lo);
      out1[o] = make_float2(v1.hi, v1.lo);
    } else if constexpr (AX == 1) {
      row(p, 0, a, r0);
      row(p, 1, a, r1);
      row(p, 0, b, r1);
      const dfv v0 = df_acc_value(r0), v1 = df_acc_value(r1);
      out0[o] = make_float2(v0.hi, v0.lo);
      out1[o] = make_float2(v1.hi, v1.lo);
    } else {
      row(p, 1, a, r0);
      row(p, 0, b, r0);
      double v = alpha * df_to_double(df_acc_value(r0));
      if (bvec) v = fma(beta, bvec[o], v);
      yout[o] = v;
    }
  }
}

template <int K>
static int staged_apply_impl(const ApplyLaunch& al, const T* x, T* y, const T* bvec, cudaStream_t s) {
  const LevelGeom& g = al.g;
  const long long ne = g.pz * g.N;
  T* P = static_cast<T*>(al.ws);
  T* Q = P + ne;
  T* A1 = Q + ne;
  T* A2 = A1 + ne;
  const long long N = g.N, n = g.n;
  const long long t2 = N * N * n, t1 = N * (N - 2) * n, t0 = n * (N - 2) * (N - 2);
  auto blocks = [](long long t) { return (unsigned)((t + 127) / 128); };
  if constexpr (sizeof(T) == 8) {  // double-float passes (pairs in the workspace)
    float2 *P2 = reinterpret_cast<float2*>(P), *Q2 = reinterpret_cast<float2*>(Q);
    float2 *A12 = reinterpret_cast<float2*>(A1), *A22 = reinterpret_cast<float2*>(A2);
    axis_pass_df_kernel<K, 2><<<blocks(t2), 128, 0, s>>>(x, nullptr, P2, Q2, nullptr, nullptr, g, 0.0, 0.0);
    axis_pass_df_kernel<K, 1><<<blocks(t1), 128, 0, s>>>(P2, Q2, A12, A22, nullptr, nullptr, g, 0.0, 0.0);
    axis_pass_df_kernel<K, 0><<<blocks(t0), 128, 0, s>>>(A12, A22, nullptr, nullptr, y, bvec, g, al.alpha,
                                                        al.beta);
  } else {
    axis_pass_kernel<K, 2><<<blocks(t2), 128, 0, s>>>(x, nullptr, P, Q, nullptr, g, T(0), T(0));
    axis_pass_kernel<K, 1><<<blocks(t1), 128, 0, s>>>(P, Q, A1, A2, nullptr, g, T(0), T(0));
    axis_pass_kernel<K, 0><<<blocks(t0), 128, 0, s>>>(A1, A2, y, nullptr, bvec, g, (T)al.alpha, (T)al.beta);
  }
  count_launch(3);
  return cudaGetLastError() == cudaSuccess ? GMG_OK : GMG_ERR_CUDA;
}

}  // namespace GMG_NS
}  // namespace gmg

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
  axis_pass_kernel<K, 2><<<blocks(t2), 128, 0, s>>>(x, nullptr, P, Q, nullptr, g, T(0), T(0));
  axis_pass_kernel<K, 1><<<blocks(t1), 128, 0, s>>>(P, Q, A1, A2, nullptr, g, T(0), T(0));
  axis_pass_kernel<K, 0><<<blocks(t0), 128, 0, s>>>(A1, A2, y, nullptr, bvec, g, (T)al.alpha, (T)al.beta);
  count_launch(3);
  return cudaGetLastError() == cudaSuccess ? GMG_OK : GMG_ERR_CUDA;
}

}  // namespace GMG_NS
}  // namespace gmg

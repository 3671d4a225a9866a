// Learned correction of the fast-diagonalisation local solver for the
// variable-coefficient smoother (no counterpart in the paper; it extends the
// paper's remark that approximate local solvers fit the subspace-correction
// framework, Sec. 2.1).
//
// For a patch with cell coefficients a_c, normalised w_c = a_c / abar
// (abar = geometric mean), the exact reference-unit local inverse is
// Ahat(w)^{-1}; plain FD uses Ahat(1)^{-1}.  A two-layer perceptron maps the
// features x_c = log w_c to a symmetric rank-R correction U diag(s) U^T of
// the damped FD inverse theta Ahat(1)^{-1}, theta = min(1, 1.8 / max_c w_c):
//     h = tanh(W1 x + b1),  o = W2 h + b2,  U[i][q] = o[i R + q],  s[q] = o[m^d R + q]
// trained on exact patch solves generated here (dense Cholesky per patch,
// FP64) with the loss ||theta FD r + U diag(s) U^T r - Ahat(w)^{-1} r||^2 / ||Ahat(w)^{-1} r||^2.
// Training runs on the GPU with these kernels (forward, loss gradient,
// backward, Adam), master weights FP32; inference uses FP16-rounded weights
// with FP32 accumulation.  Plain FD stays the fallback and the judge: after
// inference each patch keeps its correction only if it lowers the local
// energy-norm error on a probe residual.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <random>
#include <vector>

#include "../../include/gmg.h"
#include "kernels.h"
#include "problem.h"
#include "setup.h"

using namespace gmg;
using namespace gmg::detail;

namespace {

constexpr int kMaxK = 3;
constexpr int kHidden = 32;
constexpr int kRank = 4;
// unit-cell 1D matrices (FP64) of degree <= kMaxK, and the reference FD data
__constant__ double l_Mc[(kMaxK + 1) * (kMaxK + 1)];
__constant__ double l_Kc[(kMaxK + 1) * (kMaxK + 1)];
__constant__ double l_T[(2 * kMaxK - 1) * (2 * kMaxK - 1)];

struct Shape {
  int dim, k, m, nint, ncell;  // m = 2k-1, nint = m^dim, ncell = 2^dim
  int nf, nh, rank, no;         // features, hidden, rank, outputs
  int np() const { return nh * nf + nh + no * nh + no; }
};

Shape make_shape(int dim, int k, int rank, int nh) {
  Shape s;
  s.dim = dim;
  s.k = k;
  s.m = 2 * k - 1;
  s.nint = dim == 3 ? s.m * s.m * s.m : s.m * s.m;
  s.ncell = 1 << dim;
  s.nf = s.ncell;
  s.nh = nh;
  s.rank = rank;
  s.no = s.nint * rank + rank;
  return s;
}

// entry (i, j) (closure coordinates 1..2k-1) of the cell-o 1D matrix embedded
// in the two-cell patch
__device__ __forceinline__ double emb(bool stiff, int o, int k, int i, int j) {
  const int a = i - o * k, b = j - o * k;
  if (a < 0 || a > k || b < 0 || b > k) return 0.0;
  return stiff ? l_Kc[a * (k + 1) + b] : l_Mc[a * (k + 1) + b];
}

// Exact reference solve of one patch per CTA: assemble Ahat(w) densely,
// Cholesky in shared memory, solve for r.  Outputs d_ex and d_fd = theta FD r
// (FD by dense tensor application of T diag(dinv) T^T).  When `corr` is given
// (gate mode), compares the energy-norm errors of FD and FD + correction and
// zeroes the correction's s entries if it does not help.
__global__ void exact_patch_kernel(Shape sh, int n, const double* __restrict__ W, const double* __restrict__ R,
                                   const double* __restrict__ dinv, double* __restrict__ DEX,
                                   double* __restrict__ DFD, float* __restrict__ corr,
                                   int* __restrict__ kept) {
  extern __shared__ double sm[];
  const int N = sh.nint, k = sh.k, m = sh.m, dim = sh.dim;
  double* A = sm;              // N x N
  double* x = A + N * N;       // rhs / solution
  double* r = x + N;
  double* t = r + N;           // FD work
  double* e1 = t + N;
  double* e2 = e1 + N;
  __shared__ double s_w[8];
  __shared__ double s_red[2];
  __shared__ float s_tq[8];
  for (int smp = blockIdx.x; smp < n; smp += gridDim.x) {
    if (threadIdx.x < sh.ncell) s_w[threadIdx.x] = W[(long long)smp * sh.ncell + threadIdx.x];
    for (int i = threadIdx.x; i < N; i += blockDim.x) r[i] = R[(long long)smp * N + i];
    __syncthreads();
    double wmax = s_w[0];
    for (int o = 1; o < sh.ncell; ++o) wmax = fmax(wmax, s_w[o]);
    const double theta = fmin(1.0, 1.8 / wmax);  // the FD damping (w has geometric mean 1)
    // ---- assemble Ahat(w) ----
    for (int idx = threadIdx.x; idx < N * N; idx += blockDim.x) {
      const int I = idx / N, J = idx % N;
      int ii[3] = {I % m + 1, (I / m) % m + 1, dim == 3 ? I / (m * m) + 1 : 0};
      int jj[3] = {J % m + 1, (J / m) % m + 1, dim == 3 ? J / (m * m) + 1 : 0};
      double v = 0.0;
      for (int o = 0; o < sh.ncell; ++o) {
        const int oo[3] = {o & 1, (o >> 1) & 1, (o >> 2) & 1};
        double sum_a = 0.0;
        for (int al = 0; al < dim; ++al) {
          double prod = 1.0;
          for (int be = 0; be < dim; ++be) prod *= emb(al == be, oo[be], k, ii[be], jj[be]);
          sum_a += prod;
        }
        v += s_w[o] * sum_a;
      }
      A[idx] = v;
    }
    __syncthreads();
    // ---- Cholesky A = L L^T (lower part of A) ----
    for (int j = 0; j < N; ++j) {
      if (threadIdx.x == 0) A[j * N + j] = sqrt(A[j * N + j]);
      __syncthreads();
      for (int i = j + 1 + threadIdx.x; i < N; i += blockDim.x) A[i * N + j] /= A[j * N + j];
      __syncthreads();
      const int rem = N - j - 1;
      for (int idx = threadIdx.x; idx < rem * rem; idx += blockDim.x) {
        const int i = j + 1 + idx / rem, c = j + 1 + idx % rem;
        if (c <= i) A[i * N + c] -= A[i * N + j] * A[c * N + j];
      }
      __syncthreads();
    }
    // ---- solve L L^T x = r (column-oriented substitution) ----
    for (int i = threadIdx.x; i < N; i += blockDim.x) x[i] = r[i];
    __syncthreads();
    for (int j = 0; j < N; ++j) {
      if (threadIdx.x == 0) x[j] /= A[j * N + j];
      __syncthreads();
      for (int i = j + 1 + threadIdx.x; i < N; i += blockDim.x) x[i] -= A[i * N + j] * x[j];
      __syncthreads();
    }
    for (int j = N - 1; j >= 0; --j) {
      if (threadIdx.x == 0) x[j] /= A[j * N + j];
      __syncthreads();
      for (int i = threadIdx.x; i < j; i += blockDim.x) x[i] -= A[j * N + i] * x[j];
      __syncthreads();
    }
    // ---- FD: d_fd = (T x .. x T) diag(dinv) (T x .. x T)^T r (dense tensor sums) ----
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
      const int i0 = i % m, i1 = (i / m) % m, i2 = dim == 3 ? i / (m * m) : 0;
      double acc = 0.0;
      for (int j = 0; j < N; ++j) {
        const int j0 = j % m, j1 = (j / m) % m, j2 = dim == 3 ? j / (m * m) : 0;
        double w = l_T[j0 * m + i0] * l_T[j1 * m + i1];
        if (dim == 3) w *= l_T[j2 * m + i2];
        acc += w * r[j];
      }
      t[i] = acc * dinv[i];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
      const int i0 = i % m, i1 = (i / m) % m, i2 = dim == 3 ? i / (m * m) : 0;
      double acc = 0.0;
      for (int j = 0; j < N; ++j) {
        const int j0 = j % m, j1 = (j / m) % m, j2 = dim == 3 ? j / (m * m) : 0;
        double w = l_T[i0 * m + j0] * l_T[i1 * m + j1];
        if (dim == 3) w *= l_T[i2 * m + j2];
        acc += w * t[j];
      }
      e1[i] = acc * theta;  // d_fd
    }
    __syncthreads();
    if (DEX)
      for (int i = threadIdx.x; i < N; i += blockDim.x) {
        DEX[(long long)smp * N + i] = x[i];
        DFD[(long long)smp * N + i] = e1[i];
      }
    if (corr) {
      // gate: energy-norm errors ||L^T (d - x)||^2 of FD and FD + correction
      float* Up = corr + (long long)smp * sh.no;
      const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
      for (int q = warp; q < sh.rank; q += blockDim.x / 32) {
        float acc = 0.f;
        for (int i = lane; i < N; i += 32) acc += Up[i * sh.rank + q] * (float)r[i];
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) s_tq[q] = acc * Up[N * sh.rank + q];
      }
      __syncthreads();
      for (int i = threadIdx.x; i < N; i += blockDim.x) {
        float c = 0.f;
        for (int q = 0; q < sh.rank; ++q) c += Up[i * sh.rank + q] * s_tq[q];
        e2[i] = e1[i] + (double)c - x[i];
        e1[i] = e1[i] - x[i];
      }
      if (threadIdx.x < 2) s_red[threadIdx.x] = 0.0;
      __syncthreads();
      double a1 = 0.0, a2 = 0.0;
      for (int i = threadIdx.x; i < N; i += blockDim.x) {  // (L^T e)_i = sum_{j>=i} L[j][i] e_j
        double v1 = 0.0, v2 = 0.0;
        for (int j = i; j < N; ++j) {
          v1 += A[j * N + i] * e1[j];
          v2 += A[j * N + i] * e2[j];
        }
        a1 += v1 * v1;
        a2 += v2 * v2;
      }
      atomicAdd(&s_red[0], a1);
      atomicAdd(&s_red[1], a2);
      __syncthreads();
      if (threadIdx.x == 0) {
        const bool keep = s_red[1] < s_red[0];
        if (!keep)
          for (int q = 0; q < sh.rank; ++q) Up[N * sh.rank + q] = 0.f;
        if (kept) kept[smp] = keep ? 1 : 0;
      }
    }
    __syncthreads();
  }
}

// ---- perceptron kernels (FP32) ----
// params: W1 [nh x nf] | b1 [nh] | W2 [no x nh] | b2 [no]
__global__ void mlp_forward_kernel(Shape sh, int n, const float* __restrict__ P, const float* __restrict__ X,
                                   float* __restrict__ H, float* __restrict__ O) {
  const float* W1 = P;
  const float* b1 = W1 + sh.nh * sh.nf;
  const float* W2 = b1 + sh.nh;
  const float* b2 = W2 + sh.no * sh.nh;
  __shared__ float hs[kHidden];
  for (int smp = blockIdx.x; smp < n; smp += gridDim.x) {
    if (threadIdx.x < sh.nh) {
      float acc = b1[threadIdx.x];
      for (int f = 0; f < sh.nf; ++f) acc += W1[threadIdx.x * sh.nf + f] * X[(long long)smp * sh.nf + f];
      const float h = tanhf(acc);
      hs[threadIdx.x] = h;
      if (H) H[(long long)smp * sh.nh + threadIdx.x] = h;
    }
    __syncthreads();
    for (int o = threadIdx.x; o < sh.no; o += blockDim.x) {
      float acc = b2[o];
      for (int h = 0; h < sh.nh; ++h) acc += W2[o * sh.nh + h] * hs[h];
      O[(long long)smp * sh.no + o] = acc;
    }
    __syncthreads();
  }
}

// d loss / d O for loss = mean_n ||DFD + U diag(s) U^T R - DEX||^2 / ||DEX||^2
__global__ void mlp_loss_grad_kernel(Shape sh, int n, const float* __restrict__ O, const double* __restrict__ R,
                                     const double* __restrict__ DFD, const double* __restrict__ DEX,
                                     float* __restrict__ dO, float* __restrict__ loss) {
  const int N = sh.nint, RK = sh.rank;
  extern __shared__ float fs[];
  float* e = fs;           // N
  float* g = e + N;        // N
  __shared__ float t[kRank], gu[kRank], red[2];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int smp = blockIdx.x; smp < n; smp += gridDim.x) {
    const float* U = O + (long long)smp * sh.no;
    const float* s = U + N * RK;
    const double* r = R + (long long)smp * N;
    for (int q = warp; q < RK; q += blockDim.x / 32) {
      float acc = 0.f;
      for (int i = lane; i < N; i += 32) acc += U[i * RK + q] * (float)r[i];
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) t[q] = acc;
    }
    if (threadIdx.x < 2) red[threadIdx.x] = 0.f;
    __syncthreads();
    float le = 0.f, ln = 0.f;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
      float c = 0.f;
      for (int q = 0; q < RK; ++q) c += U[i * RK + q] * s[q] * t[q];
      const float dex = (float)DEX[(long long)smp * N + i];
      const float ei = (float)DFD[(long long)smp * N + i] + c - dex;
      e[i] = ei;
      le += ei * ei;
      ln += dex * dex;
    }
    atomicAdd(&red[0], le);
    atomicAdd(&red[1], ln);
    __syncthreads();
    const float scale = 2.f / ((float)n * red[1]);
    for (int i = threadIdx.x; i < N; i += blockDim.x) g[i] = scale * e[i];
    __syncthreads();
    for (int q = warp; q < RK; q += blockDim.x / 32) {
      float acc = 0.f;
      for (int i = lane; i < N; i += 32) acc += U[i * RK + q] * g[i];
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) gu[q] = acc;
    }
    __syncthreads();
    float* d = dO + (long long)smp * sh.no;
    for (int idx = threadIdx.x; idx < N * RK; idx += blockDim.x) {
      const int i = idx / RK, q = idx % RK;
      d[idx] = g[i] * s[q] * t[q] + (float)r[i] * s[q] * gu[q];
    }
    if (threadIdx.x < RK) d[N * RK + threadIdx.x] = t[threadIdx.x] * gu[threadIdx.x];
    if (threadIdx.x == 0) loss[smp] = red[0] / (red[1] * (float)n);
    __syncthreads();
  }
}

// gradient of the two layers; one thread per parameter, sums over samples
__global__ void mlp_backward_w2_kernel(Shape sh, int n, const float* __restrict__ H, const float* __restrict__ dO,
                                       float* __restrict__ G) {
  float* gW2 = G + sh.nh * sh.nf + sh.nh;
  float* gb2 = gW2 + sh.no * sh.nh;
  const int tot = sh.no * sh.nh + sh.no;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < tot; idx += gridDim.x * blockDim.x) {
    float acc = 0.f;
    if (idx < sh.no * sh.nh) {
      const int o = idx / sh.nh, h = idx % sh.nh;
      for (int s = 0; s < n; ++s) acc += dO[(long long)s * sh.no + o] * H[(long long)s * sh.nh + h];
      gW2[idx] = acc;
    } else {
      const int o = idx - sh.no * sh.nh;
      for (int s = 0; s < n; ++s) acc += dO[(long long)s * sh.no + o];
      gb2[o] = acc;
    }
  }
}

__global__ void mlp_backward_dh_kernel(Shape sh, int n, const float* __restrict__ P, const float* __restrict__ H,
                                       const float* __restrict__ dO, float* __restrict__ dH) {
  const float* W2 = P + sh.nh * sh.nf + sh.nh;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < (long long)n * sh.nh;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long s = idx / sh.nh;
    const int h = (int)(idx % sh.nh);
    float acc = 0.f;
    for (int o = 0; o < sh.no; ++o) acc += dO[s * sh.no + o] * W2[o * sh.nh + h];
    const float hv = H[idx];
    dH[idx] = acc * (1.f - hv * hv);
  }
}

__global__ void mlp_backward_w1_kernel(Shape sh, int n, const float* __restrict__ X, const float* __restrict__ dH,
                                       float* __restrict__ G) {
  const int tot = sh.nh * sh.nf + sh.nh;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < tot; idx += gridDim.x * blockDim.x) {
    float acc = 0.f;
    if (idx < sh.nh * sh.nf) {
      const int h = idx / sh.nf, f = idx % sh.nf;
      for (int s = 0; s < n; ++s) acc += dH[(long long)s * sh.nh + h] * X[(long long)s * sh.nf + f];
    } else {
      const int h = idx - sh.nh * sh.nf;
      for (int s = 0; s < n; ++s) acc += dH[(long long)s * sh.nh + h];
    }
    G[idx] = acc;
  }
}

__global__ void adam_kernel(int np, float* __restrict__ P, const float* __restrict__ G, float* __restrict__ m1,
                            float* __restrict__ m2, float lr, float c1, float c2) {
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < np; i += gridDim.x * blockDim.x) {
    const float g = G[i];
    const float a = b1 * m1[i] + (1.f - b1) * g;
    const float b = b2 * m2[i] + (1.f - b2) * g * g;
    m1[i] = a;
    m2[i] = b;
    P[i] -= lr * (a / c1) / (sqrtf(b / c2) + eps);
  }
}

__global__ void round_half_kernel(int np, const float* __restrict__ P, float* __restrict__ Q) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < np; i += gridDim.x * blockDim.x)
    Q[i] = __half2float(__float2half_rn(P[i]));
}

int upload_learned_tables(int k) {
  if (k < 1 || k > kMaxK) return GMG_ERR_UNSUPPORTED;
  const int m = 2 * k - 1;
  std::vector<double> Mc, Kc, Mi, Ki, Tp, lp;
  cell_matrices_1d(k, Mc, Kc);
  assembled_1d(k, 2, 1, m, 1, m, Mi, Ki);
  if (!generalized_eigen_mirror(m, Mi, Ki, Tp, lp)) return GMG_ERR_INVALID_ARG;
  if (cudaMemcpyToSymbol(l_Mc, Mc.data(), Mc.size() * 8) != cudaSuccess ||
      cudaMemcpyToSymbol(l_Kc, Kc.data(), Kc.size() * 8) != cudaSuccess ||
      cudaMemcpyToSymbol(l_T, Tp.data(), Tp.size() * 8) != cudaSuccess)
    return GMG_ERR_CUDA;
  return GMG_OK;
}

std::vector<double> fd_diag(int dim, int k) {
  const int m = 2 * k - 1;
  std::vector<double> Mi, Ki, Tp, lp;
  assembled_1d(k, 2, 1, m, 1, m, Mi, Ki);
  generalized_eigen_mirror(m, Mi, Ki, Tp, lp);
  const int nint = dim == 3 ? m * m * m : m * m;
  std::vector<double> d(nint);
  for (int t = 0; t < nint; ++t)
    d[t] = 1.0 / (lp[t % m] + lp[(t / m) % m] + (dim == 3 ? lp[t / (m * m)] : 0.0));
  return d;
}

int exact_smem(const Shape& sh) { return (sh.nint * sh.nint + 6 * sh.nint) * 8; }

int launch_exact(const Shape& sh, int n, const double* W, const double* R, const double* dinv, double* DEX,
                 double* DFD, float* corr, int* kept, cudaStream_t s) {
  const int smem = exact_smem(sh);
  if (smem > 220 * 1024) return GMG_ERR_UNSUPPORTED;
  if (cudaFuncSetAttribute(exact_patch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
    return GMG_ERR_CUDA;
  exact_patch_kernel<<<std::min(n, 152 * 8), 256, smem, s>>>(sh, n, W, R, dinv, DEX, DFD, corr, kept);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? GMG_OK : GMG_ERR_CUDA;
}

// loss and gradient of one batch (device arrays); loss summed on the host
int batch_loss_grad(const Shape& sh, int n, const float* P, const float* X, const double* R, const double* DFD,
                    const double* DEX, float* H, float* O, float* dO, float* dH, float* lossv, float* G,
                    double* loss_host, cudaStream_t s) {
  const int grid = std::min(n, 152 * 16);
  mlp_forward_kernel<<<grid, 128, 0, s>>>(sh, n, P, X, H, O);
  mlp_loss_grad_kernel<<<grid, 128, 2 * sh.nint * sizeof(float), s>>>(sh, n, O, R, DFD, DEX, dO, lossv);
  mlp_backward_w2_kernel<<<(sh.no * sh.nh + sh.no + 255) / 256, 256, 0, s>>>(sh, n, H, dO, G);
  mlp_backward_dh_kernel<<<(int)std::min<long long>(((long long)n * sh.nh + 255) / 256, 152 * 16), 256, 0, s>>>(
      sh, n, P, H, dO, dH);
  mlp_backward_w1_kernel<<<(sh.nh * sh.nf + sh.nh + 255) / 256, 256, 0, s>>>(sh, n, X, dH, G);
  count_launch(5);
  if (cudaGetLastError() != cudaSuccess) return GMG_ERR_CUDA;
  if (loss_host) {
    std::vector<float> lv(n);
    if (cudaMemcpyAsync(lv.data(), lossv, n * sizeof(float), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return GMG_ERR_CUDA;
    double L = 0.0;
    for (float v : lv) L += v;
    *loss_host = L;
  }
  return GMG_OK;
}

struct DevBuf {
  std::vector<void*> ptrs;
  template <typename T>
  T* get(size_t count) {
    void* p = nullptr;
    if (cudaMalloc(&p, std::max<size_t>(count, 1) * sizeof(T)) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    cudaMemset(p, 0, std::max<size_t>(count, 1) * sizeof(T));
    ptrs.push_back(p);
    return static_cast<T*>(p);
  }
  ~DevBuf() {
    for (void* p : ptrs) cudaFree(p);
  }
};

// features (log w) and weights w of the 2^d cells of each vertex in `verts`
void patch_features(const std::vector<double>& coef, int dim, int n, const std::vector<int>& verts,
                    std::vector<float>& X, std::vector<double>& W) {
  const int nc = 1 << dim;
  X.assign(verts.size() * nc, 0.f);
  W.assign(verts.size() * nc, 0.0);
  for (size_t s = 0; s < verts.size(); ++s) {
    const int vid = verts[s];
    const int v0 = vid % (n - 1) + 1, v1 = (vid / (n - 1)) % (n - 1) + 1, v2 = dim == 3 ? vid / ((n - 1) * (n - 1)) + 1 : 1;
    double lg[8], mean = 0.0;
    for (int o = 0; o < nc; ++o) {
      const long long c = (long long)(v0 - 1 + (o & 1)) +
                          (long long)n * ((v1 - 1 + ((o >> 1) & 1)) + (dim == 3 ? (long long)n * (v2 - 1 + ((o >> 2) & 1)) : 0));
      lg[o] = std::log(coef[c]);
      mean += lg[o];
    }
    mean /= nc;
    for (int o = 0; o < nc; ++o) {
      X[s * nc + o] = (float)(lg[o] - mean);
      W[s * nc + o] = std::exp(lg[o] - mean);
    }
  }
}

// Level judge: plain FD is the fallback and the judge of the learned
// correction at the level of the whole solver.  With the corrections of no
// level in use, the FP64 CG (V-cycle preconditioner, the problem's own
// settings) solves a fixed probe right-hand side to the benchmark tolerance;
// then, level by level from the coarsest, a level's correction stays in use
// only if it lowers the iteration count below the best so far.  Levels that
// buy no iteration cost only time, so they fall back to damped FD.
int judge_levels(gmg_problem* p) {
  const int L = (int)p->levels.size();
  const Level& F = p->levels[L - 1];
  const LevelGeom& g = F.g;
  std::vector<double> probe((size_t)F.n_elems, 0.0);
  unsigned long long x = 0x9E3779B97F4A7C15ull;  // fixed xorshift sequence
  for (int i2 = (g.dim == 3 ? 1 : 0); i2 < (g.dim == 3 ? g.N - 1 : 1); ++i2)
    for (int i1 = 1; i1 < g.N - 1; ++i1)
      for (int i0 = 1; i0 < g.N - 1; ++i0) {
        x ^= x << 13;
        x ^= x >> 7;
        x ^= x << 17;
        probe[(size_t)(i0 + (long long)g.py * i1 + g.pz * i2)] = (double)(x >> 11) * 0x1.0p-52 - 1.0;
      }
  DevBuf buf;
  double* b = buf.get<double>(probe.size());
  double* u = buf.get<double>(probe.size());
  if (!b || !u) return GMG_ERR_OOM;
  if (cudaMemcpy(b, probe.data(), probe.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess) return GMG_ERR_CUDA;
  auto iterations = [&](unsigned mask, int* its) -> int {
    p->corr_levels = mask;
    drop_cg_graph(p);
    if (cudaMemsetAsync(u, 0, probe.size() * 8, p->stream) != cudaSuccess) return GMG_ERR_CUDA;
    gmg_solve_stats st;
    const int rc = cg_gmg_solve(p, u, b, 1e-10, 500, &st);
    if (rc == GMG_ERR_CUDA || rc == GMG_ERR_INVALID_ARG) return rc;
    *its = rc == GMG_OK ? st.iterations : 1 << 30;  // breakdown or no convergence: reject
    return GMG_OK;
  };
  int best = 0;
  CHECK(iterations(0u, &best));
  unsigned mask = 0u;
  for (int l = 0; l < L; ++l) {
    if (!p->corr[l]) continue;
    int its = 0;
    CHECK(iterations(mask | (1u << l), &its));
    if (its < best) {
      best = its;
      mask |= 1u << l;
    }
  }
  p->corr_levels = mask;
  drop_cg_graph(p);
  return cudaDeviceSynchronize() == cudaSuccess ? GMG_OK : GMG_ERR_CUDA;
}

}  // namespace

extern "C" {

int gmg_mlp_loss_grad(int dim, int degree, int rank, int hidden, int n, const float* params, const float* X,
                      const double* R, const double* DFD, const double* DEX, double* loss, float* grads) {
  if ((dim != 2 && dim != 3) || degree < 1 || degree > kMaxK || rank < 1 || rank > kRank || hidden < 1 ||
      hidden > kHidden || n < 1 || !params || !X || !R || !DFD || !DEX || !grads)
    return GMG_ERR_INVALID_ARG;
  const Shape sh = make_shape(dim, degree, rank, hidden);
  DevBuf buf;
  float* H = buf.get<float>((size_t)n * sh.nh);
  float* O = buf.get<float>((size_t)n * sh.no);
  float* dO = buf.get<float>((size_t)n * sh.no);
  float* dH = buf.get<float>((size_t)n * sh.nh);
  float* lv = buf.get<float>(n);
  if (!H || !O || !dO || !dH || !lv) return GMG_ERR_OOM;
  return batch_loss_grad(sh, n, params, X, R, DFD, DEX, H, O, dO, dH, lv, grads, loss, nullptr);
}

int gmg_learned_train(gmg_problem* p, int n_samples, const int* sample_vertices, const double* residuals,
                      int steps, int batch, double lr, unsigned seed, double* loss_history,
                      int* kept_patches) {
  if (!p || !p->varcoef || n_samples < 1 || !sample_vertices || !residuals || steps < 0 || batch < 1)
    return GMG_ERR_INVALID_ARG;
  drop_cg_graph(p);
  const int dim = p->desc.dim, k = p->desc.degree, L = (int)p->levels.size();
  const Shape sh = make_shape(dim, k, kRank, kHidden);
  if (exact_smem(sh) > 220 * 1024) return GMG_ERR_UNSUPPORTED;
  cudaStream_t s = p->stream;
  CHECK(upload_learned_tables(k));
  // level coefficients back on the host
  std::vector<std::vector<double>> lev(L);
  for (int l = 0; l < L; ++l) {
    const int n = p->levels[l].g.n;
    const long long nc = dim == 3 ? (long long)n * n * n : (long long)n * n;
    lev[l].resize(nc);
    if (p->esize == 8) {
      if (cudaMemcpy(lev[l].data(), p->coef[l], nc * 8, cudaMemcpyDeviceToHost) != cudaSuccess) return GMG_ERR_CUDA;
    } else {
      std::vector<float> f(nc);
      if (cudaMemcpy(f.data(), p->coef[l], nc * 4, cudaMemcpyDeviceToHost) != cudaSuccess) return GMG_ERR_CUDA;
      for (long long c = 0; c < nc; ++c) lev[l][c] = f[c];
    }
  }
  DevBuf buf;
  const std::vector<double> dinv_h = fd_diag(dim, k);
  double* dinv = buf.get<double>(sh.nint);
  if (!dinv || cudaMemcpy(dinv, dinv_h.data(), sh.nint * 8, cudaMemcpyHostToDevice) != cudaSuccess)
    return GMG_ERR_CUDA;
  // ---- training data: exact solves of the sample patches; sample ids run
  // over the patches of all levels, finest level first ----
  std::vector<long long> first(L + 1, 0);  // first id of level l; first[L] = total
  {
    long long acc = 0;
    for (int l = L - 1; l >= 0; --l) {
      const long long nl = p->levels[l].g.n - 1;
      first[l] = acc;
      acc += dim == 3 ? nl * nl * nl : nl * nl;
    }
    first[L] = acc;  // total
  }
  for (int i = 0; i < n_samples; ++i)
    if (sample_vertices[i] < 0 || sample_vertices[i] >= first[L]) return GMG_ERR_INVALID_ARG;
  std::vector<float> Xh((size_t)n_samples * sh.nf);
  std::vector<double> Wh((size_t)n_samples * sh.nf);
  for (int l = 0; l < L; ++l) {
    const long long lo = first[l];
    std::vector<int> idx, vl;
    const long long nl = p->levels[l].g.n - 1, cnt = dim == 3 ? nl * nl * nl : nl * nl;
    for (int i = 0; i < n_samples; ++i)
      if (sample_vertices[i] >= lo && sample_vertices[i] < lo + cnt) {
        idx.push_back(i);
        vl.push_back((int)(sample_vertices[i] - lo));
      }
    if (idx.empty()) continue;
    std::vector<float> Xl;
    std::vector<double> Wl;
    patch_features(lev[l], dim, p->levels[l].g.n, vl, Xl, Wl);
    for (size_t j = 0; j < idx.size(); ++j)
      for (int c = 0; c < sh.nf; ++c) {
        Xh[(size_t)idx[j] * sh.nf + c] = Xl[j * sh.nf + c];
        Wh[(size_t)idx[j] * sh.nf + c] = Wl[j * sh.nf + c];
      }
  }
  float* X = buf.get<float>(Xh.size());
  double* W = buf.get<double>(Wh.size());
  double* DEX = buf.get<double>((size_t)n_samples * sh.nint);
  double* DFD = buf.get<double>((size_t)n_samples * sh.nint);
  if (!X || !W || !DEX || !DFD) return GMG_ERR_OOM;
  if (cudaMemcpy(X, Xh.data(), Xh.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(W, Wh.data(), Wh.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess)
    return GMG_ERR_CUDA;
  CHECK(launch_exact(sh, n_samples, W, residuals, dinv, DEX, DFD, nullptr, nullptr, s));
  // ---- parameters: W1 ~ U(+-1/sqrt(nf)), b1 = 0, W2 small, b2: U = the
  // lowest FD modes, s = 0 (a zero correction, away from the U = 0 saddle) ----
  const int np = sh.np();
  std::vector<float> P0(np, 0.f);
  std::mt19937 rng(seed);
  std::uniform_real_distribution<float> uni(-1.f, 1.f);
  const float a1 = 1.f / std::sqrt((float)sh.nf);
  for (int i = 0; i < sh.nh * sh.nf; ++i) P0[i] = a1 * uni(rng);
  float* W2h = P0.data() + sh.nh * sh.nf + sh.nh;
  for (int i = 0; i < sh.no * sh.nh; ++i) W2h[i] = 1e-3f * uni(rng);
  float* b2h = W2h + sh.no * sh.nh;
  {
    const int m = sh.m;
    std::vector<double> Mi, Ki, Tp, lp;
    assembled_1d(k, 2, 1, m, 1, m, Mi, Ki);
    generalized_eigen_mirror(m, Mi, Ki, Tp, lp);
    std::vector<std::pair<double, int>> modes;
    for (int t = 0; t < sh.nint; ++t) modes.push_back({1.0 / dinv_h[t], t});
    std::sort(modes.begin(), modes.end());
    for (int q = 0; q < sh.rank; ++q) {
      const int t = modes[q].second;
      const int t0 = t % m, t1 = (t / m) % m, t2 = dim == 3 ? t / (m * m) : 0;
      for (int i = 0; i < sh.nint; ++i) {
        const int i0 = i % m, i1 = (i / m) % m, i2 = dim == 3 ? i / (m * m) : 0;
        double v = Tp[i0 * m + t0] * Tp[i1 * m + t1];
        if (dim == 3) v *= Tp[i2 * m + t2];
        b2h[i * sh.rank + q] = (float)v;
      }
    }
  }
  float* P = buf.get<float>(np);
  float* G = buf.get<float>(np);
  float* m1 = buf.get<float>(np);
  float* m2 = buf.get<float>(np);
  const int B = std::min(batch, n_samples);
  float* H = buf.get<float>((size_t)B * sh.nh);
  float* O = buf.get<float>((size_t)B * sh.no);
  float* dO = buf.get<float>((size_t)B * sh.no);
  float* dH = buf.get<float>((size_t)B * sh.nh);
  float* lv = buf.get<float>(B);
  if (!P || !G || !m1 || !m2 || !H || !O || !dO || !dH || !lv) return GMG_ERR_OOM;
  if (cudaMemcpy(P, P0.data(), np * 4, cudaMemcpyHostToDevice) != cudaSuccess) return GMG_ERR_CUDA;
  // ---- Adam over consecutive minibatches of the (caller-shuffled) samples ----
  for (int it = 0; it < steps; ++it) {
    const int start = (int)(((long long)it * B) % n_samples);
    const int nb = std::min(B, n_samples - start);
    double L_it = 0.0;
    CHECK(batch_loss_grad(sh, nb, P, X + (size_t)start * sh.nf, residuals + (size_t)start * sh.nint,
                          DFD + (size_t)start * sh.nint, DEX + (size_t)start * sh.nint, H, O, dO, dH, lv, G,
                          loss_history ? &L_it : nullptr, s));
    if (loss_history) loss_history[it] = L_it;
    const float c1 = 1.f - std::pow(0.9f, (float)(it + 1)), c2 = 1.f - std::pow(0.999f, (float)(it + 1));
    adam_kernel<<<(np + 255) / 256, 256, 0, s>>>(np, P, G, m1, m2, (float)lr, c1, c2);
    count_launch();
  }
  // ---- inference with FP16-rounded weights, then the per-patch gate ----
  float* Ph = buf.get<float>(np);
  if (!Ph) return GMG_ERR_OOM;
  round_half_kernel<<<(np + 255) / 256, 256, 0, s>>>(np, P, Ph);
  count_launch();
  p->corr_rank = sh.rank;
  p->corr.assign(L, nullptr);
  int kept_total = 0;
  for (int l = 0; l < L; ++l) {
    const int n = p->levels[l].g.n;
    const int npatch = dim == 3 ? (n - 1) * (n - 1) * (n - 1) : (n - 1) * (n - 1);
    if (npatch <= 0) continue;
    std::vector<int> all(npatch);
    for (int i = 0; i < npatch; ++i) all[i] = i;
    std::vector<float> Xl;
    std::vector<double> Wl;
    patch_features(lev[l], dim, n, all, Xl, Wl);
    DevBuf lb;
    float* Xd = lb.get<float>(Xl.size());
    double* Wd = lb.get<double>(Wl.size());
    double* Rp = lb.get<double>((size_t)npatch * sh.nint);
    int* kept = lb.get<int>(npatch);
    void* cd = nullptr;
    CHECK(dalloc(p, &cd, (size_t)npatch * sh.no * sizeof(float)));
    float* corr = static_cast<float*>(cd);
    if (!Xd || !Wd || !Rp || !kept) return GMG_ERR_OOM;
    std::vector<double> probe((size_t)npatch * sh.nint);
    for (size_t i = 0; i < probe.size(); ++i) probe[i] = std::sin(0.7 * (double)(i % sh.nint) + 1.3 * (double)(i / sh.nint) + 0.1);
    if (cudaMemcpy(Xd, Xl.data(), Xl.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(Wd, Wl.data(), Wl.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(Rp, probe.data(), probe.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess)
      return GMG_ERR_CUDA;
    mlp_forward_kernel<<<std::min(npatch, 152 * 16), 128, 0, s>>>(sh, npatch, Ph, Xd, nullptr, corr);
    count_launch();
    CHECK(launch_exact(sh, npatch, Wd, Rp, dinv, nullptr, nullptr, corr, kept, s));
    std::vector<int> kh(npatch);
    if (cudaMemcpy(kh.data(), kept, npatch * 4, cudaMemcpyDeviceToHost) != cudaSuccess) return GMG_ERR_CUDA;
    for (int v : kh) kept_total += v;
    p->corr[l] = corr;
  }
  if (kept_patches) *kept_patches = kept_total;
  p->local_solver = GMG_LOCAL_LEARNED;
  if (cudaDeviceSynchronize() != cudaSuccess) return GMG_ERR_CUDA;
  return judge_levels(p);
}

int gmg_learned_levels(const gmg_problem* p) {
  if (!p || !p->varcoef) return GMG_ERR_INVALID_ARG;
  return (int)p->corr_levels;
}

int gmg_learned_set_levels(gmg_problem* p, int mask) {
  if (!p || !p->varcoef || mask < 0) return GMG_ERR_INVALID_ARG;
  const int L = (int)p->levels.size();
  if (L < 31 && (mask >> L) != 0) return GMG_ERR_INVALID_ARG;
  for (int l = 0; l < L; ++l)
    if (((mask >> l) & 1) && ((int)p->corr.size() <= l || !p->corr[l])) return GMG_ERR_INVALID_ARG;
  drop_cg_graph(p);
  p->corr_levels = (unsigned)mask;
  return GMG_OK;
}

int gmg_exact_patch_solve(int dim, int degree, int n, const double* w, const double* r, double* d_exact,
                          double* d_fd) {
  if ((dim != 2 && dim != 3) || degree < 1 || degree > kMaxK || n < 0 || (n > 0 && (!w || !r || !d_exact || !d_fd)))
    return GMG_ERR_INVALID_ARG;
  if (n == 0) return GMG_OK;
  const Shape sh = make_shape(dim, degree, kRank, kHidden);
  if (exact_smem(sh) > 220 * 1024) return GMG_ERR_UNSUPPORTED;
  CHECK(upload_learned_tables(degree));
  DevBuf buf;
  const std::vector<double> dinv_h = fd_diag(dim, degree);
  double* dinv = buf.get<double>(sh.nint);
  if (!dinv) return GMG_ERR_OOM;
  if (cudaMemcpy(dinv, dinv_h.data(), sh.nint * 8, cudaMemcpyHostToDevice) != cudaSuccess) return GMG_ERR_CUDA;
  CHECK(launch_exact(sh, n, w, r, dinv, d_exact, d_fd, nullptr, nullptr, nullptr));
  return cudaDeviceSynchronize() == cudaSuccess ? GMG_OK : GMG_ERR_CUDA;
}

int gmg_learned_corrections(const gmg_problem* p, int level, float* out, long long count) {
  if (!p || level < 0 || level >= (int)p->levels.size() || !out) return GMG_ERR_INVALID_ARG;
  if ((int)p->corr.size() <= level || !p->corr[level]) return GMG_ERR_INVALID_ARG;
  const int n = p->levels[level].g.n, dim = p->desc.dim;
  const long long npatch = dim == 3 ? (long long)(n - 1) * (n - 1) * (n - 1) : (long long)(n - 1) * (n - 1);
  const Shape sh = make_shape(dim, p->desc.degree, p->corr_rank, kHidden);
  if (count < npatch * sh.no) return GMG_ERR_INVALID_ARG;
  return cudaMemcpy(out, p->corr[level], npatch * sh.no * sizeof(float), cudaMemcpyDeviceToHost) == cudaSuccess
             ? GMG_OK : GMG_ERR_CUDA;
}

}  // extern "C"

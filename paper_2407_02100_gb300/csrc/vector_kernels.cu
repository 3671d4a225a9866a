// Grid transfer (tensor-product 1D contractions along one axis), diagonal
// scaling, precision conversion and the FP64 vector kernels of the outer CG.
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/gmg.h"
#include "kernels.h"

namespace gmg {

namespace {

constexpr int kThreads = 256;

inline int grid_for(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  return (int)std::max<long long>(1, std::min<long long>(b, 152LL * 16));
}

// out[o + out_off] (+)= sum_w coef[(o_ax % R) W + w] in[(o_ax / R) S + off + w]
// with one thread per output element: the (x, y) plane is flattened over
// the threads (x fastest, so loads and stores along the contiguous axis
// coalesce and no block runs mostly idle), z planes over grid.y
// (grid-strided beyond its limit), the contracted axis AX a template
// parameter.
template <typename T, int AX>
__global__ void axis_op_kernel(const T* __restrict__ in, T* __restrict__ out,
                               const T* __restrict__ coef, AxisOp op) {
  // one thread per output of a (x, y) plane, planes z strided over grid.y
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)op.cnt[0] * op.cnt[1]) return;
  const int o0 = (int)(t % op.cnt[0]), o1 = (int)(t / op.cnt[0]);
  const long long sa = op.in_stride[AX];
  const int lim = op.in_dim[AX];
  for (int o2 = blockIdx.y; o2 < op.cnt[2]; o2 += gridDim.y) {
    {
      const int o[3] = {o0, o1, o2};
      long long ibase = 0, obase = 0;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        obase += (long long)(o[a] + op.out_off[a]) * op.out_stride[a];
        if (a != AX) ibase += (long long)(o[a] + op.in_off[a]) * op.in_stride[a];
      }
      const int oa = o[AX] + op.shift;
      const int start = (oa / op.R) * op.S + op.off;
      const T* __restrict__ c = coef + (oa % op.R) * op.W;
      T acc = T(0);
      for (int w = 0; w < op.W; ++w) {
        const int i = start + w;
        if (i >= 0 && i < lim) acc += __ldg(c + w) * in[ibase + i * sa];
      }
      if (op.accumulate) out[obase] += acc;
      else out[obase] = acc;
    }
  }
}

template <typename T>
__global__ void scale_kernel(long long n, T* __restrict__ x, const T* __restrict__ d) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    x[i] *= d[i];
}

__global__ void f64_to_f32_kernel(long long n, const double* __restrict__ x, float* __restrict__ y) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = (float)x[i];
}

__global__ void f32_to_f64_kernel(long long n, const float* __restrict__ x, double* __restrict__ y) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = (double)x[i];
}

// block-level sum (kThreads threads) of one value per thread
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double warp_part[kThreads / 32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) warp_part[wid] = v;
  __syncthreads();
  v = (threadIdx.x < kThreads / 32) ? warp_part[threadIdx.x] : 0.0;
  if (wid == 0)
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  return v;  // valid in thread 0
}

__global__ void dot_partial_kernel(long long n, const double* __restrict__ x,
                                   const double* __restrict__ y, double* __restrict__ partial) {
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    s += x[i] * y[i];
  s = block_sum(s);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// single block: result = sum of `count` partials (fixed order: deterministic)
__global__ void final_sum_kernel(int count, const double* __restrict__ partial, double* __restrict__ result) {
  double s = 0.0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) s += partial[i];
  s = block_sum(s);
  if (threadIdx.x == 0) *result = s;
}

__global__ void cg_update_kernel(long long n, double* __restrict__ x, double* __restrict__ r,
                                 const double* __restrict__ p, const double* __restrict__ q,
                                 const double* __restrict__ num, const double* __restrict__ den,
                                 double* __restrict__ partial) {
  const double alpha = *num / *den;
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    x[i] += alpha * p[i];
    double ri = r[i] - alpha * q[i];
    r[i] = ri;
    s += ri * ri;
  }
  s = block_sum(s);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void cg_direction_kernel(long long n, double* __restrict__ p, const double* __restrict__ z,
                                    const double* __restrict__ num, const double* __restrict__ den) {
  const double beta = *num / *den;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    p[i] = z[i] + beta * p[i];
}

// one warp per row of the dense inverse
template <typename T>
__global__ void dense_solve_kernel(LevelGeom g, const double* __restrict__ Ainv, int n_int,
                                   const T* __restrict__ b, T* __restrict__ x) {
  const int m = g.N - 2;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= n_int) return;
  auto node = [&](int i) -> long long {
    const int ix = i % m + 1, iy = (i / m) % m + 1, iz = g.dim == 3 ? i / (m * m) + 1 : 0;
    return ix + (long long)g.py * iy + (g.dim == 3 ? g.pz * iz : 0);
  };
  double acc = 0.0;
  for (int j = lane; j < n_int; j += 32) acc += Ainv[(long long)warp * n_int + j] * (double)b[node(j)];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) x[node(warp)] = (T)acc;
}

constexpr int kSegThreads = 256;

__global__ void seg_dot_kernel(Segments sg, const double* __restrict__ x, const double* __restrict__ y,
                               double* __restrict__ partial) {
  const int c = blockIdx.x;
  const long long s0 = sg.start[c];
  const int n = sg.len[c];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += kSegThreads) acc += x[s0 + i] * y[s0 + i];
  acc = block_sum(acc);
  if (threadIdx.x == 0) partial[c] = acc;
}

__global__ void seg_final_kernel(Segments sg, const double* __restrict__ partial, double* __restrict__ result) {
  const int i = blockIdx.x;
  double acc = 0.0;
  for (int c = sg.begin[i] + threadIdx.x; c < sg.begin[i + 1]; c += kSegThreads) acc += partial[c];
  acc = block_sum(acc);
  if (threadIdx.x == 0) result[i] = acc;
}

__global__ void seg_update_kernel(Segments sg, double* __restrict__ x, double* __restrict__ r,
                                  const double* __restrict__ p, const double* __restrict__ q,
                                  const double* __restrict__ num, const double* __restrict__ den,
                                  const int* __restrict__ active, double* __restrict__ partial) {
  const int c = blockIdx.x;
  const int owner = sg.owner[c];
  const long long s0 = sg.start[c];
  const int n = sg.len[c];
  const bool on = active[owner] != 0;
  const double alpha = on ? num[owner] / den[owner] : 0.0;
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += kSegThreads) {
    double ri = r[s0 + i];
    if (on) {
      x[s0 + i] += alpha * p[s0 + i];
      ri -= alpha * q[s0 + i];
      r[s0 + i] = ri;
    }
    acc += ri * ri;
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) partial[c] = acc;
}

__global__ void seg_direction_kernel(Segments sg, double* __restrict__ p, const double* __restrict__ z,
                                     const double* __restrict__ num, const double* __restrict__ den,
                                     const int* __restrict__ active) {
  const int c = blockIdx.x;
  const int owner = sg.owner[c];
  if (!active[owner]) return;
  const long long s0 = sg.start[c];
  const int n = sg.len[c];
  const double beta = num[owner] / den[owner];
  for (int i = threadIdx.x; i < n; i += kSegThreads) p[s0 + i] = z[s0 + i] + beta * p[s0 + i];
}

inline int status(int launches = 1) {
  count_launch(launches);
  return cudaGetLastError() == cudaSuccess ? GMG_OK : GMG_ERR_CUDA;
}

}  // namespace

template <typename T>
int launch_axis_op(const AxisOp& op, const T* in, T* out, const T* coef, cudaStream_t s) {
  if ((long long)op.cnt[0] * op.cnt[1] * op.cnt[2] <= 0) return GMG_OK;
  const int tx = 256;
  const long long plane = (long long)op.cnt[0] * op.cnt[1];
  if ((plane + tx - 1) / tx > 0x7FFFFFFFLL) return GMG_ERR_UNSUPPORTED;
  const dim3 grid((unsigned)((plane + tx - 1) / tx), std::min(op.cnt[2], 65535));
  switch (op.axis) {
    case 0: axis_op_kernel<T, 0><<<grid, tx, 0, s>>>(in, out, coef, op); break;
    case 1: axis_op_kernel<T, 1><<<grid, tx, 0, s>>>(in, out, coef, op); break;
    default: axis_op_kernel<T, 2><<<grid, tx, 0, s>>>(in, out, coef, op); break;
  }
  return status();
}
template int launch_axis_op<double>(const AxisOp&, const double*, double*, const double*, cudaStream_t);
template int launch_axis_op<float>(const AxisOp&, const float*, float*, const float*, cudaStream_t);

template <typename T>
int launch_dense_solve(const LevelGeom& g, const double* Ainv, int n_int, const T* b, T* x,
                       cudaStream_t s) {
  if (n_int <= 0) return GMG_OK;
  const int threads = 256, blocks = (n_int * 32 + threads - 1) / threads;
  dense_solve_kernel<T><<<blocks, threads, 0, s>>>(g, Ainv, n_int, b, x);
  return status();
}
template int launch_dense_solve<double>(const LevelGeom&, const double*, int, const double*, double*, cudaStream_t);
template int launch_dense_solve<float>(const LevelGeom&, const double*, int, const float*, float*, cudaStream_t);

template <typename T>
int launch_scale(long long n, T* x, const T* d, cudaStream_t s) {
  if (n <= 0) return GMG_OK;
  scale_kernel<T><<<grid_for(n, kThreads), kThreads, 0, s>>>(n, x, d);
  return status();
}
template int launch_scale<double>(long long, double*, const double*, cudaStream_t);
template int launch_scale<float>(long long, float*, const float*, cudaStream_t);

int launch_convert_f64_f32(long long n, const double* x, float* y, cudaStream_t s) {
  f64_to_f32_kernel<<<grid_for(n, kThreads), kThreads, 0, s>>>(n, x, y);
  return status();
}
int launch_convert_f32_f64(long long n, const float* x, double* y, cudaStream_t s) {
  f32_to_f64_kernel<<<grid_for(n, kThreads), kThreads, 0, s>>>(n, x, y);
  return status();
}

int launch_dot(long long n, const double* x, const double* y, double* partial, double* result,
               cudaStream_t s) {
  int g = std::min(grid_for(n, kThreads), kReduceBlocks);
  dot_partial_kernel<<<g, kThreads, 0, s>>>(n, x, y, partial);
  final_sum_kernel<<<1, kThreads, 0, s>>>(g, partial, result);
  return status(2);
}

int launch_cg_update(long long n, double* x, double* r, const double* p, const double* q,
                     const double* num, const double* den, double* partial, double* result,
                     cudaStream_t s) {
  int g = std::min(grid_for(n, kThreads), kReduceBlocks);
  cg_update_kernel<<<g, kThreads, 0, s>>>(n, x, r, p, q, num, den, partial);
  final_sum_kernel<<<1, kThreads, 0, s>>>(g, partial, result);
  return status(2);
}

int launch_seg_dot(const Segments& sg, const double* x, const double* y, double* partial,
                   double* result, cudaStream_t s) {
  if (sg.n_chunks <= 0) return GMG_OK;
  seg_dot_kernel<<<sg.n_chunks, kSegThreads, 0, s>>>(sg, x, y, partial);
  seg_final_kernel<<<sg.n_problems, kSegThreads, 0, s>>>(sg, partial, result);
  return status(2);
}

int launch_seg_cg_update(const Segments& sg, double* x, double* r, const double* p, const double* q,
                         const double* num, const double* den, const int* active, double* partial,
                         double* result, cudaStream_t s) {
  if (sg.n_chunks <= 0) return GMG_OK;
  seg_update_kernel<<<sg.n_chunks, kSegThreads, 0, s>>>(sg, x, r, p, q, num, den, active, partial);
  seg_final_kernel<<<sg.n_problems, kSegThreads, 0, s>>>(sg, partial, result);
  return status(2);
}

int launch_seg_cg_direction(const Segments& sg, double* p, const double* z, const double* num,
                            const double* den, const int* active, cudaStream_t s) {
  if (sg.n_chunks <= 0) return GMG_OK;
  seg_direction_kernel<<<sg.n_chunks, kSegThreads, 0, s>>>(sg, p, z, num, den, active);
  return status();
}

int launch_cg_direction(long long n, double* p, const double* z, const double* num,
                        const double* den, cudaStream_t s) {
  cg_direction_kernel<<<grid_for(n, kThreads), kThreads, 0, s>>>(n, p, z, num, den);
  return status();
}

}  // namespace gmg

// Level transfers of FP64 problems in double-float arithmetic.
//
// Prolongation is the embedding of the coarse Q_k space into the fine one,
// applied as a tensor product of the 1D cell interpolation (one axis per
// pass); restriction is its transpose (Sec. 2, the V-cycle's transfer
// operators).  In FP64 arithmetic each pass is bound by GB300's FP64 pipe
// (88-94 % busy at 5-20 % of the DRAM bandwidth), so FP64 problems run the
// passes in double-float arithmetic on the FP32 pipe (df_arith.cuh): node
// values are split once per load, the intermediate arrays between passes
// hold float pairs, and only the last pass writes doubles.
//
// Work per thread: all outputs of one coarse cell along the pass axis, which
// share one input window kept in registers.
//   prolongation: coarse cell j gives fine nodes 2k j + r (r = 0..2k-1) from
//     coarse nodes k j .. k j + k; an extra group j = n_c gives the last fine
//     node (the coarse vertex k n_c).
//   restriction: coarse cell j gives coarse nodes c = k j + r (r = 0..k-1,
//     c = 0 excluded: a Dirichlet node) from the fine window
//     2k j - (2k-1) .. 2k j + 2k - 1.  The vertex row (r = 0) spans the whole
//     window; a cell-interior node's coarse basis function lives in cell j
//     only and vanishes at its vertices, so its row has non-zeros only at
//     fine nodes 2k j + 1 .. 2k j + 2k - 1 (window taps 2k .. 4k-2).  The
//     host checks that structure in the table before launching.
// The other two axes are batch axes with the same index ranges, offsets and
// strides as the FP64 pass (AxisOp).
#include <cuda_runtime.h>

#include <type_traits>

#include "../../include/gmg.h"
#include "df_arith.cuh"
#include "kernels.h"

namespace gmg {

namespace {

constexpr int kXferMaxTaps = 8 * (4 * 8 - 1);  // k (4k - 1) at k = 8; 2k (k + 1) is smaller

struct XferArgs {
  AxisOp op;
  int n_cells;  // coarse cells along the pass axis
  float2 c[kXferMaxTaps];  // coefficient table as float pairs (hi, lo), rows of W
};

template <typename TI>
__device__ __forceinline__ dfv load_df(const TI* p) {
  if constexpr (sizeof(TI) == 8 && !std::is_same<TI, float2>::value) return df_from_double(__ldg(p));
  else {
    const float2 v = __ldg(p);
    return {v.x, v.y};
  }
}

template <typename TO, bool ACC>
__device__ __forceinline__ void store_df(TO* p, dfv v) {
  if constexpr (std::is_same<TO, float2>::value) {
    *p = make_float2(v.hi, v.lo);
  } else {
    if constexpr (ACC) v = df_add(df_from_double(*p), v);
    *p = df_to_double(v);
  }
}

template <int K, int AX, bool RESTRICT, typename TI, typename TO, bool ACC>
__global__ void __launch_bounds__(256) transfer_df_kernel(const TI* __restrict__ in, TO* __restrict__ out,
                                                          const __grid_constant__ XferArgs a) {
  constexpr int W = RESTRICT ? 4 * K - 1 : K + 1;  // window (= table row length)
  const AxisOp& op = a.op;
  const int ng = RESTRICT ? a.n_cells : a.n_cells + 1;  // groups along AX
  // lanes along x when the pass contracts y or z (coalesced batch loads),
  // along the groups when it contracts x
  constexpr int LA = AX == 0 ? 1 : 0;           // batch axis next to the groups
  constexpr int LB = AX == 2 ? 1 : 2;           // the other batch axis
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nla = op.cnt[LA], nlb = op.cnt[LB];
  if (t >= (long long)ng * nla * nlb) return;
  int j, oa, ob;
  if (AX == 0) {
    j = (int)(t % ng);
    const long long r = t / ng;
    oa = (int)(r % nla);
    ob = (int)(r / nla);
  } else {
    oa = (int)(t % nla);
    const long long r = t / nla;
    j = (int)(r % ng);
    ob = (int)(r / ng);
  }
  const long long ibase = (long long)(oa + op.in_off[LA]) * op.in_stride[LA] +
                          (long long)(ob + op.in_off[LB]) * op.in_stride[LB];
  const long long obase = (long long)(oa + op.out_off[LA]) * op.out_stride[LA] +
                          (long long)(ob + op.out_off[LB]) * op.out_stride[LB];
  const long long sa = op.in_stride[AX], so = op.out_stride[AX];
  const int lim = op.in_dim[AX];
  dfv x[W];
  if constexpr (RESTRICT) {
    const int start = 2 * K * j - (2 * K - 1);
#pragma unroll
    for (int w = 0; w < W; ++w) {
      const int i = start + w;
      x[w] = (i >= 0 && i < lim) ? load_df(in + ibase + (long long)i * sa) : dfv{0.f, 0.f};
    }
    // coarse node c = K j + r sits at output index c - 1 + out_off = c along AX
    if (j > 0) {
      df_acc acc = {0.f, 0.f};
#pragma unroll
      for (int w = 0; w < W; ++w) df_acc_add(acc, a.c[w].x, a.c[w].y, x[w]);
      store_df<TO, ACC>(out + obase + (long long)(K * j) * so, df_acc_value(acc));
    }
#pragma unroll
    for (int r = 1; r < K; ++r) {
      df_acc acc = {0.f, 0.f};
#pragma unroll
      for (int w = 2 * K; w < W; ++w) df_acc_add(acc, a.c[r * W + w].x, a.c[r * W + w].y, x[w]);
      store_df<TO, ACC>(out + obase + (long long)(K * j + r) * so, df_acc_value(acc));
    }
  } else {
    const int start = K * j;
#pragma unroll
    for (int q = 0; q < W; ++q) {
      const int i = start + q;
      x[q] = i < lim ? load_df(in + ibase + (long long)i * sa) : dfv{0.f, 0.f};
    }
    const int nr = j < a.n_cells ? 2 * K : 1;  // the extra group: the last fine node only
#pragma unroll
    for (int r = 0; r < 2 * K; ++r) {
      if (r < nr) {
        df_acc acc = {0.f, 0.f};
#pragma unroll
        for (int q = 0; q < W; ++q) df_acc_add(acc, a.c[r * W + q].x, a.c[r * W + q].y, x[q]);
        store_df<TO, ACC>(out + obase + (long long)(2 * K * j + r) * so, df_acc_value(acc));
      }
    }
  }
}

template <int K, int AX, bool RESTRICT, typename TI, typename TO, bool ACC>
int launch_one(const XferArgs& a, const void* in, void* out, cudaStream_t s) {
  const int ng = RESTRICT ? a.n_cells : a.n_cells + 1;
  const long long n = (long long)ng * a.op.cnt[AX == 0 ? 1 : 0] * a.op.cnt[AX == 2 ? 1 : 2];
  if (n <= 0) return GMG_OK;
  const long long blocks = (n + 255) / 256;
  if (blocks > 0x7FFFFFFFLL) return GMG_ERR_UNSUPPORTED;
  transfer_df_kernel<K, AX, RESTRICT, TI, TO, ACC>
      <<<(unsigned)blocks, 256, 0, s>>>(static_cast<const TI*>(in), static_cast<TO*>(out), a);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? GMG_OK : GMG_ERR_CUDA;
}

// The passes run x, y (, z): the first reads doubles and writes float pairs,
// a middle one (3D) float pairs to float pairs, the last float pairs to
// doubles (added to the fine vector by the prolongation).
template <int K, bool RESTRICT>
int launch_k(const XferArgs& a, const void* in, bool in_df, void* out, bool out_df, cudaStream_t s) {
  const bool acc = a.op.accumulate != 0;
  if (a.op.axis == 0 && !in_df && out_df && !acc)
    return launch_one<K, 0, RESTRICT, double, float2, false>(a, in, out, s);
  if (a.op.axis == 1 && in_df && out_df && !acc)
    return launch_one<K, 1, RESTRICT, float2, float2, false>(a, in, out, s);
  if ((a.op.axis == 1 || a.op.axis == 2) && in_df && !out_df && acc == !RESTRICT)
    return a.op.axis == 1 ? launch_one<K, 1, RESTRICT, float2, double, !RESTRICT>(a, in, out, s)
                          : launch_one<K, 2, RESTRICT, float2, double, !RESTRICT>(a, in, out, s);
  return GMG_ERR_UNSUPPORTED;
}

template <bool RESTRICT>
int launch_any(int k, const XferArgs& a, const void* in, bool in_df, void* out, bool out_df, cudaStream_t s) {
  switch (k) {
    case 1: return launch_k<1, RESTRICT>(a, in, in_df, out, out_df, s);
    case 2: return launch_k<2, RESTRICT>(a, in, in_df, out, out_df, s);
    case 3: return launch_k<3, RESTRICT>(a, in, in_df, out, out_df, s);
    case 4: return launch_k<4, RESTRICT>(a, in, in_df, out, out_df, s);
    case 5: return launch_k<5, RESTRICT>(a, in, in_df, out, out_df, s);
    case 6: return launch_k<6, RESTRICT>(a, in, in_df, out, out_df, s);
    case 7: return launch_k<7, RESTRICT>(a, in, in_df, out, out_df, s);
    case 8: return launch_k<8, RESTRICT>(a, in, in_df, out, out_df, s);
    default: return GMG_ERR_UNSUPPORTED;
  }
}

}  // namespace

int transfer_table_df_ok(int k, bool restrict_op, const double* table) {
  if (k < 1 || k > 8 || !table) return 0;
  if (!restrict_op) return 1;  // prolongation rows are used in full
  const int W = 4 * k - 1;
  for (int r = 1; r < k; ++r)
    for (int w = 0; w < 2 * k; ++w)
      if (table[r * W + w] != 0.0) return 0;
  return 1;
}

int launch_transfer_df(const AxisOp& op, int k, int n_cells, bool restrict_op, const double* table,
                       const void* in, bool in_df, void* out, bool out_df, cudaStream_t s) {
  if (k < 1 || k > 8 || n_cells < 1 || !table || !in || !out) return GMG_ERR_INVALID_ARG;
  const int W = restrict_op ? 4 * k - 1 : k + 1, rows = restrict_op ? k : 2 * k;
  if (rows * W > kXferMaxTaps) return GMG_ERR_UNSUPPORTED;
  // the pass must be the one the kernel assumes: window starts and lengths
  if (restrict_op ? (op.R != k || op.S != 2 * k || op.off != -(2 * k - 1) || op.W != W || op.shift != 1)
                  : (op.R != 2 * k || op.S != k || op.off != 0 || op.W != W || op.shift != 0))
    return GMG_ERR_INVALID_ARG;
  XferArgs a;
  a.op = op;
  a.n_cells = n_cells;
  for (int i = 0; i < rows * W; ++i) {
    const float hi = (float)table[i];
    a.c[i] = make_float2(hi, (float)(table[i] - (double)hi));
  }
  return restrict_op ? launch_any<true>(k, a, in, in_df, out, out_df, s)
                     : launch_any<false>(k, a, in, in_df, out, out_df, s);
}

}  // namespace gmg

// Patch sweep on the 5th-generation tensor cores (3D, FP32 data, degree
// 4..7): the same local_update as patch_colour_kernel (Sec. 3.1; gather,
// local residual by sum factorisation over the patch, fast-diagonalisation
// solve of App. A.3, scatter), with every 1D contraction executed as a TF32
// tcgen05.mma with FP32 accumulation in tensor memory.
//
// A contraction along one axis of a patch tensor is a GEMM whose rows are
// the lines of the tensor along that axis (the other two indices, enumerated
// compactly), whose K dimension is the contracted index (padded to 16) and
// whose N columns are the outputs of the 1D matrix (padded to 16; two
// matrices side by side give N = 32):
//     D[line][n] = sum_k X[line][k] B[n][k].
// Nine such GEMMs make one patch (3 for the residual, 6 for the solve):
//   Z : rows (x,y) in C^2,  K = z:  [P | Q]  = U [Mp ; Kp]^T
//   Y : rows (x,z') C*M,    K = y:  [A1 | A2] = P [Mp ; Kp]^T + Q [0 ; Mp]^T
//   X : rows (y',z') M^2,   K = x:  S = A1 Kp^T + A2 Mp^T,  r = h^{2-d} b - S
//   FX, FY, FZ : T^T along x, y, z (then times the FD diagonal)
//   BZ, BY, BX : T along z, y, x, then u += omega d
// (C = 2k+1 closure nodes, M = 2k-1 interior nodes per direction; Mp, Kp are
// the two-cell patch matrices, T the M-orthonormal FD eigenvectors.)  One CTA
// of 4 warps owns a patch: one thread issues the MMAs (M = 128 lines per
// tile, one or two tiles), the accumulator tiles come back with tcgen05.ld
// (warp w reads TMEM lanes 32w..32w+31, i.e. lines 32w.. of each tile) and
// every thread writes its lines' outputs, rounded to TF32, into the next
// stage's operand in shared memory: the axis permutation between stages is
// done by these writes.
//
// Operands use the canonical K-major layout without swizzle: 8-line x 16-byte
// core matrices, contiguous along K (LBO = 128 B), 8-line groups 512 B apart
// (SBO).  Padding columns are zero-initialised once and only ever hold finite
// values, and the padding rows of B are zero, so padding never reaches a
// result.  Every wait on the MMA-completion mbarrier is bounded; on expiry
// the kernel records GMG_ERR_TIMEOUT in a device flag (gmg_tc_status), frees
// its tensor memory and returns.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "../../include/gmg.h"
#include "async.cuh"
#include "kernels.h"

namespace gmg {
namespace tc {

using async::fence_proxy_async;
using async::kWaitLimit;
using async::mbar_init;
using async::mbar_wait;
using async::smem_u32;

constexpr int kKP = 16;                // padded contraction length (TF32: 2 MMA K-steps of 8)
constexpr int kRowB = kKP * 4;         // bytes per operand line
constexpr int kGroupB = 8 * kRowB;     // bytes per 8-line group: SBO
constexpr int kChunkB = 128;           // bytes per core matrix: LBO
constexpr int kTileB = 128 * kRowB;    // bytes per 128-line tile
constexpr int kBopsFloats = 2048;      // B operands of one degree (8 KB), TF32
constexpr int kBLo = kBopsFloats * 4;  // byte offset of the remainders' block
constexpr int kMinK = 4, kMaxK = 7;
// B operands (byte offsets inside the 8 KB block)
constexpr int kBZ = 0;       // [Mp ; Kp]  N = 32
constexpr int kBY2 = 2048;   // [0 ; Mp]   N = 32
constexpr int kBKP = 4096;   // Kp         N = 16
constexpr int kBMP = 5120;   // Mp         N = 16
constexpr int kBTT = 6144;   // T^T (rows = modes, K = nodes)   N = 16
constexpr int kBTN = 7168;   // T   (rows = nodes, K = modes)   N = 16

// per degree: the B operands rounded to TF32, then the TF32 roundings of the
// remainders (used by the split form)
__device__ float g_bops[kMaxK - kMinK + 1][2 * kBopsFloats];
__device__ int g_tc_error;

__host__ __device__ constexpr uint32_t op_off(int r, int k) {
  return (uint32_t)((r >> 3) * kGroupB + (k >> 2) * kChunkB + (r & 7) * 16 + (k & 3) * 4);
}

// instruction descriptor: D = F32, A = B = TF32, both K-major, M x N
__host__ __device__ constexpr uint32_t idesc_tf32(int m, int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

// shared-memory matrix descriptor, K-major, no swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(kChunkB >> 4) << 16) |
         ((uint64_t)(kGroupB >> 4) << 32) | (1ull << 46);
}

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                   smem_u32(mbar))
               : "memory");
}
__device__ __forceinline__ float tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// 16 / 32 consecutive accumulator columns of this thread's TMEM lane
// (32x32b shape: lane = thread of the warp), waited for before returning
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void st_op(unsigned char* base, int r, int k, float v) {
  *reinterpret_cast<float*>(base + op_off(r, k)) = tf32(v);
}
// store v as an operand: its TF32 rounding hi, and with LO != 0 also the
// TF32 rounding of the remainder v - hi in the twin buffer LO bytes further
// (hi + lo carries 22 significant bits: the products with the TF32 matrix
// entries then see the data to about FP32 accuracy)
template <int LO>
__device__ __forceinline__ void st_op2(unsigned char* base, int r, int k, float v) {
  const uint32_t o = op_off(r, k);
  const float hi = tf32(v);
  *reinterpret_cast<float*>(base + o) = hi;
  if (LO) *reinterpret_cast<float*>(base + LO + o) = tf32(v - hi);
}

// MMAs of one stage for `tiles` line tiles: D[t] (TMEM columns t*ncol..)
// = A[t] B1^T (+ A2[t] B2^T when a2 != 0), issued by one thread, then one
// commit to the mbarrier.  With lo != 0 (split form) each product is
// A_hi B_hi + A_lo B_hi + A_hi B_lo, the remainders A_lo lo bytes after
// their A and B_lo kBLo bytes after their B (3xTF32: FP32-level products).
__device__ __forceinline__ void stage_mma(uint32_t tmem, int tiles, int ncol, uint32_t idesc, uint32_t a1,
                                          uint32_t b1, uint32_t a2, uint32_t b2, uint64_t* mbar,
                                          uint32_t lo = 0) {
  fence_after();
  const uint32_t aoff[3] = {0u, lo, 0u}, boff[3] = {0u, 0u, (uint32_t)kBLo};
  const int parts = lo ? 3 : 1;
  for (int t = 0; t < tiles; ++t) {
    const uint32_t d = tmem + (uint32_t)(t * ncol);
    for (int h = 0; h < parts; ++h) {
      const uint32_t o = t * kTileB + aoff[h];
#pragma unroll
      for (int kk = 0; kk < 2; ++kk)
        mma_tf32(d, sdesc(a1 + o + kk * 2 * kChunkB), sdesc(b1 + boff[h] + kk * 2 * kChunkB), idesc,
                 (h > 0 || kk > 0) ? 1u : 0u);
      if (a2)
#pragma unroll
        for (int kk = 0; kk < 2; ++kk)
          mma_tf32(d, sdesc(a2 + o + kk * 2 * kChunkB), sdesc(b2 + boff[h] + kk * 2 * kChunkB), idesc, 1);
    }
  }
  mma_commit(mbar);
}

__device__ __forceinline__ void async_copy4(void* smem_dst, const float* gmem_src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_u32(smem_dst)), "l"(gmem_src) : "memory");
}

template <int K, bool SPLIT>
struct TcDims {
  static constexpr int C = 2 * K + 1, M = 2 * K - 1;
  static constexpr int RZ = C * C, RY = C * M, RX = M * M;  // lines per stage
  static constexpr int TZ = (RZ + 127) / 128, TY = (RY + 127) / 128, TX = (RX + 127) / 128;
  static constexpr int TCOLS = TZ * 32 <= 32 ? 32 : 64;  // TMEM columns (power of two)
  static constexpr int OPB = TZ * kTileB;                  // bytes per operand buffer
  static constexpr int NINT = M * M * M;
  // two operand buffers (and their remainder twins at +LO): the closure U
  // is dead once stage Z's MMAs are done, so P takes its buffer
  static constexpr int LO = SPLIT ? 2 * OPB : 0;
  static constexpr int OFF_U = 0, OFF_P = 0, OFF_Q = OPB, OFF_B = (SPLIT ? 4 : 2) * OPB;
  static constexpr int SMEM = OFF_B + (SPLIT ? 2 : 1) * kBopsFloats * 4;
  static_assert(C <= kKP, "closure must fit the padded contraction length");
  static_assert(TZ <= 2 && TY <= TZ && TX <= TZ, "at most two line tiles per stage");
};

template <int K, bool SPLIT>
__global__ void __launch_bounds__(128, K >= 6 ? 3 : 4) patch_tc_kernel(const __grid_constant__ PatchTable tab,
                                                       const float* __restrict__ dinv,
                                                       const float* __restrict__ bops, int* __restrict__ err) {
  using D = TcDims<K, SPLIT>;
  constexpr int LO = D::LO;
  constexpr int C = D::C, M = D::M;
  constexpr uint32_t I32 = idesc_tf32(128, 32), I16 = idesc_tf32(128, 16);
  extern __shared__ __align__(1024) unsigned char sm[];
  unsigned char* const OPU = sm + D::OFF_U;
  unsigned char* const OPP = sm + D::OFF_P;
  unsigned char* const OPQ = sm + D::OFF_Q;
  const uint32_t aU = smem_u32(OPU), aP = smem_u32(OPP), aQ = smem_u32(OPQ), aB = smem_u32(sm + D::OFF_B);
  __shared__ uint64_t s_mbar;
  __shared__ uint32_t s_tmem;
  __shared__ long long s_origin;
  __shared__ int s_entry;
  __shared__ volatile int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5;

  // zero the operand buffers once (padding stays finite), load B
  for (int i = tid; i < D::OFF_B / 4; i += 128) reinterpret_cast<float*>(sm)[i] = 0.f;
  for (int i = tid; i < (SPLIT ? 2 : 1) * kBopsFloats; i += 128)
    reinterpret_cast<float*>(sm + D::OFF_B)[i] = bops[i];
  if (warp == 0) tmem_alloc(&s_tmem, D::TCOLS);
  if (tid == 0) {
    mbar_init(&s_mbar, 1);
    s_fail = 0;
  }
  fence_proxy_async();
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = s_tmem;
  const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
  uint32_t parity = 0;
  bool ok = true, failed = false;
  const float om = (float)tab.omega;

  // wait for the stage's MMAs (bounded), then order the TMEM reads after them
  auto wait_mma = [&]() {
    if (!s_fail) {
      if (!mbar_wait(&s_mbar, parity)) {
        ok = false;
        s_fail = 1;
      }
    }
    parity ^= 1u;
    fence_after();
  };
  // publish this thread's operand writes and TMEM reads before the next MMA
  auto stage_sync = [&]() {
    fence_proxy_async();
    fence_before();
    __syncthreads();
  };

  for (int grp = blockIdx.x; grp < tab.total_groups; grp += gridDim.x) {
    if (tid == 0) {
      int lo = 0, hi = tab.n - 1;  // last entry with group_begin <= grp
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tab.e[mid].group_begin <= grp) lo = mid;
        else hi = mid - 1;
      }
      const PatchEntry& e = tab.e[lo];
      int pid = grp - e.group_begin;
      if (e.plist) pid = e.plist[pid];
      const int i0 = pid % e.count[0], rest = pid / e.count[0];
      const int i1 = rest % e.count[1], i2 = rest / e.count[1];
      s_origin = (long long)(e.first[0] + 2 * i0 - 1) * K + e.py * ((long long)(e.first[1] + 2 * i1 - 1) * K) +
                 e.pz * ((long long)(e.first[2] + 2 * i2 - 1) * K);
      s_entry = lo;
    }
    __syncthreads();
    const PatchEntry& e = tab.e[s_entry];
    const long long org = s_origin, py = e.py, pz = e.pz;
    const float* __restrict__ ug = static_cast<const float*>(e.u);
    const float* __restrict__ bg = static_cast<const float*>(e.b);
    float* __restrict__ uo = static_cast<float*>(e.u);
    const float sb = (float)e.sb;

    // ---- gather: closure of u into the Z operand (line x + C y, K = z);
    // b is read where the residual is formed ----
    for (int t = tid; t < C * C * C; t += 128) {
      const int x = t % C, y = (t / C) % C, z = t / (C * C);
      async_copy4(OPU + op_off(x + C * y, z), ug + org + x + py * y + pz * z);
    }
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
    if (SPLIT)  // split this thread's own copies into TF32 hi and remainder
      for (int t = tid; t < C * C * C; t += 128) {
        const int x = t % C, y = (t / C) % C, z = t / (C * C);
        const uint32_t o = op_off(x + C * y, z);
        const float v = *reinterpret_cast<const float*>(OPU + o);
        const float hi = tf32(v);
        *reinterpret_cast<float*>(OPU + o) = hi;
        *reinterpret_cast<float*>(OPU + LO + o) = tf32(v - hi);
      }
    stage_sync();

    // ---- Z: [P | Q] = U [Mp ; Kp]^T ----
    if (tid == 0) stage_mma(tmem, D::TZ, 32, I32, aU, aB + kBZ, 0, 0, &s_mbar, LO);
    wait_mma();
#pragma unroll
    for (int t = 0; t < D::TZ; ++t) {
      float v[32];
      tmem_ld32(tmem + lane_base + t * 32, v);
      const int row = t * 128 + tid;
      if (row < D::RZ) {
        const int x = row % C, y = row / C;
#pragma unroll
        for (int i = 0; i < M; ++i) {
          st_op2<LO>(OPP, x + C * i, y, v[i]);
          st_op2<LO>(OPQ, x + C * i, y, v[16 + i]);
        }
      }
    }
    stage_sync();
    // ---- Y: [A1 | A2] = P [Mp ; Kp]^T + Q [0 ; Mp]^T ----
    if (tid == 0) stage_mma(tmem, D::TY, 32, I32, aP, aB + kBZ, aQ, aB + kBY2, &s_mbar, LO);
    wait_mma();
#pragma unroll
    for (int t = 0; t < D::TY; ++t) {
      float v[32];
      tmem_ld32(tmem + lane_base + t * 32, v);
      const int row = t * 128 + tid;
      if (row < D::RY) {
        const int x = row % C, z = row / C;
#pragma unroll
        for (int i = 0; i < M; ++i) {
          st_op2<LO>(OPP, i + M * z, x, v[i]);
          st_op2<LO>(OPQ, i + M * z, x, v[16 + i]);
        }
      }
    }
    stage_sync();
    // ---- X: r = h^{2-d} b - (A1 Kp^T + A2 Mp^T) ----
    if (tid == 0) stage_mma(tmem, D::TX, 32, I16, aP, aB + kBKP, aQ, aB + kBMP, &s_mbar, LO);
    wait_mma();
#pragma unroll
    for (int t = 0; t < D::TX; ++t) {
      float v[16];
      tmem_ld16(tmem + lane_base + t * 32, v);
      const int row = t * 128 + tid;
      if (row < D::RX) {
        const float* __restrict__ brow = bg + org + 1 + py * (row % M + 1) + pz * (row / M + 1);
#pragma unroll
        for (int i = 0; i < M; ++i) st_op2<LO>(OPP, row, i, sb * __ldg(brow + i) - v[i]);
      }
    }
    stage_sync();
    // ---- FX: modes along x (lines (y,z)) -> operand of FY (lines (ix,z), K = y) ----
    if (tid == 0) stage_mma(tmem, D::TX, 32, I16, aP, aB + kBTT, 0, 0, &s_mbar, LO);
    wait_mma();
#pragma unroll
    for (int t = 0; t < D::TX; ++t) {
      float v[16];
      tmem_ld16(tmem + lane_base + t * 32, v);
      const int row = t * 128 + tid;
      if (row < D::RX) {
        const int y = row % M, z = row / M;
#pragma unroll
        for (int i = 0; i < M; ++i) st_op2<LO>(OPQ, i + M * z, y, v[i]);
      }
    }
    stage_sync();
    // ---- FY -> operand of FZ (lines (ix,iy), K = z) ----
    if (tid == 0) stage_mma(tmem, D::TX, 32, I16, aQ, aB + kBTT, 0, 0, &s_mbar, LO);
    wait_mma();
#pragma unroll
    for (int t = 0; t < D::TX; ++t) {
      float v[16];
      tmem_ld16(tmem + lane_base + t * 32, v);
      const int row = t * 128 + tid;
      if (row < D::RX) {
        const int ix = row % M, z = row / M;
#pragma unroll
        for (int i = 0; i < M; ++i) st_op2<LO>(OPP, ix + M * i, z, v[i]);
      }
    }
    stage_sync();
    // ---- FZ, times the FD diagonal -> operand of BZ (same lines, K = iz) ----
    if (tid == 0) stage_mma(tmem, D::TX, 32, I16, aP, aB + kBTT, 0, 0, &s_mbar, LO);
    wait_mma();
#pragma unroll
    for (int t = 0; t < D::TX; ++t) {
      float v[16];
      tmem_ld16(tmem + lane_base + t * 32, v);
      const int row = t * 128 + tid;
      if (row < D::RX) {
#pragma unroll
        for (int i = 0; i < M; ++i) st_op2<LO>(OPQ, row, i, v[i] * __ldg(dinv + row + M * M * i));
      }
    }
    stage_sync();
    // ---- BZ -> operand of BY (lines (ix,z), K = iy) ----
    if (tid == 0) stage_mma(tmem, D::TX, 32, I16, aQ, aB + kBTN, 0, 0, &s_mbar, LO);
    wait_mma();
#pragma unroll
    for (int t = 0; t < D::TX; ++t) {
      float v[16];
      tmem_ld16(tmem + lane_base + t * 32, v);
      const int row = t * 128 + tid;
      if (row < D::RX) {
        const int ix = row % M, iy = row / M;
#pragma unroll
        for (int i = 0; i < M; ++i) st_op2<LO>(OPP, ix + M * i, iy, v[i]);
      }
    }
    stage_sync();
    // ---- BY -> operand of BX (lines (y,z), K = ix) ----
    if (tid == 0) stage_mma(tmem, D::TX, 32, I16, aP, aB + kBTN, 0, 0, &s_mbar, LO);
    wait_mma();
#pragma unroll
    for (int t = 0; t < D::TX; ++t) {
      float v[16];
      tmem_ld16(tmem + lane_base + t * 32, v);
      const int row = t * 128 + tid;
      if (row < D::RX) {
        const int ix = row % M, z = row / M;
#pragma unroll
        for (int i = 0; i < M; ++i) st_op2<LO>(OPQ, i + M * z, ix, v[i]);
      }
    }
    stage_sync();
    // ---- BX and scatter: u_interior += omega d ----
    if (tid == 0) stage_mma(tmem, D::TX, 32, I16, aQ, aB + kBTN, 0, 0, &s_mbar, LO);
    wait_mma();
#pragma unroll
    for (int t = 0; t < D::TX; ++t) {
      float v[16];
      tmem_ld16(tmem + lane_base + t * 32, v);
      const int row = t * 128 + tid;
      if (row < D::RX) {
        const int y = row % M, z = row / M;
        const long long g = org + 1 + py * (y + 1) + pz * (z + 1);
#pragma unroll
        for (int i = 0; i < M; ++i) {
          // same-colour patches never write this patch's interior: the
          // value read is the gathered one
          uo[g + i] = fmaf(om, v[i], uo[g + i]);
        }
      }
    }
    fence_before();
    failed = __syncthreads_or(!ok) != 0;
    if (failed) break;
  }
  if (failed && tid == 0) atomicExch(err, GMG_ERR_TIMEOUT);
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0) tmem_dealloc(tmem, D::TCOLS);
}

// One 128 x 16 by 16 x 32 TF32 product on the tensor cores (the encoding
// check of the descriptors used above): D = A B^T.  With no_commit the MMAs
// are issued but their completion is never signalled, so the bounded wait
// expires and the kernel reports GMG_ERR_TIMEOUT (the failure path of the
// sweep kernel, exercised without a fault).
__global__ void __launch_bounds__(128) tc_probe_kernel(const float* __restrict__ A, const float* __restrict__ B,
                                                       float* __restrict__ Dout, int* __restrict__ err,
                                                       int no_commit) {
  __shared__ __align__(1024) unsigned char sa[kTileB];
  __shared__ __align__(1024) unsigned char sbm[32 * kRowB];
  __shared__ uint64_t s_mbar;
  __shared__ uint32_t s_tmem;
  const int tid = threadIdx.x, warp = tid >> 5;
  for (int k = 0; k < kKP; ++k) st_op(sa, tid, k, A[tid * kKP + k]);
  if (tid < 32)
    for (int k = 0; k < kKP; ++k) st_op(sbm, tid, k, B[tid * kKP + k]);
  if (warp == 0) tmem_alloc(&s_tmem, 32);
  if (tid == 0) mbar_init(&s_mbar, 1);
  fence_proxy_async();
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = s_tmem;
  if (tid == 0) {
    if (no_commit) {
      fence_after();
      for (int kk = 0; kk < 2; ++kk)
        mma_tf32(tmem, sdesc(smem_u32(sa) + kk * 2 * kChunkB), sdesc(smem_u32(sbm) + kk * 2 * kChunkB),
                 idesc_tf32(128, 32), kk);
    } else {
      stage_mma(tmem, 1, 32, idesc_tf32(128, 32), smem_u32(sa), smem_u32(sbm), 0, 0, &s_mbar);
    }
  }
  const bool ok = mbar_wait(&s_mbar, 0, no_commit ? 4096u : kWaitLimit);
  if (no_commit) {  // let the uncommitted MMAs retire before the TMEM is read and freed
    if (tid == 0) mma_commit(&s_mbar);
    mbar_wait(&s_mbar, 0);
  }
  fence_after();
  float v[32];
  tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16), v);
  for (int n = 0; n < 32; ++n) Dout[tid * 32 + n] = v[n];
  if (!ok) atomicExch(err, GMG_ERR_TIMEOUT);
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0) tmem_dealloc(tmem, 32);
}

float tf32_host(float x) {  // round to nearest (ties away) to a 10-bit mantissa
  uint32_t u;
  std::memcpy(&u, &x, 4);
  u = (u + 0x1000u) & ~0x1FFFu;
  float r;
  std::memcpy(&r, &u, 4);
  return r;
}

template <int K, bool SPLIT>
int launch_k(PatchTable& tab, const float* dinv, cudaStream_t s) {
  using D = TcDims<K, SPLIT>;
  auto kern = patch_tc_kernel<K, SPLIT>;
  static PerDevice<int> per_sm_dev;
  int* const per_sm_p = per_sm_dev.get();
  if (!per_sm_p) return GMG_ERR_CUDA;
  int& per_sm = *per_sm_p;
  if (per_sm == 0) {
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, D::SMEM) != cudaSuccess)
      return GMG_ERR_CUDA;
    // resident CTAs per SM from the kernel's own limits (the occupancy query
    // reports one CTA for kernels that allocate tensor memory): shared memory,
    // registers, warps and the 512 tensor-memory columns of an SM
    cudaFuncAttributes fa;
    int dev = 0, smem_sm = 0, regs_sm = 0;
    if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) != cudaSuccess)
      return GMG_ERR_CUDA;
    const int by_smem = smem_sm / (D::SMEM + (int)fa.sharedSizeBytes + 1024);
    const int by_regs = regs_sm / (std::max(fa.numRegs, 1) * 128);
    per_sm = std::max(1, std::min({by_smem, by_regs, 16, 512 / D::TCOLS}));
  }
  int g = 0;
  for (int i = 0; i < tab.n; ++i) {
    tab.e[i].group_begin = g;
    g += tab.e[i].n_patches;
  }
  tab.total_groups = g;
  if (g <= 0) return GMG_OK;
  static PerDevice<int> sms_dev;
  int* const sms_p = sms_dev.get();
  if (!sms_p) return GMG_ERR_CUDA;
  int& sms = *sms_p;
  if (sms == 0) {
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, current_device()) != cudaSuccess || sms <= 0)
      sms = 152;
  }
  void* bops = nullptr;
  void* errp = nullptr;
  if (cudaGetSymbolAddress(&bops, g_bops) != cudaSuccess || cudaGetSymbolAddress(&errp, g_tc_error) != cudaSuccess)
    return GMG_ERR_CUDA;
  const float* bk = static_cast<const float*>(bops) + (size_t)(K - kMinK) * 2 * kBopsFloats;
  kern<<<std::min(g, per_sm * sms), 128, D::SMEM, s>>>(tab, dinv, bk, static_cast<int*>(errp));
  count_launch();
  return cudaGetLastError() == cudaSuccess ? GMG_OK : GMG_ERR_CUDA;
}

int launch_table(int k, bool split, PatchTable& tab, const float* dinv, cudaStream_t s) {
  switch (k * 2 + (split ? 1 : 0)) {
    case 8: return launch_k<4, false>(tab, dinv, s);
    case 9: return launch_k<4, true>(tab, dinv, s);
    case 10: return launch_k<5, false>(tab, dinv, s);
    case 11: return launch_k<5, true>(tab, dinv, s);
    case 12: return launch_k<6, false>(tab, dinv, s);
    case 13: return launch_k<6, true>(tab, dinv, s);
    case 14: return launch_k<7, false>(tab, dinv, s);
    case 15: return launch_k<7, true>(tab, dinv, s);
    default: return GMG_ERR_UNSUPPORTED;
  }
}

void fill(PatchEntry& e, const PatchLaunch& pl, void* u, const void* b) {
  e.N = pl.g.N;
  e.py = pl.g.py;
  e.pz = pl.g.pz;
  for (int a = 0; a < 3; ++a) {
    e.first[a] = pl.first[a];
    e.count[a] = pl.count[a];
  }
  e.n_patches = pl.n_patches;
  e.group_begin = 0;
  e.sb = pl.sb;
  e.u = u;
  e.b = b;
  e.plist = pl.plist;
}

}  // namespace tc

int* device_wait_flag() {
  static PerDevice<int*> flag_dev;
  int** const flag = flag_dev.get();
  if (!flag) return nullptr;
  if (!*flag) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, tc::g_tc_error) == cudaSuccess)
      *flag = static_cast<int*>(p);
    else
      cudaGetLastError();
  }
  return *flag;
}

bool tc_supported(int dim, int k) { return dim == 3 && k >= tc::kMinK && k <= tc::kMaxK; }

int upload_tc_tables(int k, const double* Mp, const double* Kp, const double* That) {
  if (k < tc::kMinK || k > tc::kMaxK) return GMG_OK;  // nothing to do for other degrees
  const int C = 2 * k + 1, M = 2 * k - 1;
  std::vector<float> h(2 * tc::kBopsFloats, 0.f);
  auto put = [&](int base, int n, int kk, double v) {
    const float f = (float)v, hi = tc::tf32_host(f);
    h[(base + tc::op_off(n, kk)) / 4] = hi;
    h[(tc::kBLo + base + tc::op_off(n, kk)) / 4] = tc::tf32_host(f - hi);
  };
  for (int n = 0; n < M; ++n)
    for (int j = 0; j < C; ++j) {
      put(tc::kBZ, n, j, Mp[n * C + j]);
      put(tc::kBZ, 16 + n, j, Kp[n * C + j]);
      put(tc::kBY2, 16 + n, j, Mp[n * C + j]);
      put(tc::kBKP, n, j, Kp[n * C + j]);
      put(tc::kBMP, n, j, Mp[n * C + j]);
    }
  for (int i = 0; i < M; ++i)
    for (int j = 0; j < M; ++j) {
      put(tc::kBTT, i, j, That[j * M + i]);  // row = mode i, K = node j
      put(tc::kBTN, j, i, That[j * M + i]);  // row = node j, K = mode i
    }
  return cudaMemcpyToSymbol(tc::g_bops, h.data(), h.size() * 4, (size_t)(k - tc::kMinK) * 2 * tc::kBopsFloats * 4) ==
                 cudaSuccess
             ? GMG_OK
             : GMG_ERR_CUDA;
}

int launch_patch_tc(const PatchLaunch& pl, float* u, const float* b, const float* dinv, bool split,
                    cudaStream_t s) {
  if (pl.n_patches <= 0) return GMG_OK;
  if (pl.mode != 0 || !tc_supported(pl.g.dim, pl.g.k)) return GMG_ERR_UNSUPPORTED;
  PatchTable tab;
  tab.n = 1;
  tab.mode = 0;
  tab.omega = pl.omega;
  tc::fill(tab.e[0], pl, u, b);
  return tc::launch_table(pl.g.k, split, tab, dinv, s);
}

int launch_patch_table_tc(int dim, int k, const PatchLaunch* pls, float* const* us, const float* const* bs, int n,
                          const float* dinv, bool split, cudaStream_t s) {
  if (!tc_supported(dim, k)) return GMG_ERR_UNSUPPORTED;
  for (int i0 = 0; i0 < n; i0 += kMaxTable) {
    PatchTable tab;
    tab.n = 0;
    tab.mode = 0;
    tab.omega = pls[i0].omega;
    for (int i = i0; i < std::min(n, i0 + kMaxTable); ++i) {
      if (pls[i].n_patches <= 0) continue;
      if (pls[i].mode != 0) return GMG_ERR_UNSUPPORTED;
      tc::fill(tab.e[tab.n++], pls[i], us[i], bs[i]);
    }
    if (tab.n == 0) continue;
    const int st = tc::launch_table(k, split, tab, dinv, s);
    if (st != GMG_OK) return st;
  }
  return GMG_OK;
}

}  // namespace gmg

extern "C" {

int gmg_tc_status(void) {
  int h = 0, zero = 0;
  if (cudaDeviceSynchronize() != cudaSuccess) return GMG_ERR_CUDA;
  if (cudaMemcpyFromSymbol(&h, gmg::tc::g_tc_error, sizeof(int)) != cudaSuccess ||
      cudaMemcpyToSymbol(gmg::tc::g_tc_error, &zero, sizeof(int)) != cudaSuccess)
    return GMG_ERR_CUDA;
  return h == 0 ? GMG_OK : h;
}

int gmg_tc_probe(const float* A, const float* B, float* Dout, int force_timeout) {
  if (!A || !B || !Dout) return GMG_ERR_INVALID_ARG;
  float *dA = nullptr, *dB = nullptr, *dD = nullptr;
  int* dE = nullptr;
  int st = GMG_OK;
  if (cudaMalloc(&dA, 128 * 16 * 4) != cudaSuccess || cudaMalloc(&dB, 32 * 16 * 4) != cudaSuccess ||
      cudaMalloc(&dD, 128 * 32 * 4) != cudaSuccess || cudaMalloc(&dE, 4) != cudaSuccess) {
    st = GMG_ERR_OOM;
  } else if (cudaMemcpy(dA, A, 128 * 16 * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
             cudaMemcpy(dB, B, 32 * 16 * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
             cudaMemset(dE, 0, 4) != cudaSuccess) {
    st = GMG_ERR_CUDA;
  } else {
    gmg::tc::tc_probe_kernel<<<1, 128>>>(dA, dB, dD, dE, force_timeout ? 1 : 0);
    gmg::count_launch();
    int e = 0;
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(Dout, dD, 128 * 32 * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(&e, dE, 4, cudaMemcpyDeviceToHost) != cudaSuccess)
      st = GMG_ERR_CUDA;
    else if (e != 0)
      st = e;
  }
  cudaFree(dA);
  cudaFree(dB);
  cudaFree(dD);
  cudaFree(dE);
  return st;
}

}  // extern "C"

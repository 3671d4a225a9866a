// Host side of the TMA gathers: the driver's tensor-map encoder (resolved
// once through the runtime) and the tiled maps of a level vector.
#pragma once
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace gmg {

inline PFN_cuTensorMapEncodeTiled_v12000 tma_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    else
      cudaGetLastError();
  }
  return fn;
}

// A level vector can be read by TMA boxes when its base is 16-byte aligned
// and its row and plane pitches (elements of es bytes) are multiples of 16
// bytes.
inline bool tma_vector_ok(const void* ptr, int es, int dim, long long py, long long pz) {
  if (!tma_encoder() || ((uintptr_t)ptr & 15)) return false;
  if ((py * es) % 16) return false;
  if (dim == 3 && (pz * es) % 16) return false;
  return true;
}

// Tiled map of the lattice {N, N[, N]} of one vector with box
// {xbox, rows[, rows]} (xbox * es a multiple of 16 bytes), no swizzle,
// out-of-lattice elements read as zero.
inline bool tma_encode(CUtensorMap* m, const void* ptr, int es, int dim, int N, long long py, long long pz,
                       int xbox, int rows) {
  const cuuint64_t gdim[3] = {(cuuint64_t)N, (cuuint64_t)N, (cuuint64_t)N};
  const cuuint64_t gstride[2] = {(cuuint64_t)(py * es), (cuuint64_t)(pz * es)};
  const cuuint32_t box[3] = {(cuuint32_t)xbox, (cuuint32_t)rows, (cuuint32_t)rows};
  const cuuint32_t estride[3] = {1, 1, 1};
  const CUresult r = tma_encoder()(m, es == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                                   (cuuint32_t)dim, const_cast<void*>(ptr), gdim, gstride, box, estride,
                                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                   CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace gmg

// Launchers of the variable-coefficient kernels for one scalar type;
// included after var_kernels.cuh by var_f32.cu / var_f64.cu.
#pragma once
#include <algorithm>
#include <vector>

#include "../../include/gmg.h"
#include "tma_host.h"

namespace gmg {
namespace GMG_NS {

constexpr int kVarThreads = 128;
template <int DIM, int K>
struct VarCfg {
  static constexpr int E = K + 1;
  static constexpr int CPC = DIM == 3 ? 128 / (E * E) : 128 / E;  // cells per CTA of the operator
};

template <int DIM, int K>
static int apply_var_impl(const LevelGeom& g, long long n_elems, const T* x, T* y, const T* bvec,
                          double alpha, double beta, const T* coef, cudaStream_t s) {
  init_interior_kernel<<<(int)std::min<long long>((n_elems + 255) / 256, 152LL * 16), 256, 0, s>>>(
      y, bvec, (T)beta, g, n_elems);
  count_launch();
  constexpr int CPC = VarCfg<DIM, K>::CPC;
  const long long ncell = DIM == 3 ? (long long)g.n * g.n * g.n : (long long)g.n * g.n;
  const int grid = (int)std::min<long long>((ncell + CPC - 1) / CPC, 152LL * 32);
  apply_var_kernel<DIM, K, kVarThreads, CPC><<<grid, kVarThreads, 0, s>>>(x, y, coef, g, (T)alpha);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? GMG_OK : GMG_ERR_CUDA;
}

// persistent grid of the variable-coefficient sweep kernel (resident CTAs per SM)
template <int DIM, int K, bool TMA>
static int var_grid(int n_patches) {
  static PerDevice<int> per_sm_dev;  // resident CTAs on the whole device
  int* const per_sm_p = per_sm_dev.get();
  if (!per_sm_p) return -1;
  int& per_sm = *per_sm_p;
  if (per_sm == 0) {
    int dev = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, patch_var_kernel<DIM, K, kVarThreads, TMA>,
                                                      kVarThreads, 0) != cudaSuccess ||
        per_sm <= 0 || cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return -1;
    per_sm *= sms;
  }
  return std::min(n_patches, per_sm);
}

template <int DIM, int K>
static int patch_var_impl(const PatchLaunch& pl, T* u, const T* b, const T* coef, const T* vscale, const T* dinv,
                          const float* corr, int rank, cudaStream_t s) {
  if (pl.n_patches <= 0) return GMG_OK;
  int* const flag = device_wait_flag();
  if (!flag) return GMG_ERR_CUDA;
  const int es = (int)sizeof(T);
  if (tma_vector_ok(u, es, DIM, pl.g.py, pl.g.pz) && tma_vector_ok(b, es, DIM, pl.g.py, pl.g.pz)) {
    using Z = SweepSmem<DIM, K, true>;
    TmaMaps<1> maps;
    if (!tma_encode(&maps.u[0], u, es, DIM, pl.g.N, pl.g.py, pl.g.pz, Z::XU, Z::C) ||
        !tma_encode(&maps.b[0], b, es, DIM, pl.g.N, pl.g.py, pl.g.pz, Z::XB, Z::M))
      return GMG_ERR_CUDA;
    const int grid = var_grid<DIM, K, true>(pl.n_patches);
    if (grid <= 0) return GMG_ERR_CUDA;
    patch_var_kernel<DIM, K, kVarThreads, true><<<grid, kVarThreads, 0, s>>>(u, b, coef, vscale, dinv, corr, rank,
                                                                             pl, maps, flag);
  } else {
    const int grid = var_grid<DIM, K, false>(pl.n_patches);
    if (grid <= 0) return GMG_ERR_CUDA;
    patch_var_kernel<DIM, K, kVarThreads, false><<<grid, kVarThreads, 0, s>>>(u, b, coef, vscale, dinv, corr, rank,
                                                                              pl, TmaMaps<0>(), flag);
  }
  count_launch();
  return cudaGetLastError() == cudaSuccess ? GMG_OK : GMG_ERR_CUDA;
}

#define GMG_VAR_DISPATCH(FN, DIMV, KV, ...)              \
  switch ((DIMV) * 16 + (KV)) {                          \
    case 2 * 16 + 1: return FN<2, 1>(__VA_ARGS__);       \
    case 2 * 16 + 2: return FN<2, 2>(__VA_ARGS__);       \
    case 2 * 16 + 3: return FN<2, 3>(__VA_ARGS__);       \
    case 3 * 16 + 1: return FN<3, 1>(__VA_ARGS__);       \
    case 3 * 16 + 2: return FN<3, 2>(__VA_ARGS__);       \
    case 3 * 16 + 3: return FN<3, 3>(__VA_ARGS__);       \
    default: return GMG_ERR_UNSUPPORTED;                 \
  }

}  // namespace GMG_NS

template <>
int upload_var_tables<GMG_T>(int k, const double* Mc, const double* Kc, const double* That) {
  if (k < 1 || k > 8) return GMG_ERR_INVALID_ARG;
  using namespace GMG_NS;
  const int M = 2 * k - 1;
  std::vector<T> mc((k + 1) * (k + 1)), kc((k + 1) * (k + 1)), tt(M * M);
  for (int i = 0; i < (k + 1) * (k + 1); ++i) { mc[i] = (T)Mc[i]; kc[i] = (T)Kc[i]; }
  for (int i = 0; i < M * M; ++i) tt[i] = (T)That[i];
  cudaError_t e = cudaMemcpyToSymbol(c_Mc, mc.data(), mc.size() * sizeof(T), off_cell(k) * sizeof(T));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_Kc, kc.data(), kc.size() * sizeof(T), off_cell(k) * sizeof(T));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_T, tt.data(), tt.size() * sizeof(T), off_t(k) * sizeof(T));
  if (sizeof(T) == 8) {  // float pairs (hi, lo) for the double-float kernels
    auto split = [](const double* v, int n, std::vector<float>& hi, std::vector<float>& lo) {
      hi.resize(n);
      lo.resize(n);
      for (int i = 0; i < n; ++i) {
        hi[i] = (float)v[i];
        lo[i] = (float)(v[i] - (double)hi[i]);
      }
    };
    std::vector<float> h, l;
    const int nc = (k + 1) * (k + 1);
    const size_t co = off_cell(k) * sizeof(float), cb = nc * sizeof(float);
    split(Mc, nc, h, l);
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_Mchi, h.data(), cb, co);
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_Mclo, l.data(), cb, co);
    split(Kc, nc, h, l);
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_Kchi, h.data(), cb, co);
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_Kclo, l.data(), cb, co);
    split(That, M * M, h, l);
    const size_t to = off_t(k) * sizeof(float), tb = M * M * sizeof(float);
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_Thi, h.data(), tb, to);
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_Tlo, l.data(), tb, to);
  }
  return e == cudaSuccess ? GMG_OK : GMG_ERR_CUDA;
}

template <>
int launch_apply_var<GMG_T>(const LevelGeom& g, long long n_elems, const GMG_T* x, GMG_T* y,
                            const GMG_T* bvec, double alpha, double beta, const GMG_T* coef,
                            cudaStream_t s) {
  GMG_VAR_DISPATCH(GMG_NS::apply_var_impl, g.dim, g.k, g, n_elems, x, y, bvec, alpha, beta, coef, s)
}

template <>
int launch_patch_var<GMG_T>(const PatchLaunch& pl, GMG_T* u, const GMG_T* b, const GMG_T* coef,
                            const GMG_T* vscale, const GMG_T* dinv, const float* corr, int rank, cudaStream_t s) {
  GMG_VAR_DISPATCH(GMG_NS::patch_var_impl, pl.g.dim, pl.g.k, pl, u, b, coef, vscale, dinv, corr, rank, s)
}

}  // namespace gmg

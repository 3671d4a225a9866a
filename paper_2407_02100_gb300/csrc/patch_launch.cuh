// Launchers for one scalar type; included after patch_kernels.cuh by
// patch_f64.cu / patch_f32.cu.
#pragma once
#include <algorithm>
#include <vector>

#include "../../include/gmg.h"
#include "tma_host.h"
#include "staged_apply.cuh"

namespace gmg {
namespace GMG_NS {

constexpr int kApplyThreads = 128;

// Sweep kernel configuration: patches per CTA (enough interior lines per
// stage to fill whole warps), threads, and double buffering of the inputs
// whenever two input buffers fit in about half of the shared memory.
template <int DIM, int K>
struct SweepCfg {
  // FP64 is bound by the FP64 pipe: many patches per CTA for full warps, one
  // input buffer (occupancy hides the gather).  FP32 is bound by issue and
  // latency: fewer patches per CTA, double-buffered inputs.
  static constexpr bool F64 = sizeof(T) == 8;
  // FP32 3D k = 4: one patch per CTA of 64 threads (many small CTAs hide the
  // stage barriers better; measured 1.023 -> 0.934 ms per 64^3 sweep)
  static constexpr int PPC = DIM == 2 ? 8
                           : F64 ? (K <= 2 ? 8 : K <= 4 ? 4 : K <= 6 ? 2 : 1)
                                 : (K <= 2 ? 8 : K == 3 ? 4 : 1);
  static constexpr int NT = DIM == 3 && !F64 && K == 4 ? 64
                          : DIM == 3 && (K >= 6 || (F64 && K >= 3)) ? 256 : 128;
  static constexpr int NBUF =
      !F64 && PPC * SweepSmem<DIM, K>::per_patch(2) * (int)sizeof(T) <= 110 * 1024 ? 2 : 1;
  static constexpr int SMEM = PPC * SweepSmem<DIM, K>::per_patch(NBUF) * (int)sizeof(T);
  static_assert(SMEM <= 227 * 1024, "sweep kernel shared memory exceeds the per-CTA limit");
};

// Tile of the operator kernel (cells per direction x, y, z) and its threads.
// A tile recomputes a halo of K + 1 nodes below it in each direction, so
// flat tiles (large in x and y, one cell in z) do less redundant work; the
// shapes below were measured on GB300 (3D, against cubes): FP64 k = 3 -34 %,
// k = 4 -37 %, k = 7 -39 %; FP32 k = 3 -49 %, k = 7 -50 %; FP32 k = 4 and the
// small degrees are fastest with cubes.
template <int DIM, int K>
struct ApplyCfg {
  static constexpr bool F64 = sizeof(T) == 8;
  static constexpr int BC = DIM == 3 ? (K == 1 ? 8 : K == 2 ? 4 : K <= 4 ? 2 : 1)
                                     : (K == 1 ? 16 : K == 2 ? 8 : K <= 4 ? 4 : 2);
  static constexpr bool FLAT = DIM == 3 && (F64 ? (K >= 3 && K <= 7) : (K == 3 || K == 7));
  static constexpr int BX = !FLAT ? BC : K == 3 ? (F64 ? 8 : 4) : K == 4 ? 8 : K == 7 ? 4 : 2;
  static constexpr int BY = !FLAT ? BC : K == 3 ? (F64 ? 8 : 4) : K == 4 ? 4 : 2;
  static constexpr int BZ = FLAT ? 1 : BC;
  static constexpr int NT = FLAT && !(K == 3 && !F64) ? 256 : kApplyThreads;
};

static int sm_count() {
  static PerDevice<int> sms_dev;
  int* const sms = sms_dev.get();
  if (!sms) return 152;
  if (*sms == 0) {
    if (cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, current_device()) != cudaSuccess || *sms <= 0)
      *sms = 152;
  }
  return *sms;
}

template <typename KernelT>
// opt the kernel in to its dynamic shared memory (the 48 KB default covers
// static plus dynamic memory, so the attribute is set whatever the size)
static int prepare(KernelT kern, int smem) {
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
    return GMG_ERR_CUDA;
  return GMG_OK;
}

// Fill the table entries' group ranges for PPC patches per CTA.
static inline int table_groups(PatchTable& tab, int ppc) {
  int g = 0;
  for (int i = 0; i < tab.n; ++i) {
    tab.e[i].group_begin = g;
    g += (tab.e[i].n_patches + ppc - 1) / ppc;
  }
  tab.total_groups = g;
  return g;
}

// ---- TMA gather: every vector of the table must allow the boxes ----
static bool tma_usable(const PatchTable& tab, int dim) {
  for (int i = 0; i < tab.n; ++i) {
    const PatchEntry& e = tab.e[i];
    if (e.N < 2 || !tma_vector_ok(e.u, (int)sizeof(T), dim, e.py, e.pz) ||
        !tma_vector_ok(e.b, (int)sizeof(T), dim, e.py, e.pz))
      return false;
  }
  return true;
}

template <int DIM, int K, int PPC, int NT, int NBUF, int ME>
static int launch_table_cfg(PatchTable& tab, const T* dinv, cudaStream_t s) {
  using Z = SweepSmem<DIM, K, (ME > 0)>;
  constexpr int SMEM = PPC * Z::per_patch(NBUF) * (int)sizeof(T) + (ME > 0 ? 128 : 0);
  static_assert(SMEM <= 227 * 1024, "sweep kernel shared memory exceeds the per-CTA limit");
  auto kern = patch_colour_kernel<DIM, K, NT, PPC, NBUF, ME>;
  static PerDevice<int> per_sm_dev;  // resident CTAs per SM (persistent grid)
  int* const per_sm_p = per_sm_dev.get();
  if (!per_sm_p) return GMG_ERR_CUDA;
  int& per_sm = *per_sm_p;
  if (per_sm == 0) {
    if (prepare(kern, SMEM) != GMG_OK) return GMG_ERR_CUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, SMEM) != cudaSuccess ||
        per_sm <= 0)
      return GMG_ERR_CUDA;
  }
  const int ngroups = table_groups(tab, PPC);
  if (ngroups <= 0) return GMG_OK;
  TmaMaps<ME> maps;
  if constexpr (ME > 0) {
    for (int i = 0; i < tab.n; ++i) {
      const PatchEntry& e = tab.e[i];
      if (!tma_encode(&maps.u[i], e.u, (int)sizeof(T), DIM, e.N, e.py, e.pz, Z::XU, Z::C) ||
          !tma_encode(&maps.b[i], e.b, (int)sizeof(T), DIM, e.N, e.py, e.pz, Z::XB, Z::M))
        return GMG_ERR_CUDA;
    }
  }
  int* const flag = device_wait_flag();
  if (!flag) return GMG_ERR_CUDA;
  const int grid = std::min(ngroups, per_sm * sm_count());
  kern<<<grid, NT, SMEM, s>>>(tab, dinv, maps, flag);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? GMG_OK : GMG_ERR_CUDA;
}

// the TMA-gather variant when every vector of the table allows it, else the
// per-element cp.async gather
template <int DIM, int K, int PPC, int NT, int NBUF>
static int launch_table_gather(PatchTable& tab, const T* dinv, cudaStream_t s) {
  if (tma_usable(tab, DIM)) {
    if (tab.n == 1) return launch_table_cfg<DIM, K, PPC, NT, NBUF, 1>(tab, dinv, s);
    return launch_table_cfg<DIM, K, PPC, NT, NBUF, kMaxTable>(tab, dinv, s);
  }
  return launch_table_cfg<DIM, K, PPC, NT, NBUF, 0>(tab, dinv, s);
}

// default configuration (SweepCfg), or a tuned patches-per-CTA variant
template <int DIM, int K>
static int launch_table(PatchTable& tab, const T* dinv, int ppc, cudaStream_t s) {
  using Cfg = SweepCfg<DIM, K>;
  if constexpr (DIM == 3 && sizeof(T) == 4 && K <= 4) {
    constexpr int NB = SweepCfg<DIM, K>::NBUF;
    if (ppc == 1) return launch_table_gather<DIM, K, 1, 128, NB>(tab, dinv, s);
    if (ppc == 2) return launch_table_gather<DIM, K, 2, 128, NB>(tab, dinv, s);
    if (ppc == 4) return launch_table_gather<DIM, K, 4, 128, NB>(tab, dinv, s);
  }
  return launch_table_gather<DIM, K, Cfg::PPC, Cfg::NT, Cfg::NBUF>(tab, dinv, s);
}

static void fill_entry(PatchEntry& e, const PatchLaunch& pl, void* u, const void* b) {
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

template <int DIM, int K>
static int patch_impl(const PatchLaunch& pl, T* u, const T* b, const T* dinv, cudaStream_t s) {
  if (pl.n_patches <= 0) return GMG_OK;
  PatchTable tab;
  tab.n = 1;
  tab.mode = pl.mode;
  tab.omega = pl.omega;
  fill_entry(tab.e[0], pl, u, b);
  return launch_table<DIM, K>(tab, dinv, 0, s);
}

template <int DIM, int K>
static int table_impl(const PatchLaunch* pls, T* const* us, const T* const* bs, int n, const T* dinv,
                      int ppc, cudaStream_t s) {
  for (int i0 = 0; i0 < n; i0 += kMaxTable) {
    PatchTable tab;
    tab.n = 0;
    tab.mode = pls[i0].mode;
    tab.omega = pls[i0].omega;
    for (int i = i0; i < std::min(n, i0 + kMaxTable); ++i) {
      if (pls[i].n_patches <= 0) continue;
      fill_entry(tab.e[tab.n++], pls[i], us[i], bs[i]);
    }
    if (tab.n == 0) continue;
    const int st = launch_table<DIM, K>(tab, dinv, ppc, s);
    if (st != GMG_OK) return st;
  }
  return GMG_OK;
}

template <int DIM, int K, int BX, int BY, int BZ, int NT>
static int apply_cfg(const ApplyLaunch& al, const T* x, T* y, const T* bvec, cudaStream_t s) {
  using D = ApplyDims<DIM, K, BX, BY, BZ>;
  auto kern = apply_kernel<DIM, K, BX, BY, BZ, NT>;
  static PerDevice<bool> ready_dev;  // attribute set once per device (also keeps graph capture free of it)
  bool* const ready = ready_dev.get();
  if (!ready) return GMG_ERR_CUDA;
  if (!*ready) {
    if (prepare(kern, D::SMEM_BYTES) != GMG_OK) return GMG_ERR_CUDA;
    *ready = true;
  }
  const long long n = al.g.n;
  const long long ntile = ((n + BX - 1) / BX) * ((n + BY - 1) / BY) * (DIM == 3 ? (n + BZ - 1) / BZ : 1);
  int grid = (int)std::min<long long>(ntile, 1 << 30);
  kern<<<grid, NT, D::SMEM_BYTES, s>>>(x, y, bvec, al);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? GMG_OK : GMG_ERR_CUDA;
}

// degrees at which the FP64 3D three-pass form beats the tile kernel
constexpr bool staged_apply_degree(int k) { return k >= 3; }

// a tile variant of the operator if its shared memory fits, else the default
template <int DIM, int K, int BX, int BY, int BZ, int NT>
static int apply_variant(const ApplyLaunch& al, const T* x, T* y, const T* bvec, cudaStream_t s) {
  if constexpr (ApplyDims<DIM, K, BX, BY, BZ>::SMEM_BYTES <= 227 * 1024) {
    return apply_cfg<DIM, K, BX, BY, BZ, NT>(al, x, y, bvec, s);
  } else {
    using Cfg = ApplyCfg<DIM, K>;
    return apply_cfg<DIM, K, Cfg::BX, Cfg::BY, Cfg::BZ, Cfg::NT>(al, x, y, bvec, s);
  }
}

template <int DIM, int K>
static int apply_impl(const ApplyLaunch& al, const T* x, T* y, const T* bvec, cudaStream_t s) {
  if constexpr (DIM == 3 && sizeof(T) == 8 && staged_apply_degree(K))
    if (al.ws) return staged_apply_impl<K>(al, x, y, bvec, s);
  if constexpr (DIM == 3 && (K == 3 || K == 4 || K == 7)) {
    constexpr int BC = ApplyCfg<DIM, K>::BC;
    switch (al.tile) {
      case 1: return apply_variant<DIM, K, BC, BC, BC, kApplyThreads>(al, x, y, bvec, s);
      case 2: return apply_variant<DIM, K, 4, 4, 1, 128>(al, x, y, bvec, s);
      case 3: return apply_variant<DIM, K, 8, 4, 1, 256>(al, x, y, bvec, s);
      default: break;
    }
  }
  using Cfg = ApplyCfg<DIM, K>;
  static_assert(ApplyDims<DIM, K, Cfg::BX, Cfg::BY, Cfg::BZ>::SMEM_BYTES <= 227 * 1024,
                "operator tile exceeds the shared memory of a CTA");
  return apply_cfg<DIM, K, Cfg::BX, Cfg::BY, Cfg::BZ, Cfg::NT>(al, x, y, bvec, s);
}

#define GMG_DISPATCH(FN, DIMV, KV, ...)                                  \
  switch ((DIMV) * 16 + (KV)) {                                          \
    case 2 * 16 + 1: return FN<2, 1>(__VA_ARGS__);                       \
    case 2 * 16 + 2: return FN<2, 2>(__VA_ARGS__);                       \
    case 2 * 16 + 3: return FN<2, 3>(__VA_ARGS__);                       \
    case 2 * 16 + 4: return FN<2, 4>(__VA_ARGS__);                       \
    case 2 * 16 + 5: return FN<2, 5>(__VA_ARGS__);                       \
    case 2 * 16 + 6: return FN<2, 6>(__VA_ARGS__);                       \
    case 2 * 16 + 7: return FN<2, 7>(__VA_ARGS__);                       \
    case 2 * 16 + 8: return FN<2, 8>(__VA_ARGS__);                       \
    case 3 * 16 + 1: return FN<3, 1>(__VA_ARGS__);                       \
    case 3 * 16 + 2: return FN<3, 2>(__VA_ARGS__);                       \
    case 3 * 16 + 3: return FN<3, 3>(__VA_ARGS__);                       \
    case 3 * 16 + 4: return FN<3, 4>(__VA_ARGS__);                       \
    case 3 * 16 + 5: return FN<3, 5>(__VA_ARGS__);                       \
    case 3 * 16 + 6: return FN<3, 6>(__VA_ARGS__);                       \
    case 3 * 16 + 7: return FN<3, 7>(__VA_ARGS__);                       \
    case 3 * 16 + 8: return FN<3, 8>(__VA_ARGS__);                       \
    default: return GMG_ERR_INVALID_ARG;                                 \
  }

static int upload(int k, const double* Mp, const double* Kp, const double* That, const double* Mc,
                  const double* Kc) {
  if (k < 1 || k > 8) return GMG_ERR_INVALID_ARG;
  const int C = 2 * k + 1, M = 2 * k - 1;
  std::vector<T> mp(M * C), kp(M * C), tt(M * M), mc((k + 1) * (k + 1)), kc((k + 1) * (k + 1));
  for (int i = 0; i < M * C; ++i) { mp[i] = (T)Mp[i]; kp[i] = (T)Kp[i]; }
  for (int i = 0; i < M * M; ++i) tt[i] = (T)That[i];
  for (int i = 0; i < (k + 1) * (k + 1); ++i) { mc[i] = (T)Mc[i]; kc[i] = (T)Kc[i]; }
  cudaError_t e = cudaSuccess;
  e = e == cudaSuccess ? cudaMemcpyToSymbol(c_Mp, mp.data(), mp.size() * sizeof(T), off_patch(k) * sizeof(T)) : e;
  e = e == cudaSuccess ? cudaMemcpyToSymbol(c_Kp, kp.data(), kp.size() * sizeof(T), off_patch(k) * sizeof(T)) : e;
  e = e == cudaSuccess ? cudaMemcpyToSymbol(c_T, tt.data(), tt.size() * sizeof(T), off_t(k) * sizeof(T)) : e;
  e = e == cudaSuccess ? cudaMemcpyToSymbol(c_Mc, mc.data(), mc.size() * sizeof(T), off_cell(k) * sizeof(T)) : e;
  e = e == cudaSuccess ? cudaMemcpyToSymbol(c_Kc, kc.data(), kc.size() * sizeof(T), off_cell(k) * sizeof(T)) : e;
  std::vector<float> thi(M * M), tlo(M * M);
  for (int i = 0; i < M * M; ++i) {
    thi[i] = (float)That[i];
    tlo[i] = (float)(That[i] - (double)thi[i]);
  }
  e = e == cudaSuccess ? cudaMemcpyToSymbol(c_Thi, thi.data(), thi.size() * sizeof(float), off_t(k) * sizeof(float)) : e;
  e = e == cudaSuccess ? cudaMemcpyToSymbol(c_Tlo, tlo.data(), tlo.size() * sizeof(float), off_t(k) * sizeof(float)) : e;
  std::vector<float> mhi(M * C), mlo(M * C), khi(M * C), klo(M * C);
  for (int i = 0; i < M * C; ++i) {
    mhi[i] = (float)Mp[i];
    mlo[i] = (float)(Mp[i] - (double)mhi[i]);
    khi[i] = (float)Kp[i];
    klo[i] = (float)(Kp[i] - (double)khi[i]);
  }
  const size_t po = off_patch(k) * sizeof(float), pb = mhi.size() * sizeof(float);
  e = e == cudaSuccess ? cudaMemcpyToSymbol(c_Mphi, mhi.data(), pb, po) : e;
  e = e == cudaSuccess ? cudaMemcpyToSymbol(c_Mplo, mlo.data(), pb, po) : e;
  e = e == cudaSuccess ? cudaMemcpyToSymbol(c_Kphi, khi.data(), pb, po) : e;
  e = e == cudaSuccess ? cudaMemcpyToSymbol(c_Kplo, klo.data(), pb, po) : e;
  const int nc = (k + 1) * (k + 1);
  std::vector<float> mch(nc), mcl(nc), kch(nc), kcl(nc);
  for (int i = 0; i < nc; ++i) {
    mch[i] = (float)Mc[i];
    mcl[i] = (float)(Mc[i] - (double)mch[i]);
    kch[i] = (float)Kc[i];
    kcl[i] = (float)(Kc[i] - (double)kch[i]);
  }
  const size_t co = off_cell(k) * sizeof(float), cb = nc * sizeof(float);
  e = e == cudaSuccess ? cudaMemcpyToSymbol(c_Mchi, mch.data(), cb, co) : e;
  e = e == cudaSuccess ? cudaMemcpyToSymbol(c_Mclo, mcl.data(), cb, co) : e;
  e = e == cudaSuccess ? cudaMemcpyToSymbol(c_Kchi, kch.data(), cb, co) : e;
  e = e == cudaSuccess ? cudaMemcpyToSymbol(c_Kclo, kcl.data(), cb, co) : e;
  return e == cudaSuccess ? GMG_OK : GMG_ERR_CUDA;
}

}  // namespace GMG_NS

template <>
int upload_patch_tables<GMG_T>(int k, const double* Mp, const double* Kp, const double* That,
                               const double* Mc, const double* Kc, cudaStream_t) {
  return GMG_NS::upload(k, Mp, Kp, That, Mc, Kc);
}

template <>
int launch_patch_colour<GMG_T>(const PatchLaunch& pl, GMG_T* u, const GMG_T* b, const GMG_T* dinv,
                               cudaStream_t s) {
  GMG_DISPATCH(GMG_NS::patch_impl, pl.g.dim, pl.g.k, pl, u, b, dinv, s)
}

template <>
int launch_patch_table<GMG_T>(int dim, int k, const PatchLaunch* pls, GMG_T* const* us,
                              const GMG_T* const* bs, int n, const GMG_T* dinv, int ppc,
                              cudaStream_t s) {
  GMG_DISPATCH(GMG_NS::table_impl, dim, k, pls, us, bs, n, dinv, ppc, s)
}

template <>
int launch_apply<GMG_T>(const ApplyLaunch& al, const GMG_T* x, GMG_T* y, const GMG_T* bvec,
                        cudaStream_t s) {
  GMG_DISPATCH(GMG_NS::apply_impl, al.g.dim, al.g.k, al, x, y, bvec, s)
}

}  // namespace gmg

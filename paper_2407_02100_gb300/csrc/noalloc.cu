// gmg_smooth_noalloc: the FP64 patch smoother of one uniform level for
// callers that cannot allocate device memory.
//
// Who needs it: applications whose device memory is owned by another
// allocator (a framework arena or memory pool that has reserved the GPU), and
// callers that must not trigger cudaMalloc's implicit device-wide
// synchronisation in the middle of their own pipeline.  gmg_create() cannot
// serve them because it allocates the level hierarchy with cudaMalloc.
//
// The only device memory the sweep needs beyond the caller's u and b is the
// fast-diagonalisation diagonal 1/(lambda_x + lambda_y [+ lambda_z]) of the
// patch.  Here it lives in a file-scope __device__ array sized for the
// largest supported patch, (2*8-1)^3 doubles = 27 KB, which every GPU that
// loads the library keeps until the process exits.  The coefficient tables go
// to __constant__ memory with cudaMemcpyToSymbol, which allocates nothing.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <vector>

#include "../../include/gmg.h"
#include "kernels.h"
#include "setup.h"

namespace {

constexpr int kNoAllocMaxDiag = 15 * 15 * 15;  // (2k-1)^3 for the largest degree k = 8
constexpr int kMaxDevices = 64;

__device__ __align__(256) double g_fd_diag[kNoAllocMaxDiag];

std::mutex g_mutex;
double* g_fd_diag_addr[kMaxDevices] = {};

// Device address of g_fd_diag on the current device.  Host code cannot use
// the symbol itself (it names a host-side shadow), so the address is looked
// up once per device with that device current, then cached.
int scratch_address(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return GMG_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_fd_diag_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_fd_diag) != cudaSuccess || !p) {
      cudaGetLastError();
      return GMG_ERR_CUDA;
    }
    g_fd_diag_addr[dev] = static_cast<double*>(p);
  }
  *out = g_fd_diag_addr[dev];
  return GMG_OK;
}

}  // namespace

extern "C" int gmg_smooth_noalloc(int dim, int degree, int n_cells, double damping, double* u,
                                  const double* b, int n_sweeps, int reverse, void* stream) {
  using namespace gmg;
  if (dim != 2 && dim != 3) return GMG_ERR_INVALID_ARG;
  if (degree < 1 || degree > kMaxDegree || n_cells < 2) return GMG_ERR_INVALID_ARG;
  if ((long long)n_cells * degree + 1 > (1 << 20)) return GMG_ERR_INVALID_ARG;
  if (!std::isfinite(damping) || n_sweeps < 0 || !u || !b || (const double*)u == b)
    return GMG_ERR_INVALID_ARG;
  const int k = degree, m = 2 * k - 1, C = 2 * k + 1;
  const long long nint = dim == 3 ? (long long)m * m * m : (long long)m * m;
  if (nint > kNoAllocMaxDiag) return GMG_ERR_INVALID_ARG;

  double* diag = nullptr;
  int st = scratch_address(&diag);
  if (st != GMG_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  // host set-up math (unit cells, level independent) and constant tables
  std::vector<double> Mc, Kc, Mp, Kp, Mi, Ki, Tp, lp;
  cell_matrices_1d(k, Mc, Kc);
  assembled_1d(k, 2, 1, m, 0, C, Mp, Kp);
  assembled_1d(k, 2, 1, m, 1, m, Mi, Ki);
  if (!generalized_eigen_mirror(m, Mi, Ki, Tp, lp)) return GMG_ERR_INVALID_ARG;
  st = upload_patch_tables<double>(k, Mp.data(), Kp.data(), Tp.data(), Mc.data(), Kc.data(), s);
  if (st != GMG_OK) return st;
  std::vector<double> dinv(nint);
  for (long long t = 0; t < nint; ++t) {
    int x = (int)(t % m), y = (int)((t / m) % m), z = (int)(t / ((long long)m * m));
    dinv[t] = 1.0 / (lp[x] + lp[y] + (dim == 3 ? lp[z] : 0.0));
  }
  // the whole used part of the shared array is rewritten by every call
  if (cudaMemcpyAsync(diag, dinv.data(), nint * sizeof(double), cudaMemcpyHostToDevice, s) !=
      cudaSuccess)
    return GMG_ERR_CUDA;

  PatchLaunch pl;
  pl.g.dim = dim;
  pl.g.k = k;
  pl.g.n = n_cells;
  pl.g.N = n_cells * k + 1;
  pl.g.py = (pl.g.N + 3) / 4 * 4;
  pl.g.pz = (long long)pl.g.py * pl.g.N;
  pl.sb = dim == 3 ? (double)n_cells : 1.0;  // h^{2-d}
  pl.omega = damping;
  pl.plist = nullptr;
  pl.mode = 0;
  const int nc = 1 << dim;
  for (int sweep = 0; sweep < n_sweeps; ++sweep) {
    for (int i = 0; i < nc; ++i) {
      const int colour = reverse ? nc - 1 - i : i;
      pl.n_patches = 1;
      for (int a = 0; a < 3; ++a) {
        const bool odd = a < dim && ((colour >> a) & 1);
        pl.first[a] = a < dim ? (odd ? 1 : 2) : 1;
        pl.count[a] = a < dim ? (odd ? n_cells / 2 : (n_cells - 1) / 2) : 1;
        pl.n_patches *= pl.count[a];
      }
      if (pl.n_patches == 0) continue;
      st = launch_patch_colour<double>(pl, u, b, diag, s);
      if (st != GMG_OK) return st;
    }
  }
  return GMG_OK;
}

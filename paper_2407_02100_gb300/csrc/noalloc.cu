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
// patch, followed by the same values as float pairs (hi, lo) for the
// double-float FD transforms of the FP64 sweep kernel.  Here it lives in a
// file-scope __device__ array sized for the largest supported patch,
// 2 (2*8-1)^3 doubles = 54 KB, which every GPU that loads the library keeps
// until the process exits.  Every call writes the
// part of it that its degree uses with a small kernel on the caller's stream
// (the eigenvalues travel as a kernel argument), then launches the colours.
//
// Set-up, once per device and degree, with that device current: the array's
// device address is looked up (host code cannot use the symbol itself, which
// names a host-side shadow) and the degree's coefficient tables are copied to
// __constant__ memory with cudaMemcpyToSymbol, which allocates nothing but is
// synchronous.  The generalised eigenproblem of the degree is solved on the
// host once per process.  Later calls on that device and degree enqueue
// kernels only.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <vector>

#include "../../include/gmg.h"
#include "kernels.h"
#include "setup.h"

namespace {

constexpr int kNoAllocMaxDiag = 15 * 15 * 15;  // (2k-1)^3 for the largest degree k = 8
constexpr int kMaxM = 15;                       // 2k-1 for k = 8

__device__ __align__(256) double g_fd_diag[2 * kNoAllocMaxDiag];

// 1D eigenvalues of the two-cell patch pencil K T = M T Lambda (App. A.3)
struct Lambda1d {
  double v[kMaxM];
};

// diag[t] = 1 / (lambda_x + lambda_y [+ lambda_z]) for the interior index t
// of an m^dim patch (x fastest), and after the nint doubles the same values
// as float pairs (hi, lo), one pair per double slot
__global__ void fill_fd_diag_kernel(double* __restrict__ diag, Lambda1d lam, int m, int dim, int nint) {
  float2* const pairs = reinterpret_cast<float2*>(diag + nint);
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nint; t += gridDim.x * blockDim.x) {
    const int x = t % m, y = (t / m) % m, z = t / (m * m);
    const double v = 1.0 / (lam.v[x] + lam.v[y] + (dim == 3 ? lam.v[z] : 0.0));
    diag[t] = v;
    const float hi = (float)v;
    pairs[t] = make_float2(hi, (float)(v - (double)hi));
  }
}

struct DegreeData {
  bool ready = false;
  Lambda1d lam{};
  std::vector<double> Mc, Kc, Mp, Kp, Tp;
};

std::mutex g_mutex;
DegreeData g_degree[gmg::kMaxDegree + 1];                  // host set-up math per degree
double* g_fd_diag_addr[gmg::kMaxDevices] = {};             // array address per device
bool g_tables_uploaded[gmg::kMaxDevices][gmg::kMaxDegree + 1] = {};

// Host set-up of degree k (unit cells, level independent), solved once.
int degree_data(int k, const DegreeData** out) {
  DegreeData& d = g_degree[k];
  if (!d.ready) {
    const int m = 2 * k - 1, C = 2 * k + 1;
    std::vector<double> Mi, Ki, lp;
    gmg::cell_matrices_1d(k, d.Mc, d.Kc);
    gmg::assembled_1d(k, 2, 1, m, 0, C, d.Mp, d.Kp);
    gmg::assembled_1d(k, 2, 1, m, 1, m, Mi, Ki);
    if (!gmg::generalized_eigen_mirror(m, Mi, Ki, d.Tp, lp) || (int)lp.size() != m) return GMG_ERR_INVALID_ARG;
    for (int i = 0; i < m; ++i) d.lam.v[i] = lp[i];
    d.ready = true;
  }
  *out = &d;
  return GMG_OK;
}

// Per-device set-up for degree k on the current device: the array's address
// and the degree's __constant__ tables.
int device_setup(int k, double** diag, Lambda1d* lam) {
  const int dev = gmg::current_device();
  if (dev < 0) return GMG_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mutex);
  const DegreeData* d = nullptr;
  int st = degree_data(k, &d);
  if (st != GMG_OK) return st;
  if (!g_fd_diag_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_fd_diag) != cudaSuccess || !p) {
      cudaGetLastError();
      return GMG_ERR_CUDA;
    }
    g_fd_diag_addr[dev] = static_cast<double*>(p);
  }
  if (!g_tables_uploaded[dev][k]) {
    st = gmg::upload_patch_tables<double>(k, d->Mp.data(), d->Kp.data(), d->Tp.data(), d->Mc.data(),
                                          d->Kc.data(), nullptr);
    if (st != GMG_OK) return st;
    g_tables_uploaded[dev][k] = true;
  }
  *diag = g_fd_diag_addr[dev];
  *lam = d->lam;
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
  const int k = degree, m = 2 * k - 1;
  const long long nint = dim == 3 ? (long long)m * m * m : (long long)m * m;
  if (nint > kNoAllocMaxDiag || m > kMaxM) return GMG_ERR_INVALID_ARG;

  double* diag = nullptr;
  Lambda1d lam;
  int st = device_setup(k, &diag, &lam);
  if (st != GMG_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  // the part of the shared array this degree uses is rewritten on every call
  fill_fd_diag_kernel<<<(int)((nint + 255) / 256), 256, 0, s>>>(diag, lam, m, dim, (int)nint);
  count_launch();
  if (cudaGetLastError() != cudaSuccess) return GMG_ERR_CUDA;

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

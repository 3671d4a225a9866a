// C ABI (include/gmg.h): problem set-up, level operations, V-cycle and the
// preconditioned conjugate gradient driver.  All numerical work runs in the
// CUDA kernels of patch_f64.cu / patch_f32.cu / vector_kernels.cu; this file
// only builds tables on the host, owns device buffers and sequences launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/gmg.h"
#include "kernels.h"
#include "problem.h"
#include "setup.h"

using namespace gmg;

static std::atomic<long long> g_launches{0};
void gmg::count_launch(int n) { g_launches += n; }
long long gmg::launch_count() { return g_launches.load(); }

namespace gmg {
namespace detail {

enum { S_RZ = 0, S_PQ = 1, S_RR = 2, S_RZN = 3, S_BB = 4, S_COUNT = 8 };

void drop_cg_graph(gmg_problem* p) {
  if (p->cg_exec) cudaGraphExecDestroy(p->cg_exec);
  if (p->cg_graph) cudaGraphDestroy(p->cg_graph);
  p->cg_exec = nullptr;
  p->cg_graph = nullptr;
  p->cg_graph_u = nullptr;
}

static cudaEvent_t take_event(gmg_problem* p) {
  if (!p->event_pool.empty()) {
    cudaEvent_t e = p->event_pool.back();
    p->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

PhaseScope::PhaseScope(gmg_problem* p, int phase) : p_(p), phase_(phase) {
  if (!p_->phase_timing) return;
  if (p_->phase_depth++ > 0) return;
  start_ = take_event(p_);
  if (start_ && cudaEventRecord(start_, p_->stream) != cudaSuccess) {
    cudaGetLastError();
    p_->event_pool.push_back(start_);
    start_ = nullptr;
  }
}

PhaseScope::~PhaseScope() {
  if (!p_->phase_timing) return;
  --p_->phase_depth;
  if (!start_) return;
  cudaEvent_t stop = take_event(p_);
  if (stop && cudaEventRecord(stop, p_->stream) == cudaSuccess) {
    p_->phase_marks.push_back({phase_, start_, stop});
    return;
  }
  cudaGetLastError();
  p_->event_pool.push_back(start_);
  if (stop) p_->event_pool.push_back(stop);
}

void collect_phases(gmg_problem* p) {
  for (const auto& m : p->phase_marks) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, m.start, m.stop) == cudaSuccess)
      p->phase_ms[m.phase] += ms;
    else
      cudaGetLastError();
    p->event_pool.push_back(m.start);
    p->event_pool.push_back(m.stop);
  }
  p->phase_marks.clear();
}

void release_phase_events(gmg_problem* p) {
  for (const auto& m : p->phase_marks) {
    cudaEventDestroy(m.start);
    cudaEventDestroy(m.stop);
  }
  p->phase_marks.clear();
  for (cudaEvent_t e : p->event_pool) cudaEventDestroy(e);
  p->event_pool.clear();
}

int dalloc(gmg_problem* p, void** ptr, size_t bytes) {
  *ptr = nullptr;
  if (bytes == 0) bytes = 16;
  if (cudaMalloc(ptr, bytes) != cudaSuccess) {
    cudaGetLastError();
    return GMG_ERR_OOM;
  }
  p->owned.push_back(*ptr);
  if (cudaMemset(*ptr, 0, bytes) != cudaSuccess) return GMG_ERR_CUDA;
  return GMG_OK;
}

// upload host doubles as the problem precision
int upload_table(gmg_problem* p, void** dst, const std::vector<double>& src) {
  int st = dalloc(p, dst, src.size() * p->esize);
  if (st) return st;
  cudaError_t e;
  if (p->esize == 8) {
    e = cudaMemcpy(*dst, src.data(), src.size() * 8, cudaMemcpyHostToDevice);
  } else {
    std::vector<float> f(src.begin(), src.end());
    e = cudaMemcpy(*dst, f.data(), f.size() * 4, cudaMemcpyHostToDevice);
  }
  return e == cudaSuccess ? GMG_OK : GMG_ERR_CUDA;
}

// Append to a table of doubles the same entries as float pairs (hi, lo),
// two per double slot, for the double-float kernels of FP64 problems.
void append_float_pairs(std::vector<double>& t) {
  const size_t n = t.size();
  t.resize(2 * n);
  for (size_t i = 0; i < n; ++i) {
    const float pair[2] = {(float)t[i], (float)(t[i] - (double)(float)t[i])};
    std::memcpy(&t[n + i], pair, sizeof(pair));
  }
}

LevelGeom make_geom(int dim, int k, int n) {
  LevelGeom g;
  g.dim = dim;
  g.k = k;
  g.n = n;
  g.N = n * k + 1;
  g.py = (g.N + 3) / 4 * 4;
  g.pz = (long long)g.py * g.N;
  return g;
}

long long geom_elems(const LevelGeom& g) { return g.dim == 3 ? g.pz * g.N : (long long)g.py * g.N; }

bool valid_level(const gmg_problem* p, int level) {
  return p && level >= 0 && level < (int)p->levels.size();
}


// ---- typed dispatch helpers ----
int apply_level(gmg_problem* p, int level, const void* x, void* y, const void* bvec, double alpha,
                double beta) {
  PhaseScope ph(p, GMG_PHASE_OPERATOR);
  const Level& L = p->levels[level];
  if (p->varcoef) {
    if (p->esize == 8)
      return launch_apply_var<double>(L.g, L.n_elems, (const double*)x, (double*)y, (const double*)bvec,
                                      alpha, beta, (const double*)p->coef[level], p->stream);
    return launch_apply_var<float>(L.g, L.n_elems, (const float*)x, (float*)y, (const float*)bvec,
                                   alpha, beta, (const float*)p->coef[level], p->stream);
  }
  ApplyLaunch al;
  al.g = L.g;
  al.alpha = alpha;
  al.beta = beta;
  al.tile = p->apply_tile;
  if (p->esize == 8) {
    al.ws = p->op_ws();
    return launch_apply<double>(al, (const double*)x, (double*)y, (const double*)bvec, p->stream);
  }
  return launch_apply<float>(al, (const float*)x, (float*)y, (const float*)bvec, p->stream);
}

double op_scale(const Level& L) { return L.g.dim == 3 ? L.h : 1.0; }  // h^{d-2}

PatchLaunch colour_launch(const Level& L, int colour, double omega) {
  const int dim = L.g.dim, n = L.g.n;
  PatchLaunch pl;
  pl.g = L.g;
  pl.n_patches = 1;
  pl.plist = nullptr;
  pl.mode = 0;
  for (int a = 0; a < 3; ++a) {
    if (a < dim) {
      bool odd = (colour >> a) & 1;
      pl.first[a] = odd ? 1 : 2;
      pl.count[a] = odd ? n / 2 : (n - 1) / 2;
    } else {
      pl.first[a] = 1;
      pl.count[a] = 1;
    }
    pl.n_patches *= pl.count[a];
  }
  pl.sb = dim == 3 ? 1.0 / L.h : 1.0;
  pl.omega = omega;
  return pl;
}

int launch_colour(gmg_problem* p, const PatchLaunch& pl, void* u, const void* b) {
  if (pl.n_patches == 0) return GMG_OK;
  if (p->esize == 8) {
    if (pl.n_patches <= p->small_patches) {  // a coarse level: one output per thread
      const int st = launch_patch_small<double>(pl, (double*)u, (const double*)b, (const double*)p->dinv, p->stream);
      if (st != GMG_ERR_UNSUPPORTED) return st;
    }
    if (p->faces && p->shared_faces) {
      const int st = launch_patch_faces<double>(pl, (double*)u, (const double*)b, (const double*)p->dinv,
                                                (double*)p->faces, p->stream);
      if (st != GMG_ERR_UNSUPPORTED) return st;
    }
    return launch_patch_colour<double>(pl, (double*)u, (const double*)b, (const double*)p->dinv, p->stream);
  }
  const int pr = p->desc.precision;
  if (pr == GMG_FP32 && p->faces && p->shared_faces) {
    const int st = launch_patch_faces<float>(pl, (float*)u, (const float*)b, (const float*)p->dinv,
                                             (float*)p->faces, p->stream);
    if (st != GMG_ERR_UNSUPPORTED) return st;
  }
  if ((pr == GMG_FP32_TC || pr == GMG_FP32_TF32) && pl.mode == 0 && tc_supported(pl.g.dim, pl.g.k))
    return launch_patch_tc(pl, (float*)u, (const float*)b, (const float*)p->dinv, pr == GMG_FP32_TC, p->stream);
  return launch_patch_colour<float>(pl, (float*)u, (const float*)b, (const float*)p->dinv, p->stream);
}

int smooth_colour(gmg_problem* p, int level, void* u, const void* b, int colour) {
  const PatchLaunch pl = colour_launch(p->levels[level], colour, p->desc.damping);
  if (p->varcoef) {
    if (pl.n_patches == 0) return GMG_OK;
    const float* corr =
        p->local_solver == GMG_LOCAL_LEARNED && ((p->corr_levels >> level) & 1u) ? p->corr[level] : nullptr;
    if (p->esize == 8)
      return launch_patch_var<double>(pl, (double*)u, (const double*)b, (const double*)p->coef[level],
                                      (const double*)p->vscale[level], (const double*)p->dinv, corr, p->corr_rank, p->stream);
    return launch_patch_var<float>(pl, (float*)u, (const float*)b, (const float*)p->coef[level],
                                   (const float*)p->vscale[level], (const float*)p->dinv, corr, p->corr_rank, p->stream);
  }
  return launch_colour(p, pl, u, b);
}

// Skewed-slab schedule (the GPU form of the locality-ordered batches of
// Sec. 4.1): the patch at vertex v of colour c, at position o in the colour
// order (o = c forward, n_colours - 1 - c in reverse), belongs to slab
// floor((v_s + o) / W), v_s its vertex index along the slowest axis.  Slabs
// run in order and colour positions in order inside a slab.  A patch that
// overlaps a patch of an earlier position (|v - v'|_inf <= 1) never lands in
// an earlier slab, and patches of one colour do not interact, so every patch
// reads exactly the values Algorithm 4 gives it: the sweep does not depend
// on W.  Only the working set between consecutive launches changes: about
// (W + 2) k node planes of u and b.
// Largest number of patches in one colour of level L.
long long max_colour_patches(const gmg_problem* p, const Level& L) {
  long long m = 0;
  for (int c = 0; c < (1 << L.g.dim); ++c) m = std::max<long long>(m, colour_launch(L, c, p->desc.damping).n_patches);
  return m;
}

// FP64 levels whose colours all take the coarse-level kernel (gmg_set_small_sweep)
bool small_level(const gmg_problem* p, const Level& L) {
  return p->esize == 8 && !p->varcoef && max_colour_patches(p, L) <= p->small_patches;
}

int slab_width_for(const gmg_problem* p, const Level& L) {
  // a small FP64 level is swept by the coarse-level kernel, one CTA per patch
  if (p->varcoef || p->slab_width == 0 || small_level(p, L)) return 0;
  const int nc = 1 << L.g.dim, span = L.g.n - 1 + nc;  // slab index range at W = 1
  int W = p->slab_width;
  if (W < 0) {  // the largest slab whose node planes of u and b fill half of the 126 MB L2
    const long long plane = (L.g.dim == 3 ? L.g.pz : (long long)L.g.py) * (long long)p->esize * 2;
    W = (int)std::max<long long>(1, (63ll << 20) / std::max<long long>(plane * L.g.k, 1) - 2);
  }
  return W >= span ? 0 : W;
}

int build_slabs(gmg_problem* p, int level, int W) {
  Level& L = p->levels[level];
  if (L.slab_w == W) return GMG_OK;
  for (int d = 0; d < 2; ++d) {
    if (L.slist[d]) {
      cudaFree(L.slist[d]);
      p->owned.erase(std::find(p->owned.begin(), p->owned.end(), (void*)L.slist[d]));
      L.slist[d] = nullptr;
    }
    L.soff[d].clear();
  }
  L.slab_w = 0;
  if (W <= 0) return GMG_OK;
  const int dim = L.g.dim, nc = 1 << dim, slow = dim - 1;
  const int nslab = (L.g.n - 1 + nc - 1) / W + 1;
  for (int d = 0; d < 2; ++d) {
    std::vector<std::vector<int>> bucket((size_t)nslab * nc);
    for (int c = 0; c < nc; ++c) {
      const int o = d == 0 ? c : nc - 1 - c;
      const PatchLaunch pl = colour_launch(L, c, 1.0);
      for (int pid = 0; pid < pl.n_patches; ++pid) {
        int rest = pid, v[3] = {0, 0, 0};
        for (int a = 0; a < dim; ++a) {
          v[a] = pl.first[a] + 2 * (rest % pl.count[a]);
          rest /= pl.count[a];
        }
        bucket[(size_t)((v[slow] + o) / W) * nc + o].push_back(pid);
      }
    }
    std::vector<int> flat;
    L.soff[d].assign(1, 0);
    for (const auto& bk : bucket) {
      flat.insert(flat.end(), bk.begin(), bk.end());
      L.soff[d].push_back((int)flat.size());
    }
    void* dptr = nullptr;
    CHECK(dalloc(p, &dptr, std::max<size_t>(flat.size(), 1) * sizeof(int)));
    L.slist[d] = static_cast<int*>(dptr);
    if (!flat.empty() &&
        cudaMemcpy(dptr, flat.data(), flat.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess)
      return GMG_ERR_CUDA;
  }
  L.slab_w = W;
  return GMG_OK;
}

int smooth(gmg_problem* p, int level, void* u, const void* b, int n_sweeps, int reverse) {
  PhaseScope ph(p, GMG_PHASE_SMOOTH);
  Level& L = p->levels[level];
  const int nc = 1 << L.g.dim;
  if (L.slab_w > 0 && !p->varcoef) {
    const int d = reverse ? 1 : 0;
    const int nslab = (int)(L.soff[d].size() - 1) / nc;
    for (int sw = 0; sw < n_sweeps; ++sw)
      for (int s = 0; s < nslab; ++s)
        for (int o = 0; o < nc; ++o) {
          const int lo = L.soff[d][s * nc + o], cnt = L.soff[d][s * nc + o + 1] - lo;
          if (cnt == 0) continue;
          PatchLaunch pl = colour_launch(L, d ? nc - 1 - o : o, p->desc.damping);
          pl.plist = L.slist[d] + lo;
          pl.n_patches = cnt;
          CHECK(launch_colour(p, pl, u, b));
        }
    return GMG_OK;
  }
  for (int s = 0; s < n_sweeps; ++s)
    for (int i = 0; i < nc; ++i) CHECK(smooth_colour(p, level, u, b, reverse ? nc - 1 - i : i));
  return GMG_OK;
}

// Z-curve (Morton) key of a vertex: bits of v_0, v_1 (, v_2) interleaved,
// v_0 lowest (Sec. 4.1 step 1).
unsigned long long morton(int dim, const int v[3]) {
  unsigned long long key = 0;
  for (int bit = 0; bit < 20; ++bit)
    for (int a = 0; a < dim; ++a)
      key |= (unsigned long long)((v[a] >> bit) & 1) << (dim * bit + a);
  return key;
}

// Patches of every colour sorted along the Z-curve (Sec. 4.1 steps 1-2),
// as lexicographic ids within the colour; built once per level.
int build_zlists(gmg_problem* p, int level) {
  Level& L = p->levels[level];
  if (L.zlist) return GMG_OK;
  const int nc = 1 << L.g.dim;
  std::vector<int> all;
  for (int c = 0; c < nc; ++c) {
    PatchLaunch pl = colour_launch(L, c, 1.0);
    std::vector<std::pair<unsigned long long, int>> keyed(pl.n_patches);
    for (int pid = 0; pid < pl.n_patches; ++pid) {
      int rest = pid, v[3] = {0, 0, 0};
      for (int a = 0; a < L.g.dim; ++a) {
        v[a] = pl.first[a] + 2 * (rest % pl.count[a]);
        rest /= pl.count[a];
      }
      keyed[pid] = {morton(L.g.dim, v), pid};
    }
    std::stable_sort(keyed.begin(), keyed.end(),
                     [](const auto& x, const auto& y) { return x.first < y.first; });
    L.zoff[c] = (int)all.size();
    for (const auto& kv : keyed) all.push_back(kv.second);
  }
  L.zoff[nc] = (int)all.size();
  void* d = nullptr;
  CHECK(dalloc(p, &d, std::max<size_t>(all.size(), 1) * sizeof(int)));
  if (!all.empty() &&
      cudaMemcpy(d, all.data(), all.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess)
    return GMG_ERR_CUDA;
  L.zlist = static_cast<int*>(d);
  return GMG_OK;
}

// Algorithm 3: per colour, r = b - A u on the whole level, then the local
// solves of the colour from r (solve-only kernel mode).
int smooth_separated(gmg_problem* p, int level, void* u, const void* b, int reverse) {
  Level& L = p->levels[level];
  const int nc = 1 << L.g.dim;
  for (int i = 0; i < nc; ++i) {
    const int c = reverse ? nc - 1 - i : i;
    CHECK(apply_level(p, level, u, L.r, b, -op_scale(L), 1.0));
    PatchLaunch pl = colour_launch(L, c, p->desc.damping);
    pl.mode = 1;
    CHECK(launch_colour(p, pl, u, L.r));
  }
  return GMG_OK;
}

// Algorithm 5: batches of n_b patches per colour in Z-curve order; for each
// batch index, every colour's batch in turn.
int smooth_batched(gmg_problem* p, int level, void* u, const void* b, long long n_b, int reverse) {
  CHECK(build_zlists(p, level));
  Level& L = p->levels[level];
  const int nc = 1 << L.g.dim;
  long long nbatch = 0;
  for (int c = 0; c < nc; ++c)
    nbatch = std::max(nbatch, ((long long)(L.zoff[c + 1] - L.zoff[c]) + n_b - 1) / n_b);
  for (long long bi = 0; bi < nbatch; ++bi) {
    const long long bb = reverse ? nbatch - 1 - bi : bi;
    for (int i = 0; i < nc; ++i) {
      const int c = reverse ? nc - 1 - i : i;
      const long long size = L.zoff[c + 1] - L.zoff[c];
      const long long s0 = bb * n_b, s1 = std::min(size, s0 + n_b);
      if (s0 >= s1) continue;
      PatchLaunch pl = colour_launch(L, c, p->desc.damping);
      pl.plist = L.zlist + L.zoff[c] + s0;
      pl.n_patches = (int)(s1 - s0);
      CHECK(launch_colour(p, pl, u, b));
    }
  }
  return GMG_OK;
}

int axis_op(gmg_problem* p, const AxisOp& op, const void* in, void* out, const void* coef) {
  if (p->esize == 8) return launch_axis_op<double>(op, (const double*)in, (double*)out, (const double*)coef, p->stream);
  return launch_axis_op<float>(op, (const float*)in, (float*)out, (const float*)coef, p->stream);
}

// Describe a dense array of extents e[3] (x fastest) with given strides.
struct Arr {
  int e[3];
  long long s[3];
};
Arr level_arr(const LevelGeom& g) {
  Arr a;
  a.e[0] = g.N; a.e[1] = g.N; a.e[2] = g.dim == 3 ? g.N : 1;
  a.s[0] = 1; a.s[1] = g.py; a.s[2] = g.dim == 3 ? g.pz : 0;
  return a;
}
Arr compact_arr(int e0, int e1, int e2) {
  Arr a;
  a.e[0] = e0; a.e[1] = e1; a.e[2] = e2;
  a.s[0] = 1; a.s[1] = e0; a.s[2] = (long long)e0 * e1;
  return a;
}

// One pass along `axis`: computes cnt[] outputs at out_off[] from `in`.
AxisOp make_op(int axis, const Arr& in, const int in_off[3], const Arr& out, const int cnt[3],
               const int out_off[3], int R, int S, int off, int W, int acc) {
  AxisOp op;
  op.axis = axis;
  for (int a = 0; a < 3; ++a) {
    op.cnt[a] = cnt[a];
    op.in_dim[a] = in.e[a];
    op.in_stride[a] = in.s[a];
    op.in_off[a] = in_off[a];
    op.out_stride[a] = out.s[a];
    op.out_off[a] = out_off[a];
  }
  op.R = R; op.S = S; op.off = off; op.W = W;
  op.shift = 0;
  op.accumulate = acc;
  return op;
}

// fine += P coarse (tensor product of the 1D embedding, one axis per pass)
int prolongate_add(gmg_problem* p, int cl, const void* coarse, void* fine) {
  PhaseScope ph(p, GMG_PHASE_TRANSFER);
  const LevelGeom& gc = p->levels[cl].g;
  const LevelGeom& gf = p->levels[cl + 1].g;
  const int k = gc.k, dim = gc.dim, Nc = gc.N, Nf = gf.N;
  const int zero[3] = {0, 0, 0};
  Arr cur = level_arr(gc);
  const void* src = coarse;
  int ext[3] = {Nc, Nc, dim == 3 ? Nc : 1};
  for (int a = 0; a < dim; ++a) {
    ext[a] = Nf;
    const bool last = (a == dim - 1);
    Arr out = last ? level_arr(gf) : compact_arr(ext[0], ext[1], ext[2]);
    void* dst = last ? fine : (a % 2 == 0 ? p->tmp1 : p->tmp2);
    AxisOp op = make_op(a, cur, zero, out, ext, zero, 2 * k, k, 0, k + 1, last ? 1 : 0);
    if (p->xfer_df)  // FP64 problems: double-float passes, float pairs in between
      CHECK(launch_transfer_df(op, k, gc.n, false, p->prol_h.data(), src, a > 0, dst, !last, p->stream));
    else
      CHECK(axis_op(p, op, src, dst, p->coef_prol));
    cur = out;
    src = dst;
  }
  return GMG_OK;
}

// coarse = P^T fine on the interior coarse nodes (Dirichlet ones stay zero):
// one axis per pass; along axes already restricted only interior coarse
// nodes are computed, stored at their lattice index.
int restrict_to(gmg_problem* p, int fl, const void* fine, void* coarse) {
  PhaseScope ph(p, GMG_PHASE_TRANSFER);
  const LevelGeom& gf = p->levels[fl].g;
  const LevelGeom& gc = p->levels[fl - 1].g;
  const int k = gc.k, dim = gc.dim, Nc = gc.N, Nf = gf.N;
  Arr cur = level_arr(gf);
  const void* src = fine;
  int ext[3] = {Nf, Nf, dim == 3 ? Nf : 1};
  for (int a = 0; a < dim; ++a) {
    int store[3] = {ext[0], ext[1], ext[2]};
    store[a] = Nc;
    int cnt[3], ooff[3], ioff[3];
    for (int b2 = 0; b2 < 3; ++b2) {
      const bool restricted = b2 < dim && b2 <= a;
      cnt[b2] = restricted ? Nc - 2 : store[b2];
      ooff[b2] = restricted ? 1 : 0;
      ioff[b2] = (b2 < dim && b2 < a) ? 1 : 0;
    }
    const bool last = (a == dim - 1);
    Arr out = last ? level_arr(gc) : compact_arr(store[0], store[1], store[2]);
    void* dst = last ? coarse : (a % 2 == 0 ? p->tmp1 : p->tmp2);
    // coarse node c = o + 1 gathers fine nodes 2k(c/k) - (2k-1) .. + (2k-1)
    AxisOp op = make_op(a, cur, ioff, out, cnt, ooff, k, 2 * k, -(2 * k - 1), 4 * k - 1, 0);
    op.shift = 1;
    if (p->xfer_df)
      CHECK(launch_transfer_df(op, k, gc.n, true, p->rest_h.data(), src, a > 0, dst, !last, p->stream));
    else
      CHECK(axis_op(p, op, src, dst, p->coef_rest));
    cur = out;
    src = dst;
    ext[a] = Nc;
  }
  return GMG_OK;
}

// Exact coarsest-level solve of the constant-coefficient problem by global
// fast diagonalisation (App. A.3 applied to the whole level): x = (T..T)
// diag(h^{2-d} / sum lambda) (T..T)^T b on the interior, in element type E.
template <typename E>
int coarse_fd(gmg_problem* p, const void* b, void* x, const void* fwd, const void* bwd, const void* dinv,
              void* t1, void* t2) {
  const LevelGeom& g = p->levels[0].g;
  const int dim = g.dim, m = p->m0;
  const int zero[3] = {0, 0, 0};
  const int one[3] = {1, 1, dim == 3 ? 1 : 0};
  int cnt[3] = {m, m, dim == 3 ? m : 1};
  Arr lev = level_arr(g);
  Arr cmp = compact_arr(m, m, dim == 3 ? m : 1);
  // forward: t = (T^T x .. x T^T) b on the interior
  const void* src = b;
  Arr cur = lev;
  for (int a = 0; a < dim; ++a) {
    const bool first = (a == 0);
    void* dst = (a % 2 == 0) ? t1 : t2;
    int in_off[3];
    for (int b2 = 0; b2 < 3; ++b2) in_off[b2] = first ? one[b2] : 0;
    AxisOp op = make_op(a, cur, in_off, cmp, cnt, zero, m, 0, first ? 1 : 0, m, 0);
    CHECK(launch_axis_op<E>(op, (const E*)src, (E*)dst, (const E*)fwd, p->stream));
    cur = cmp;
    src = dst;
  }
  long long nm = (long long)m * m * (dim == 3 ? m : 1);
  CHECK(launch_scale<E>(nm, (E*)src, (const E*)dinv, p->stream));
  // backward: x = (T x .. x T) t into the level interior
  for (int a = 0; a < dim; ++a) {
    const bool last = (a == dim - 1);
    void* dst = last ? x : (src == t1 ? t2 : t1);
    Arr out = last ? lev : cmp;
    const int* ooff = last ? one : zero;
    AxisOp op = make_op(a, cur, zero, out, cnt, ooff, m, 0, 0, m, 0);
    CHECK(launch_axis_op<E>(op, (const E*)src, (E*)dst, (const E*)bwd, p->stream));
    src = dst;
  }
  return GMG_OK;
}

int coarse_solve(gmg_problem* p, const void* b, void* x) {
  PhaseScope ph(p, GMG_PHASE_COARSE);
  const LevelGeom& g = p->levels[0].g;
  if (p->varcoef) {
    if (p->esize == 8)
      return launch_dense_solve<double>(g, p->coarse_inv, p->coarse_n, (const double*)b, (double*)x, p->stream);
    return launch_dense_solve<float>(g, p->coarse_inv, p->coarse_n, (const float*)b, (float*)x, p->stream);
  }
  if (p->esize == 4) {  // single-precision problem: the coarse solve runs in FP64
    const long long n0 = p->levels[0].n_elems;
    CHECK(launch_convert_f32_f64(n0, (const float*)b, (double*)p->c64_b, p->stream));
    CHECK(coarse_fd<double>(p, p->c64_b, p->c64_x, p->c64_fwd, p->c64_bwd, p->c64_dinv, p->c64_t1, p->c64_t2));
    return launch_convert_f64_f32(n0, (const double*)p->c64_x, (float*)x, p->stream);
  }
  return coarse_fd<double>(p, b, x, p->coef_c_fwd, p->coef_c_bwd, p->dinv0, p->ctmp1, p->ctmp2);
}

int vcycle_level(gmg_problem* p, int l, void* x, const void* b) {
  Level& L = p->levels[l];
  if (l == 0) return coarse_solve(p, b, x);
  {
    PhaseScope ph(p, GMG_PHASE_VECTOR);
    if (cudaMemsetAsync(x, 0, L.n_elems * p->esize, p->stream) != cudaSuccess) return GMG_ERR_CUDA;
  }
  CHECK(smooth(p, l, x, b, p->desc.pre_sweeps, 0));
  CHECK(apply_level(p, l, x, L.r, b, -op_scale(L), 1.0));
  Level& C = p->levels[l - 1];
  CHECK(restrict_to(p, l, L.r, C.b));
  CHECK(vcycle_level(p, l - 1, C.u, C.b));
  CHECK(prolongate_add(p, l - 1, C.u, x));
  CHECK(smooth(p, l, x, b, p->desc.post_sweeps, 1));
  return GMG_OK;
}

}  // namespace detail
}  // namespace gmg

using namespace gmg::detail;

extern "C" {

long long gmg_kernel_launch_count(void) { return launch_count(); }

const char* gmg_status_string(int s) {
  switch (s) {
    case GMG_OK: return "ok";
    case GMG_ERR_INVALID_ARG: return "invalid argument";
    case GMG_ERR_OOM: return "device out of memory";
    case GMG_ERR_CUDA: return "CUDA error";
    case GMG_ERR_NONFINITE: return "non-finite value in solver";
    case GMG_ERR_BREAKDOWN: return "CG breakdown";
    case GMG_ERR_NOT_CONVERGED: return "not converged";
    case GMG_ERR_UNSUPPORTED: return "unsupported";
    case GMG_ERR_TIMEOUT: return "device wait timed out";
    default: return "unknown status";
  }
}

int gmg_patch_fd_1d(int k, double* M, double* K, double* T, double* lambda) {
  if (k < 1 || k > kMaxDegree) return GMG_ERR_INVALID_ARG;
  const int m = 2 * k - 1;
  std::vector<double> Mi, Ki, Ti, li;
  assembled_1d(k, 2, 1, m, 1, m, Mi, Ki);
  if (!generalized_eigen_mirror(m, Mi, Ki, Ti, li)) return GMG_ERR_INVALID_ARG;
  if (M) std::memcpy(M, Mi.data(), sizeof(double) * m * m);
  if (K) std::memcpy(K, Ki.data(), sizeof(double) * m * m);
  if (T) std::memcpy(T, Ti.data(), sizeof(double) * m * m);
  if (lambda) std::memcpy(lambda, li.data(), sizeof(double) * m);
  return GMG_OK;
}

int gmg_destroy(gmg_problem* p) {
  if (!p) return GMG_OK;
  cudaStreamSynchronize(p->stream);
  drop_cg_graph(p);
  release_phase_events(p);
  if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
  for (void* ptr : p->owned) cudaFree(ptr);
  delete p;
  return GMG_OK;
}

}  // extern "C"

int gmg::detail::create_problem(const gmg_desc* d, gmg_problem* p, const CreateOptions& opt) {
  p->desc = *d;
  p->stream = (cudaStream_t)d->stream;
  p->esize = d->precision == GMG_FP64 ? 8 : 4;
  if (!device_wait_flag()) return GMG_ERR_CUDA;  // resolved once, outside any graph capture
  const int dim = d->dim, k = d->degree;
  // colour steps of up to 256 patches take the one-output-per-thread kernel
  // at k <= 4, where it measured faster than the line kernels; above, a
  // patch's outputs outnumber a CTA's threads and it measured slower
  p->small_patches = k <= 4 ? 256 : 0;
  // level hierarchy: n_levels given, or halve while even and >= 2
  int L = d->n_levels;
  if (L == 0) {
    L = 1;
    int n = d->n_cells;
    while (n % 2 == 0 && n / 2 >= 2) { n /= 2; ++L; }
  }
  for (int l = 0; l < L; ++l) {
    int shift = L - 1 - l;
    int n = d->n_cells >> shift;
    if (n < 1 || (n << shift) != d->n_cells) return GMG_ERR_INVALID_ARG;
    if (l > 0 && n < 2) return GMG_ERR_INVALID_ARG;
  }
  if ((d->n_cells >> (L - 1)) < 1) return GMG_ERR_INVALID_ARG;
  p->levels.resize(L);
  for (int l = 0; l < L; ++l) {
    Level& lv = p->levels[l];
    int n = d->n_cells >> (L - 1 - l);
    lv.g = make_geom(dim, k, n);
    lv.n_elems = geom_elems(lv.g);
    lv.h = 1.0 / n;
    if (l == L - 1 && opt.finest_u) {
      p->finest_borrowed = true;
      lv.u = opt.finest_u;
      lv.b = opt.finest_b;
      lv.r = opt.finest_r;
      continue;
    }
    CHECK(dalloc(p, &lv.u, lv.n_elems * p->esize));
    CHECK(dalloc(p, &lv.b, lv.n_elems * p->esize));
    CHECK(dalloc(p, &lv.r, lv.n_elems * p->esize));
  }
  // 1D tables: unit cell, two-cell patch (interior rows x closure cols), FD
  const int m = 2 * k - 1, C = 2 * k + 1;
  std::vector<double> Mc, Kc, Mp, Kp, Mi, Ki, Tp, lp;
  cell_matrices_1d(k, Mc, Kc);
  assembled_1d(k, 2, 1, m, 0, C, Mp, Kp);
  assembled_1d(k, 2, 1, m, 1, m, Mi, Ki);
  if (!generalized_eigen_mirror(m, Mi, Ki, Tp, lp)) return GMG_ERR_INVALID_ARG;
  CHECK(upload_patch_tables<double>(k, Mp.data(), Kp.data(), Tp.data(), Mc.data(), Kc.data(), p->stream));
  CHECK(upload_patch_tables<float>(k, Mp.data(), Kp.data(), Tp.data(), Mc.data(), Kc.data(), p->stream));
  if (d->precision == GMG_FP32_TC || d->precision == GMG_FP32_TF32)
    CHECK(upload_tc_tables(k, Mp.data(), Kp.data(), Tp.data()));
  const int nint = dim == 3 ? m * m * m : m * m;
  std::vector<double> dinv(nint);
  for (int t = 0; t < nint; ++t) {
    int x = t % m, y = (t / m) % m, z = t / (m * m);
    double s = lp[x] + lp[y] + (dim == 3 ? lp[z] : 0.0);
    dinv[t] = 1.0 / s;
  }
  // FP64 problems: the table is followed by its float-pair split, read by
  // the shared-face sweep's double-float FD transforms
  if (p->esize == 8) append_float_pairs(dinv);
  CHECK(upload_table(p, &p->dinv, dinv));
  // face buffer of the shared-face sweep: the largest colour of the finest
  // level; without memory for it the closure form is used.  FP64 problems
  // use the form from k = 3 (the sweep is bound by FP64 instructions, which
  // it cuts by a third); FP32 ones from k = 7: at k = 3, 4 the FP32 closure
  // kernel is faster (it is bound by issue and latency, and the face pass
  // adds a launch and its traffic per colour), at k = 7 the form is 11 %
  // faster.  The tensor-core precisions keep their kernel.
  const bool faces_form = d->precision == GMG_FP64 ? k >= 3 : d->precision == GMG_FP32 && k >= 7;
  if (faces_form && dim == 3 && !opt.no_faces) {
    long long fe = 0;
    for (int c = 0; c < (1 << dim); ++c) {
      const PatchLaunch pl = colour_launch(p->levels[L - 1], c, d->damping);
      fe = std::max(fe, p->esize == 8 ? face_buffer_elems<double>(pl) : face_buffer_elems<float>(pl));
    }
    if (fe > 0 && dalloc(p, &p->faces, fe * p->esize) != GMG_OK) p->faces = nullptr;
  }
  // workspace of the three-pass FP64 operator (also used by the FP64 CG of
  // single-precision problems): four finest-level vectors; without memory
  // for it the tile kernel is used
  if (staged_apply_preferred(dim, k) && !opt.no_faces &&
      dalloc(p, &p->apply_ws, 4 * p->levels[L - 1].n_elems * 8) != GMG_OK)
    p->apply_ws = nullptr;
  // transfer tables
  std::vector<double> P1;
  prolongation_cell_1d(k, P1);  // (2k+1) x (k+1)
  std::vector<double> prol(2 * k * (k + 1));
  for (int r = 0; r < 2 * k; ++r)
    for (int q = 0; q <= k; ++q) prol[r * (k + 1) + q] = P1[r * (k + 1) + q];
  CHECK(upload_table(p, &p->coef_prol, prol));
  const int W = 4 * k - 1;
  std::vector<double> rest(k * W, 0.0);
  for (int q = 0; q < k; ++q)
    for (int w = 0; w < W; ++w) {
      int dd = w - (2 * k - 1);  // fine offset from 2 k cc
      double v = 0.0;
      if (q == 0) {
        if (dd < 0) v = P1[(2 * k + dd) * (k + 1) + k];
        else if (dd == 0) v = 1.0;
        else v = P1[dd * (k + 1) + 0];
      } else if (dd >= 1 && dd <= 2 * k - 1) {
        v = P1[dd * (k + 1) + q];
      }
      rest[q * W + w] = v;
    }
  CHECK(upload_table(p, &p->coef_rest, rest));
  p->prol_h = prol;
  p->rest_h = rest;
  p->xfer_df = p->esize == 8 && transfer_table_df_ok(k, false, prol.data()) &&
               transfer_table_df_ok(k, true, rest.data());
  // transfer temporaries: largest intermediate array of any pass
  long long tmax = 1;
  for (int l = 1; l < L; ++l) {
    long long Nf = p->levels[l].g.N, Nc = p->levels[l - 1].g.N;
    long long t = dim == 3 ? Nf * Nf * Nc : Nf * Nc;
    if (t > tmax) tmax = t;
  }
  CHECK(dalloc(p, &p->tmp1, tmax * p->esize));
  CHECK(dalloc(p, &p->tmp2, tmax * p->esize));
  // coarsest level: global fast diagonalisation
  const LevelGeom& g0 = p->levels[0].g;
  const int m0 = g0.n * k - 1;
  p->m0 = m0;
  if (m0 < 1) return GMG_ERR_INVALID_ARG;
  std::vector<double> M0, K0, T0, l0;
  assembled_1d(k, g0.n, 1, m0, 1, m0, M0, K0);
  if (!generalized_eigen(m0, M0, K0, T0, l0)) return GMG_ERR_INVALID_ARG;
  std::vector<double> fwd(m0 * m0), bwd(m0 * m0);
  for (int i = 0; i < m0; ++i)
    for (int j = 0; j < m0; ++j) {
      fwd[i * m0 + j] = T0[j * m0 + i];
      bwd[i * m0 + j] = T0[i * m0 + j];
    }
  CHECK(upload_table(p, &p->coef_c_fwd, fwd));
  CHECK(upload_table(p, &p->coef_c_bwd, bwd));
  const long long nm0 = (long long)m0 * m0 * (dim == 3 ? m0 : 1);
  std::vector<double> d0(nm0);
  const double s0 = dim == 3 ? (double)g0.n : 1.0;  // h0^{2-d}
  for (long long t = 0; t < nm0; ++t) {
    int x = t % m0, y = (t / m0) % m0, z = (int)(t / ((long long)m0 * m0));
    d0[t] = s0 / (l0[x] + l0[y] + (dim == 3 ? l0[z] : 0.0));
  }
  CHECK(upload_table(p, &p->dinv0, d0));
  CHECK(dalloc(p, &p->ctmp1, nm0 * p->esize));
  CHECK(dalloc(p, &p->ctmp2, nm0 * p->esize));
  if (p->esize == 4) {  // FP64 coarse solve of single-precision problems
    const size_t es = p->esize;
    p->esize = 8;
    int st = upload_table(p, &p->c64_fwd, fwd);
    if (st == GMG_OK) st = upload_table(p, &p->c64_bwd, bwd);
    if (st == GMG_OK) st = upload_table(p, &p->c64_dinv, d0);
    p->esize = es;
    CHECK(st);
    CHECK(dalloc(p, &p->c64_t1, nm0 * 8));
    CHECK(dalloc(p, &p->c64_t2, nm0 * 8));
    CHECK(dalloc(p, &p->c64_b, p->levels[0].n_elems * 8));
    CHECK(dalloc(p, &p->c64_x, p->levels[0].n_elems * 8));
  }
  // outer CG
  if (opt.no_cg) return cudaDeviceSynchronize() == cudaSuccess ? GMG_OK : GMG_ERR_CUDA;
  const long long nf = p->levels[L - 1].n_elems;
  CHECK(dalloc(p, (void**)&p->cg_r, nf * 8));
  CHECK(dalloc(p, (void**)&p->cg_z, nf * 8));
  CHECK(dalloc(p, (void**)&p->cg_p, nf * 8));
  CHECK(dalloc(p, (void**)&p->cg_q, nf * 8));
  CHECK(dalloc(p, (void**)&p->partial, kReduceBlocks * 8));
  CHECK(dalloc(p, (void**)&p->scal, S_COUNT * 8));
  return cudaDeviceSynchronize() == cudaSuccess ? GMG_OK : GMG_ERR_CUDA;
}

int gmg::detail::check_desc(const gmg_desc* d) {
  if (!d) return GMG_ERR_INVALID_ARG;
  if (d->dim != 2 && d->dim != 3) return GMG_ERR_INVALID_ARG;
  if (d->degree < 1 || d->degree > kMaxDegree) return GMG_ERR_INVALID_ARG;
  if (d->n_cells < 2 || d->n_levels < 0 || d->n_levels > 30) return GMG_ERR_INVALID_ARG;
  if (d->precision < GMG_FP64 || d->precision > GMG_FP32_TF32) return GMG_ERR_INVALID_ARG;
  if (!std::isfinite(d->damping) || d->pre_sweeps < 0 || d->post_sweeps < 0) return GMG_ERR_INVALID_ARG;
  // node counts must fit 32-bit lattice indices
  if ((long long)d->n_cells * d->degree + 1 > (1 << 20)) return GMG_ERR_INVALID_ARG;
  return GMG_OK;
}

extern "C" {

int gmg_create(const gmg_desc* d, gmg_problem** out) {
  if (!out) return GMG_ERR_INVALID_ARG;
  *out = nullptr;
  if (check_desc(d) != GMG_OK) return GMG_ERR_INVALID_ARG;
  gmg_problem* p = new (std::nothrow) gmg_problem();
  if (!p) return GMG_ERR_OOM;
  int st = create_problem(d, p, CreateOptions());
  if (st != GMG_OK) {
    gmg_destroy(p);
    return st;
  }
  *out = p;
  return GMG_OK;
}

int gmg_vector_layout(const gmg_problem* p, int level, long long* n_elems, int* nodes_1d,
                      int* pitch_y, long long* pitch_z) {
  if (!valid_level(p, level)) return GMG_ERR_INVALID_ARG;
  const Level& L = p->levels[level];
  if (n_elems) *n_elems = L.n_elems;
  if (nodes_1d) *nodes_1d = L.g.N;
  if (pitch_y) *pitch_y = L.g.py;
  if (pitch_z) *pitch_z = L.g.dim == 3 ? L.g.pz : 0;
  return GMG_OK;
}

int gmg_level_info(const gmg_problem* p, int level, int* n_cells, int* n_levels) {
  if (!valid_level(p, level)) return GMG_ERR_INVALID_ARG;
  if (n_cells) *n_cells = p->levels[level].g.n;
  if (n_levels) *n_levels = (int)p->levels.size();
  return GMG_OK;
}

int gmg_apply_operator(gmg_problem* p, int level, const void* x, void* y) {
  if (!valid_level(p, level) || !x || !y || x == y) return GMG_ERR_INVALID_ARG;
  return apply_level(p, level, x, y, nullptr, op_scale(p->levels[level]), 0.0);
}

int gmg_apply_operator_f64(gmg_problem* p, int level, const double* x, double* y) {
  if (!valid_level(p, level) || !x || !y || x == y) return GMG_ERR_INVALID_ARG;
  const Level& L = p->levels[level];
  if (p->varcoef) {
    if (level != (int)p->levels.size() - 1 || !p->coef64) return GMG_ERR_UNSUPPORTED;
    return launch_apply_var<double>(L.g, L.n_elems, x, y, nullptr, op_scale(L), 0.0, p->coef64, p->stream);
  }
  ApplyLaunch al;
  al.g = L.g;
  al.alpha = op_scale(L);
  al.beta = 0.0;
  al.ws = p->op_ws();
  al.tile = p->apply_tile;
  return launch_apply<double>(al, x, y, nullptr, p->stream);
}

int gmg_smooth(gmg_problem* p, int level, void* u, const void* b, int n_sweeps, int reverse) {
  if (!valid_level(p, level) || !u || !b || u == b || n_sweeps < 0) return GMG_ERR_INVALID_ARG;
  return smooth(p, level, u, b, n_sweeps, reverse);
}

int gmg_smooth_colour(gmg_problem* p, int level, void* u, const void* b, int colour) {
  if (!valid_level(p, level) || !u || !b || u == b) return GMG_ERR_INVALID_ARG;
  if (colour < 0 || colour >= (1 << p->levels[level].g.dim)) return GMG_ERR_INVALID_ARG;
  return smooth_colour(p, level, u, b, colour);
}

int gmg_set_coefficient(gmg_problem* p, const double* coef) {
  if (!p || !coef) return GMG_ERR_INVALID_ARG;
  drop_cg_graph(p);
  const int dim = p->desc.dim, k = p->desc.degree, L = (int)p->levels.size();
  if (k > 3) return GMG_ERR_UNSUPPORTED;
  const long long nfine = dim == 3 ? (long long)p->desc.n_cells * p->desc.n_cells * p->desc.n_cells
                                   : (long long)p->desc.n_cells * p->desc.n_cells;
  for (long long c = 0; c < nfine; ++c)
    if (!(coef[c] > 0.0) || !std::isfinite(coef[c])) return GMG_ERR_INVALID_ARG;
  // per-level coefficients: geometric mean of the 2^d children
  std::vector<std::vector<double>> lev(L);
  lev[L - 1].assign(coef, coef + nfine);
  for (int l = L - 2; l >= 0; --l) {
    const int n = p->levels[l].g.n, nf = p->levels[l + 1].g.n;
    const long long nc = dim == 3 ? (long long)n * n * n : (long long)n * n;
    lev[l].assign(nc, 0.0);
    for (long long c = 0; c < nc; ++c) {
      const int cx = (int)(c % n), cy = (int)((c / n) % n), cz = dim == 3 ? (int)(c / ((long long)n * n)) : 0;
      double lg = 0.0;
      for (int o = 0; o < (1 << dim); ++o) {
        const int fx = 2 * cx + (o & 1), fy = 2 * cy + ((o >> 1) & 1), fz = dim == 3 ? 2 * cz + ((o >> 2) & 1) : 0;
        lg += std::log(lev[l + 1][fx + (long long)nf * (fy + (long long)nf * fz)]);
      }
      lev[l][c] = std::exp(lg / (1 << dim));
    }
  }
  // tables of the variable-coefficient kernels (unit cell, mirror FD)
  const int m = 2 * k - 1;
  std::vector<double> Mc, Kc, Mi, Ki, Tp, lp;
  cell_matrices_1d(k, Mc, Kc);
  assembled_1d(k, 2, 1, m, 1, m, Mi, Ki);
  if (!generalized_eigen_mirror(m, Mi, Ki, Tp, lp)) return GMG_ERR_INVALID_ARG;
  CHECK(upload_var_tables<double>(k, Mc.data(), Kc.data(), Tp.data()));
  CHECK(upload_var_tables<float>(k, Mc.data(), Kc.data(), Tp.data()));
  // dense inverse of the coarsest level's interior matrix
  const int n0 = p->levels[0].g.n, m0 = n0 * k - 1;
  const long long nint0 = dim == 3 ? (long long)m0 * m0 * m0 : (long long)m0 * m0;
  if (nint0 > 2000) return GMG_ERR_UNSUPPORTED;
  std::vector<double> A0, A0inv;
  assemble_dense_var(dim, k, n0, lev[0].data(), A0);
  if (!spd_inverse((int)nint0, A0, A0inv)) return GMG_ERR_INVALID_ARG;
  // upload (problem precision per level; FP64 copies of the finest and the inverse)
  const size_t es = p->esize;
  p->esize = 8;
  CHECK(upload_table(p, (void**)&p->coarse_inv, A0inv));
  CHECK(upload_table(p, (void**)&p->coef64, lev[L - 1]));
  p->esize = es;
  p->coef.assign(L, nullptr);
  for (int l = 0; l < L; ++l) CHECK(upload_table(p, &p->coef[l], lev[l]));
  // per interior vertex of each level: the patch's geometric-mean
  // coefficient abar = exp(mean_c log a_c) over its 2^d cells and the FD
  // damping theta = min(1, 1.8 abar / max_c a_c)
  p->vscale.assign(L, nullptr);
  for (int l = 0; l < L; ++l) {
    const int n = p->levels[l].g.n, nv = n - 1;
    const long long ncell = dim == 3 ? (long long)n * n * n : (long long)n * n;
    const long long nvert = dim == 3 ? (long long)nv * nv * nv : (long long)nv * nv;
    std::vector<double> lg(ncell), vs(2 * nvert);
    for (long long c = 0; c < ncell; ++c) lg[c] = std::log(lev[l][c]);
    for (long long v = 0; v < nvert; ++v) {
      const int vx = (int)(v % nv), vy = (int)((v / nv) % nv), vz = dim == 3 ? (int)(v / ((long long)nv * nv)) : 0;
      double s = 0.0, amax = 0.0;
      for (int o = 0; o < (1 << dim); ++o) {
        const long long c = (vx + (o & 1)) + (long long)n * ((vy + ((o >> 1) & 1)) +
                                                          (dim == 3 ? (long long)n * (vz + ((o >> 2) & 1)) : 0));
        s += lg[c];
        amax = std::max(amax, lev[l][c]);
      }
      const double abar = std::exp(s / (1 << dim));
      vs[2 * v] = abar;
      vs[2 * v + 1] = std::min(1.0, 1.8 * abar / amax);
    }
    CHECK(upload_table(p, &p->vscale[l], vs));
  }
  p->coarse_n = (int)nint0;
  p->corr.assign(L, nullptr);
  p->corr_levels = 0;
  p->varcoef = true;
  p->local_solver = GMG_LOCAL_FD_MEAN;
  return cudaDeviceSynchronize() == cudaSuccess ? GMG_OK : GMG_ERR_CUDA;
}

int gmg_set_local_solver(gmg_problem* p, int solver) {
  if (!p || !p->varcoef) return GMG_ERR_INVALID_ARG;
  drop_cg_graph(p);
  if (solver == GMG_LOCAL_FD_MEAN) {
    p->local_solver = solver;
    return GMG_OK;
  }
  if (solver == GMG_LOCAL_LEARNED) {
    bool trained = false;
    for (float* c : p->corr) trained = trained || c;
    if (!trained) return GMG_ERR_INVALID_ARG;  // train first
    p->local_solver = solver;
    return GMG_OK;
  }
  return GMG_ERR_INVALID_ARG;
}

int gmg_set_operator_tile(gmg_problem* p, int tile) {
  if (!p || tile < 0 || tile > 3) return GMG_ERR_INVALID_ARG;
  drop_cg_graph(p);
  p->apply_tile = tile;
  return GMG_OK;
}

int gmg_autotune(gmg_problem* p, gmg_tuning* out) {
  if (!p || p->finest_borrowed) return GMG_ERR_INVALID_ARG;
  drop_cg_graph(p);
  const int Lf = (int)p->levels.size() - 1;
  Level& F = p->levels[Lf];
  cudaStream_t s = p->stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return GMG_ERR_CUDA;
  int st = GMG_OK;
  // any data will do for timing; the level's internal vectors are zeroed again below
  if (cudaMemsetAsync(F.u, 0x3F, F.n_elems * p->esize, s) != cudaSuccess ||
      cudaMemsetAsync(F.b, 0x3F, F.n_elems * p->esize, s) != cudaSuccess)
    st = GMG_ERR_CUDA;
  auto time_ms = [&](auto&& body, int reps, float* ms) -> int {
    CHECK(body());  // warm-up (sets each kernel up)
    if (cudaEventRecord(e0, s) != cudaSuccess) return GMG_ERR_CUDA;
    for (int r = 0; r < reps; ++r) CHECK(body());
    if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) return GMG_ERR_CUDA;
    if (cudaEventElapsedTime(ms, e0, e1) != cudaSuccess) return GMG_ERR_CUDA;
    *ms /= (float)reps;
    return GMG_OK;
  };
  gmg_tuning t;
  std::memset(&t, 0, sizeof(t));
  t.slab_width = p->slab_width;
  t.operator_tile = p->apply_tile;
  // ---- slab width: only where slab schedules give the whole-colour result
  // bit for bit (the whole-colour sweep uses the closure kernel) ----
  const bool faces_used = p->faces && p->shared_faces;
  const bool slabs_ok = !p->varcoef && !faces_used &&
                        !((p->desc.precision == GMG_FP32_TC || p->desc.precision == GMG_FP32_TF32) &&
                          tc_supported(F.g.dim, F.g.k));
  auto sweep = [&]() { return smooth(p, Lf, F.u, F.b, 1, 0); };
  if (st == GMG_OK && slabs_ok) {
    const int cand[6] = {0, 1, 2, 4, 8, -1};
    float best = 0.f;
    int best_w = 0;
    for (int i = 0; i < 6 && st == GMG_OK; ++i) {
      const int W = cand[i];
      p->slab_width = W;
      st = build_slabs(p, Lf, slab_width_for(p, F));
      float ms = 0.f;
      if (st == GMG_OK) st = time_ms(sweep, 3, &ms);
      if (i == 0) t.sweep_ms_default = ms;
      if (st == GMG_OK && (i == 0 || ms < best)) {
        best = ms;
        best_w = W;
      }
    }
    p->slab_width = best_w;
    for (int l = 0; l <= Lf && st == GMG_OK; ++l) st = build_slabs(p, l, slab_width_for(p, p->levels[l]));
    t.slab_width = best_w;
    t.sweep_ms = best;
  } else if (st == GMG_OK) {
    float ms = 0.f;
    st = time_ms(sweep, 3, &ms);
    t.sweep_ms = t.sweep_ms_default = ms;
  }
  // ---- tile shape of the operator kernel (3D, degrees 3, 4, 7, where the
  // level operator is the tile kernel) ----
  const bool tile_op = !p->varcoef && F.g.dim == 3 && (F.g.k == 3 || F.g.k == 4 || F.g.k == 7) &&
                       !(p->esize == 8 && p->op_ws());
  auto apply = [&]() { return apply_level(p, Lf, F.u, F.r, nullptr, op_scale(F), 0.0); };
  if (st == GMG_OK && tile_op) {
    float best = 0.f;
    int best_t = 0;
    for (int tv = 0; tv <= 3 && st == GMG_OK; ++tv) {
      p->apply_tile = tv;
      float ms = 0.f;
      st = time_ms(apply, 5, &ms);
      if (tv == 0) t.operator_ms_default = ms;
      if (st == GMG_OK && (tv == 0 || ms < best)) {
        best = ms;
        best_t = tv;
      }
    }
    p->apply_tile = best_t;
    t.operator_tile = best_t;
    t.operator_ms = best;
  } else if (st == GMG_OK) {
    float ms = 0.f;
    st = time_ms(apply, 5, &ms);
    t.operator_ms = t.operator_ms_default = ms;
  }
  if (cudaMemsetAsync(F.u, 0, F.n_elems * p->esize, s) != cudaSuccess ||
      cudaMemsetAsync(F.b, 0, F.n_elems * p->esize, s) != cudaSuccess ||
      cudaMemsetAsync(F.r, 0, F.n_elems * p->esize, s) != cudaSuccess)
    st = st == GMG_OK ? GMG_ERR_CUDA : st;
  if (cudaStreamSynchronize(s) != cudaSuccess) st = st == GMG_OK ? GMG_ERR_CUDA : st;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (out) *out = t;
  return st;
}

int gmg_set_phase_timing(gmg_problem* p, int enable) {
  if (!p) return GMG_ERR_INVALID_ARG;
  p->phase_timing = enable != 0;
  return GMG_OK;
}

int gmg_set_three_pass_operator(gmg_problem* p, int enable) {
  if (!p) return GMG_ERR_INVALID_ARG;
  drop_cg_graph(p);
  p->three_pass = enable != 0;
  return GMG_OK;
}

int gmg_three_pass_operator(const gmg_problem* p) {
  if (!p) return GMG_ERR_INVALID_ARG;
  return p->op_ws() ? 1 : 0;
}

int gmg_set_shared_faces(gmg_problem* p, int enable) {
  if (!p) return GMG_ERR_INVALID_ARG;
  drop_cg_graph(p);
  p->shared_faces = enable != 0;
  return GMG_OK;
}

int gmg_shared_faces(const gmg_problem* p) {
  if (!p) return GMG_ERR_INVALID_ARG;
  return p->shared_faces && p->faces ? 1 : 0;
}

int gmg_set_small_sweep(gmg_problem* p, int max_patches) {
  if (!p || max_patches < 0) return GMG_ERR_INVALID_ARG;
  drop_cg_graph(p);
  p->small_patches = max_patches;
  // levels that leave or join the coarse-level kernel take or drop their slabs
  for (int l = 0; l < (int)p->levels.size(); ++l) CHECK(build_slabs(p, l, slab_width_for(p, p->levels[l])));
  return GMG_OK;
}

int gmg_small_sweep(const gmg_problem* p) {
  if (!p) return GMG_ERR_INVALID_ARG;
  return p->small_patches;
}

int gmg_set_slab_width(gmg_problem* p, int width) {
  if (!p || width < -1) return GMG_ERR_INVALID_ARG;
  drop_cg_graph(p);
  p->slab_width = width;
  for (int l = 0; l < (int)p->levels.size(); ++l) CHECK(build_slabs(p, l, slab_width_for(p, p->levels[l])));
  return cudaDeviceSynchronize() == cudaSuccess ? GMG_OK : GMG_ERR_CUDA;
}

int gmg_slab_width(const gmg_problem* p, int level) {
  if (!valid_level(p, level)) return GMG_ERR_INVALID_ARG;
  return p->levels[level].slab_w;
}

int gmg_smooth_variant(gmg_problem* p, int level, void* u, const void* b, int variant,
                       long long batch_size, int reverse) {
  if (!valid_level(p, level) || !u || !b || u == b) return GMG_ERR_INVALID_ARG;
  if (p->varcoef && variant != GMG_SWEEP_COMBINED) return GMG_ERR_UNSUPPORTED;
  switch (variant) {
    case GMG_SWEEP_COMBINED: return smooth(p, level, u, b, 1, reverse);
    case GMG_SWEEP_SEPARATED: return smooth_separated(p, level, u, b, reverse);
    case GMG_SWEEP_BATCHED:
      if (batch_size < 1) return GMG_ERR_INVALID_ARG;
      return smooth_batched(p, level, u, b, batch_size, reverse);
    default: return GMG_ERR_INVALID_ARG;
  }
}

int gmg_restrict(gmg_problem* p, int fine_level, const void* fine, void* coarse) {
  if (!p || fine_level < 1 || fine_level >= (int)p->levels.size() || !fine || !coarse)
    return GMG_ERR_INVALID_ARG;
  return restrict_to(p, fine_level, fine, coarse);
}

int gmg_prolongate_add(gmg_problem* p, int coarse_level, const void* coarse, void* fine) {
  if (!p || coarse_level < 0 || coarse_level + 1 >= (int)p->levels.size() || !fine || !coarse)
    return GMG_ERR_INVALID_ARG;
  return prolongate_add(p, coarse_level, coarse, fine);
}

int gmg_coarse_solve(gmg_problem* p, const void* b, void* x) {
  if (!p || !b || !x || b == x) return GMG_ERR_INVALID_ARG;
  return coarse_solve(p, b, x);
}

int gmg_vcycle(gmg_problem* p, void* x, const void* b) {
  if (!p || !x || !b || x == b) return GMG_ERR_INVALID_ARG;
  return vcycle_level(p, (int)p->levels.size() - 1, x, b);
}

int cg_gmg_solve(gmg_problem* p, double* u, const double* b, double rtol, int max_it,
                 gmg_solve_stats* st) {
  if (!p || !u || !b || u == b || !(rtol > 0.0) || max_it < 0) return GMG_ERR_INVALID_ARG;
  const int Lf = (int)p->levels.size() - 1;
  Level& F = p->levels[Lf];
  const long long n = F.n_elems;
  cudaStream_t s = p->stream;
  double* sc = p->scal;
  gmg_solve_stats local;
  std::memset(&local, 0, sizeof(local));
  double h_sc[S_COUNT];
  const cudaStream_t user_stream = s;
  const bool timing = p->phase_timing;
  p->phase_marks.clear();
  for (double& t : p->phase_ms) t = 0.0;
  auto fetch = [&]() -> int {
    if (cudaMemcpyAsync(h_sc, sc, sizeof(h_sc), cudaMemcpyDeviceToHost, s) != cudaSuccess) return GMG_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return GMG_ERR_CUDA;
    if (timing) collect_phases(p);
    return GMG_OK;
  };
  auto precondition = [&]() -> int {  // z = V(r)
    if (p->esize == 8) return vcycle_level(p, Lf, p->cg_z, p->cg_r);
    {
      PhaseScope ph(p, GMG_PHASE_VECTOR);
      CHECK(launch_convert_f64_f32(n, p->cg_r, (float*)F.b, s));
    }
    CHECK(vcycle_level(p, Lf, F.u, F.b));
    PhaseScope ph(p, GMG_PHASE_VECTOR);
    return launch_convert_f32_f64(n, (const float*)F.u, p->cg_z, s);
  };
  auto finish = [&](int status) -> int {
    if (timing) {
      if (cudaStreamSynchronize(s) == cudaSuccess) collect_phases(p);
      cudaGetLastError();
      for (int i = 0; i < GMG_PHASE_COUNT; ++i) local.phase_ms[i] = p->phase_ms[i];
    }
    if (st) *st = local;
    return status;
  };
  // FP64 operator of the outer CG: y = sign A x + beta z
  auto cg_apply = [&](const double* x, double* y, const double* z, double sign, double beta) -> int {
    PhaseScope ph(p, GMG_PHASE_OPERATOR);
    if (p->varcoef)
      return launch_apply_var<double>(F.g, F.n_elems, x, y, z, sign * op_scale(F), beta, p->coef64, s);
    ApplyLaunch al;
    al.g = F.g;
    al.alpha = sign * op_scale(F);
    al.beta = beta;
    al.ws = p->op_ws();
    return launch_apply<double>(al, x, y, z, s);
  };
  // r = b - A u
  CHECK(cg_apply(u, p->cg_r, b, -1.0, 1.0));
  {
    PhaseScope ph(p, GMG_PHASE_VECTOR);
    CHECK(launch_dot(n, b, b, p->partial, sc + S_BB, s));
    CHECK(launch_dot(n, p->cg_r, p->cg_r, p->partial, sc + S_RR, s));
  }
  CHECK(fetch());
  const double bnorm = std::sqrt(h_sc[S_BB]);
  double rnorm = std::sqrt(h_sc[S_RR]);
  if (!std::isfinite(bnorm) || !std::isfinite(rnorm)) return finish(GMG_ERR_NONFINITE);
  local.initial_residual = rnorm;
  local.final_residual = rnorm;
  local.relative_residual = bnorm > 0 ? rnorm / bnorm : 0.0;
  local.residual_history[0] = local.relative_residual;
  if (rnorm <= rtol * bnorm || bnorm == 0.0) {
    local.converged = 1;
    return finish(GMG_OK);
  }
  CHECK(precondition());
  {
    PhaseScope ph(p, GMG_PHASE_VECTOR);
    if (cudaMemcpyAsync(p->cg_p, p->cg_z, n * 8, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      return finish(GMG_ERR_CUDA);
    CHECK(launch_dot(n, p->cg_r, p->cg_z, p->partial, sc + S_RZ, s));
  }
  // q = A p, alpha = rz / pq, u += alpha p, r -= alpha q, rr = r.r
  auto update = [&]() -> int {
    CHECK(cg_apply(p->cg_p, p->cg_q, nullptr, 1.0, 0.0));
    PhaseScope ph(p, GMG_PHASE_VECTOR);
    CHECK(launch_dot(n, p->cg_p, p->cg_q, p->partial, sc + S_PQ, s));
    return launch_cg_update(n, u, p->cg_r, p->cg_p, p->cg_q, sc + S_RZ, sc + S_PQ, p->partial, sc + S_RR, s);
  };
  // z = V(r), beta = rz_new / rz, p = z + beta p, then the update
  auto iteration_body = [&]() -> int {
    CHECK(precondition());
    {
      PhaseScope ph(p, GMG_PHASE_VECTOR);
      CHECK(launch_dot(n, p->cg_r, p->cg_z, p->partial, sc + S_RZN, s));
      CHECK(launch_cg_direction(n, p->cg_p, p->cg_z, sc + S_RZN, sc + S_RZ, s));
      if (cudaMemcpyAsync(sc + S_RZ, sc + S_RZN, 8, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return GMG_ERR_CUDA;
    }
    return update();
  };
  CHECK(update());
  for (int it = 1; it <= max_it; ++it) {
    CHECK(fetch());
    if (!std::isfinite(h_sc[S_RZ]) || !std::isfinite(h_sc[S_PQ]) || !std::isfinite(h_sc[S_RR]))
      return finish(GMG_ERR_NONFINITE);
    if (!(h_sc[S_RZ] > 0.0) || !(h_sc[S_PQ] > 0.0)) return finish(GMG_ERR_BREAKDOWN);
    rnorm = std::sqrt(h_sc[S_RR]);
    local.iterations = it;
    local.final_residual = rnorm;
    local.relative_residual = rnorm / bnorm;
    if (it < 64) local.residual_history[it] = local.relative_residual;
    if (rnorm <= rtol * bnorm) {
      local.converged = 1;
      return finish(GMG_OK);
    }
    if (it == max_it) break;
    if (timing) {  // direct launches, so that every phase gets its events
      CHECK(iteration_body());
      continue;
    }
    // next iteration up to its convergence check: a CUDA graph replay
    // (captured once the first iteration has prepared every kernel)
    if (!p->cg_exec || p->cg_graph_u != u) {
      drop_cg_graph(p);
      if (!p->cap_stream && cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
        return finish(GMG_ERR_CUDA);
      const long long before = launch_count();
      s = p->stream = p->cap_stream;  // the caller's stream may be the legacy one
      int cst = GMG_OK;
      cudaGraph_t g = nullptr;
      if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cst = GMG_ERR_CUDA;
      } else {
        cst = iteration_body();
        if (cudaStreamEndCapture(s, &g) != cudaSuccess || !g) cst = cst == GMG_OK ? GMG_ERR_CUDA : cst;
      }
      s = p->stream = user_stream;
      const long long captured = launch_count() - before;
      count_launch((int)-captured);  // captured launches run with the graph
      if (cst != GMG_OK) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return finish(cst);
      }
      p->cg_graph = g;
      if (cudaGraphInstantiate(&p->cg_exec, g, 0) != cudaSuccess) {
        drop_cg_graph(p);
        return finish(GMG_ERR_CUDA);
      }
      p->cg_graph_u = u;
      p->cg_graph_kernels = captured;
    }
    if (cudaGraphLaunch(p->cg_exec, s) != cudaSuccess) return finish(GMG_ERR_CUDA);
    count_launch((int)p->cg_graph_kernels);
  }
  return finish(GMG_ERR_NOT_CONVERGED);
}

}  // extern "C"

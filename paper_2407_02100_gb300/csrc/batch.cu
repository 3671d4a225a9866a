// Batches of independent problems (different mesh sizes, same dimension,
// degree and precision) solved together: one sweep-kernel launch per colour
// covers the patches of every problem at a given depth of its level
// hierarchy, the batched V-cycle is captured once into a CUDA graph and
// replayed, and the outer FP64 CG keeps per-problem scalars and stops each
// problem when it converges.  Each problem is the same method as a single
// gmg_problem (the paper's smoother, Algorithm 4, inside V(1,1) and PCG);
// batching only changes how the work is scheduled on the GPU.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/gmg.h"
#include "kernels.h"
#include "problem.h"

using namespace gmg;
using namespace gmg::detail;

struct gmg_batch {
  gmg_desc desc{};
  cudaStream_t stream = nullptr;
  size_t esize = 8;
  int n = 0;
  std::vector<gmg_problem*> probs;
  std::vector<long long> off;   // element offset of each problem's finest vector
  std::vector<long long> len;   // its element count
  long long total = 0;
  int max_depth = 0;            // deepest level count over the problems
  // concatenated finest-level vectors in the problem precision
  void* fu = nullptr;
  void* fb = nullptr;
  void* fr = nullptr;
  // concatenated FP64 CG vectors and per-problem scalars
  double *cr = nullptr, *cz = nullptr, *cp = nullptr, *cq = nullptr;
  double *rz = nullptr, *pq = nullptr, *rr = nullptr, *rzn = nullptr, *bb = nullptr;
  int* active = nullptr;
  double* partial = nullptr;
  // workspace of the three-pass FP64 operator, sized for the largest
  // problem and shared (the problems' operators run one after another on
  // the batch stream); null: the tile kernel
  void* apply_ws = nullptr;
  Segments seg;
  int ppc = 0;                  // tuned patches per CTA of the batched sweep (0 = default)
  cudaStream_t cap_stream = nullptr;  // private stream the graph is captured on
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t vgraph = nullptr;
  size_t graph_nodes = 0;
  std::vector<void*> owned;
};

namespace {

int balloc(gmg_batch* B, void** ptr, size_t bytes) {
  *ptr = nullptr;
  if (bytes == 0) bytes = 16;
  if (cudaMalloc(ptr, bytes) != cudaSuccess) {
    cudaGetLastError();
    return GMG_ERR_OOM;
  }
  B->owned.push_back(*ptr);
  return cudaMemset(*ptr, 0, bytes) == cudaSuccess ? GMG_OK : GMG_ERR_CUDA;
}

char* at(void* base, long long elems, size_t esize) { return static_cast<char*>(base) + elems * esize; }

int level_of(const gmg_problem* p, int depth) { return (int)p->levels.size() - 1 - depth; }

// One colour of the smoother on every problem that has a smoothed level at
// `depth` (level index >= 1), in one launch per table chunk.
int batch_colour(gmg_batch* B, int depth, int colour, bool finest_user, void* u_all, const void* b_all) {
  std::vector<PatchLaunch> pls;
  std::vector<void*> us;
  std::vector<const void*> bs;
  for (int i = 0; i < B->n; ++i) {
    gmg_problem* p = B->probs[i];
    const int l = level_of(p, depth);
    if (l < 1) continue;
    Level& L = p->levels[l];
    pls.push_back(colour_launch(L, colour, B->desc.damping));
    if (depth == 0 && finest_user) {
      us.push_back(at(u_all, B->off[i], B->esize));
      bs.push_back(at(const_cast<void*>(b_all), B->off[i], B->esize));
    } else {
      us.push_back(L.u);
      bs.push_back(L.b);
    }
  }
  if (pls.empty()) return GMG_OK;
  const int dim = B->desc.dim, k = B->desc.degree;
  if (B->esize == 8)
    return launch_patch_table<double>(dim, k, pls.data(), (double* const*)us.data(),
                                      (const double* const*)bs.data(), (int)pls.size(),
                                      (const double*)B->probs[0]->dinv, B->ppc, B->stream);
  const int pr = B->desc.precision;
  if ((pr == GMG_FP32_TC || pr == GMG_FP32_TF32) && tc_supported(dim, k))
    return launch_patch_table_tc(dim, k, pls.data(), (float* const*)us.data(), (const float* const*)bs.data(),
                                 (int)pls.size(), (const float*)B->probs[0]->dinv, pr == GMG_FP32_TC, B->stream);
  return launch_patch_table<float>(dim, k, pls.data(), (float* const*)us.data(),
                                   (const float* const*)bs.data(), (int)pls.size(),
                                   (const float*)B->probs[0]->dinv, B->ppc, B->stream);
}

int batch_smooth(gmg_batch* B, int depth, int reverse, bool finest_user, void* u_all, const void* b_all) {
  const int nc = 1 << B->desc.dim;
  const int sweeps = reverse ? B->desc.post_sweeps : B->desc.pre_sweeps;
  for (int s = 0; s < sweeps; ++s)
    for (int i = 0; i < nc; ++i)
      CHECK(batch_colour(B, depth, reverse ? nc - 1 - i : i, finest_user, u_all, b_all));
  return GMG_OK;
}

// V-cycle of every problem from `depth` down, x_0 = 0 (the same sequence of
// operations as gmg_vcycle on each problem; the sweeps are batched).
int batch_vcycle(gmg_batch* B, int depth) {
  bool any_smooth = false;
  for (int i = 0; i < B->n; ++i) {
    gmg_problem* p = B->probs[i];
    const int l = level_of(p, depth);
    if (l == 0) CHECK(coarse_solve(p, p->levels[0].b, p->levels[0].u));
    if (l >= 1) {
      any_smooth = true;
      Level& L = p->levels[l];
      if (cudaMemsetAsync(L.u, 0, L.n_elems * B->esize, B->stream) != cudaSuccess) return GMG_ERR_CUDA;
    }
  }
  if (!any_smooth) return GMG_OK;
  CHECK(batch_smooth(B, depth, 0, false, nullptr, nullptr));
  for (int i = 0; i < B->n; ++i) {
    gmg_problem* p = B->probs[i];
    const int l = level_of(p, depth);
    if (l < 1) continue;
    Level& L = p->levels[l];
    CHECK(apply_level(p, l, L.u, L.r, L.b, -op_scale(L), 1.0));
    CHECK(restrict_to(p, l, L.r, p->levels[l - 1].b));
  }
  CHECK(batch_vcycle(B, depth + 1));
  for (int i = 0; i < B->n; ++i) {
    gmg_problem* p = B->probs[i];
    const int l = level_of(p, depth);
    if (l < 1) continue;
    CHECK(prolongate_add(p, l - 1, p->levels[l - 1].u, p->levels[l].u));
  }
  return batch_smooth(B, depth, 1, false, nullptr, nullptr);
}

void drop_graph(gmg_batch* B) {
  if (B->vgraph) cudaGraphExecDestroy(B->vgraph);
  if (B->graph) cudaGraphDestroy(B->graph);
  B->vgraph = nullptr;
  B->graph = nullptr;
}

// V-cycle on the internal finest buffers fb -> fu, through the CUDA graph
// (captured on first use, after one direct run has prepared every kernel).
int run_vcycle(gmg_batch* B) {
  if (!B->vgraph) {
    CHECK(batch_vcycle(B, 0));
    if (cudaStreamSynchronize(B->stream) != cudaSuccess) return GMG_ERR_CUDA;
    // capture on a private stream (the caller's may be the legacy default
    // stream, which cannot be captured); the graph is launched on the
    // caller's stream
    if (!B->cap_stream &&
        cudaStreamCreateWithFlags(&B->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
      return GMG_ERR_CUDA;
    cudaStream_t user = B->stream;
    auto set_streams = [&](cudaStream_t st) {
      B->stream = st;
      for (gmg_problem* p : B->probs) p->stream = st;
    };
    set_streams(B->cap_stream);
    if (cudaStreamBeginCapture(B->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      set_streams(user);
      return GMG_ERR_CUDA;
    }
    const int st = batch_vcycle(B, 0);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(B->cap_stream, &g);
    set_streams(user);
    if (st != GMG_OK || e != cudaSuccess || !g) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return st != GMG_OK ? st : GMG_ERR_CUDA;
    }
    B->graph = g;
    if (cudaGraphInstantiate(&B->vgraph, g, 0) != cudaSuccess) {
      drop_graph(B);
      return GMG_ERR_CUDA;
    }
    size_t nn = 0;
    cudaGraphGetNodes(g, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    if (nn) cudaGraphGetNodes(g, nodes.data(), &nn);
    B->graph_nodes = 0;
    for (size_t i = 0; i < nn; ++i) {
      cudaGraphNodeType t;
      if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++B->graph_nodes;
    }
  }
  if (cudaGraphLaunch(B->vgraph, B->stream) != cudaSuccess) return GMG_ERR_CUDA;
  count_launch((int)B->graph_nodes);
  return GMG_OK;
}

// FP64 operator on every problem's finest level: y = alpha A x + beta z
int batch_apply_f64(gmg_batch* B, const double* x, double* y, const double* z, double sign, double beta) {
  for (int i = 0; i < B->n; ++i) {
    gmg_problem* p = B->probs[i];
    const Level& L = p->levels.back();
    ApplyLaunch al;
    al.g = L.g;
    al.alpha = sign * op_scale(L);
    al.beta = beta;
    al.ws = B->apply_ws;
    CHECK(launch_apply<double>(al, x + B->off[i], y + B->off[i], z ? z + B->off[i] : nullptr, B->stream));
  }
  return GMG_OK;
}

// z = V(r) for all problems: r (FP64) -> fb, graph, fu -> z
int batch_precondition(gmg_batch* B, const double* r, double* z) {
  if (B->esize == 8) {
    if (cudaMemcpyAsync(B->fb, r, B->total * 8, cudaMemcpyDeviceToDevice, B->stream) != cudaSuccess)
      return GMG_ERR_CUDA;
    CHECK(run_vcycle(B));
    return cudaMemcpyAsync(z, B->fu, B->total * 8, cudaMemcpyDeviceToDevice, B->stream) == cudaSuccess
               ? GMG_OK : GMG_ERR_CUDA;
  }
  CHECK(launch_convert_f64_f32(B->total, r, (float*)B->fb, B->stream));
  CHECK(run_vcycle(B));
  return launch_convert_f32_f64(B->total, (const float*)B->fu, z, B->stream);
}

bool valid_batch(const gmg_batch* B) { return B && B->n > 0; }

}  // namespace

extern "C" {

int gmg_batch_destroy(gmg_batch* B) {
  if (!B) return GMG_OK;
  cudaStreamSynchronize(B->stream);
  drop_graph(B);
  if (B->cap_stream) cudaStreamDestroy(B->cap_stream);
  for (gmg_problem* p : B->probs) gmg_destroy(p);
  for (void* ptr : B->owned) cudaFree(ptr);
  delete B;
  return GMG_OK;
}

int gmg_batch_create(const gmg_desc* desc, int n_problems, const int* n_cells, gmg_batch** out) {
  if (!out) return GMG_ERR_INVALID_ARG;
  *out = nullptr;
  if (!desc || n_problems < 1 || !n_cells) return GMG_ERR_INVALID_ARG;
  for (int i = 0; i < n_problems; ++i) {
    gmg_desc d = *desc;
    d.n_cells = n_cells[i];
    d.n_levels = 0;
    if (check_desc(&d) != GMG_OK) return GMG_ERR_INVALID_ARG;
  }
  gmg_batch* B = new (std::nothrow) gmg_batch();
  if (!B) return GMG_ERR_OOM;
  B->desc = *desc;
  B->stream = (cudaStream_t)desc->stream;
  B->esize = desc->precision == GMG_FP64 ? 8 : 4;
  B->n = n_problems;
  // layout of the concatenated finest vectors (each problem 64-element aligned)
  for (int i = 0; i < n_problems; ++i) {
    LevelGeom g = make_geom(desc->dim, desc->degree, n_cells[i]);
    const long long e = geom_elems(g);
    B->off.push_back(B->total);
    B->len.push_back(e);
    B->total += (e + 63) / 64 * 64;
  }
  int st = GMG_OK;
  auto fail = [&](int s) {
    gmg_batch_destroy(B);
    return s;
  };
  if ((st = balloc(B, &B->fu, B->total * B->esize))) return fail(st);
  if ((st = balloc(B, &B->fb, B->total * B->esize))) return fail(st);
  if ((st = balloc(B, &B->fr, B->total * B->esize))) return fail(st);
  for (int i = 0; i < n_problems; ++i) {
    gmg_desc d = *desc;
    d.n_cells = n_cells[i];
    d.n_levels = 0;
    gmg_problem* p = new (std::nothrow) gmg_problem();
    if (!p) return fail(GMG_ERR_OOM);
    B->probs.push_back(p);
    CreateOptions opt;
    opt.finest_u = at(B->fu, B->off[i], B->esize);
    opt.finest_b = at(B->fb, B->off[i], B->esize);
    opt.finest_r = at(B->fr, B->off[i], B->esize);
    opt.no_cg = true;
    opt.no_faces = true;
    if ((st = create_problem(&d, p, opt))) return fail(st);
    B->max_depth = std::max(B->max_depth, (int)p->levels.size());
  }
  // FP64 CG vectors, per-problem scalars and the chunking of the concatenation
  double** vecs[] = {&B->cr, &B->cz, &B->cp, &B->cq};
  for (double** v : vecs)
    if ((st = balloc(B, (void**)v, B->total * 8))) return fail(st);
  double** sc[] = {&B->rz, &B->pq, &B->rr, &B->rzn, &B->bb};
  for (double** v : sc)
    if ((st = balloc(B, (void**)v, n_problems * 8))) return fail(st);
  if ((st = balloc(B, (void**)&B->active, n_problems * sizeof(int)))) return fail(st);
  if (staged_apply_preferred(desc->dim, desc->degree)) {
    long long lmax = 0;
    for (long long l : B->len) lmax = std::max(lmax, l);
    if (balloc(B, &B->apply_ws, 4 * lmax * 8) != GMG_OK) B->apply_ws = nullptr;
  }
  std::vector<long long> cstart;
  std::vector<int> clen, cowner, cbegin;
  for (int i = 0; i < n_problems; ++i) {
    cbegin.push_back((int)cstart.size());
    for (long long s0 = 0; s0 < B->len[i]; s0 += kSegChunk) {
      cstart.push_back(B->off[i] + s0);
      clen.push_back((int)std::min<long long>(kSegChunk, B->len[i] - s0));
      cowner.push_back(i);
    }
  }
  cbegin.push_back((int)cstart.size());
  void *d_start, *d_len, *d_owner, *d_begin;
  if ((st = balloc(B, &d_start, cstart.size() * 8))) return fail(st);
  if ((st = balloc(B, &d_len, clen.size() * 4))) return fail(st);
  if ((st = balloc(B, &d_owner, cowner.size() * 4))) return fail(st);
  if ((st = balloc(B, &d_begin, cbegin.size() * 4))) return fail(st);
  if ((st = balloc(B, (void**)&B->partial, cstart.size() * 8))) return fail(st);
  if (cudaMemcpy(d_start, cstart.data(), cstart.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(d_len, clen.data(), clen.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(d_owner, cowner.data(), cowner.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(d_begin, cbegin.data(), cbegin.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess)
    return fail(GMG_ERR_CUDA);
  B->seg.n_chunks = (int)cstart.size();
  B->seg.n_problems = n_problems;
  B->seg.start = (const long long*)d_start;
  B->seg.len = (const int*)d_len;
  B->seg.owner = (const int*)d_owner;
  B->seg.begin = (const int*)d_begin;
  *out = B;
  return GMG_OK;
}

int gmg_batch_layout(const gmg_batch* B, int problem, long long* offset, long long* n_elems,
                     long long* total) {
  if (!valid_batch(B) || problem < 0 || problem >= B->n) return GMG_ERR_INVALID_ARG;
  if (offset) *offset = B->off[problem];
  if (n_elems) *n_elems = B->len[problem];
  if (total) *total = B->total;
  return GMG_OK;
}

int gmg_batch_problem(const gmg_batch* B, int problem, gmg_problem** out) {
  if (!valid_batch(B) || problem < 0 || problem >= B->n || !out) return GMG_ERR_INVALID_ARG;
  *out = B->probs[problem];
  return GMG_OK;
}

int gmg_batch_smooth(gmg_batch* B, void* u, const void* b, int reverse) {
  if (!valid_batch(B) || !u || !b || u == b) return GMG_ERR_INVALID_ARG;
  const int nc = 1 << B->desc.dim;
  for (int i = 0; i < nc; ++i) CHECK(batch_colour(B, 0, reverse ? nc - 1 - i : i, true, u, b));
  return GMG_OK;
}

int gmg_batch_vcycle(gmg_batch* B, void* x, const void* b) {
  if (!valid_batch(B) || !x || !b || x == b) return GMG_ERR_INVALID_ARG;
  const size_t bytes = B->total * B->esize;
  if (cudaMemcpyAsync(B->fb, b, bytes, cudaMemcpyDeviceToDevice, B->stream) != cudaSuccess)
    return GMG_ERR_CUDA;
  CHECK(run_vcycle(B));
  return cudaMemcpyAsync(x, B->fu, bytes, cudaMemcpyDeviceToDevice, B->stream) == cudaSuccess
             ? GMG_OK : GMG_ERR_CUDA;
}

int gmg_batch_autotune(gmg_batch* B, int* ppc_out) {
  if (!valid_batch(B)) return GMG_ERR_INVALID_ARG;
  const int candidates[4] = {0, 1, 2, 4};
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return GMG_ERR_CUDA;
  float best = 1e30f;
  int best_ppc = 0;
  for (int c : candidates) {
    B->ppc = c;
    int st = gmg_batch_smooth(B, B->fu, B->fb, 0);  // warm-up (prepares the variant)
    if (st != GMG_OK) break;
    cudaEventRecord(e0, B->stream);
    for (int r = 0; r < 3 && st == GMG_OK; ++r) st = gmg_batch_smooth(B, B->fu, B->fb, 0);
    cudaEventRecord(e1, B->stream);
    if (st != GMG_OK || cudaEventSynchronize(e1) != cudaSuccess) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) {
      best = ms;
      best_ppc = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  B->ppc = best_ppc;
  drop_graph(B);  // re-captured with the chosen variant on next use
  cudaMemsetAsync(B->fu, 0, B->total * B->esize, B->stream);
  if (ppc_out) *ppc_out = best_ppc;
  return cudaStreamSynchronize(B->stream) == cudaSuccess ? GMG_OK : GMG_ERR_CUDA;
}

int gmg_batch_set_ppc(gmg_batch* B, int ppc) {
  if (!valid_batch(B) || (ppc != 0 && ppc != 1 && ppc != 2 && ppc != 4)) return GMG_ERR_INVALID_ARG;
  if (B->ppc != ppc) drop_graph(B);
  B->ppc = ppc;
  return GMG_OK;
}

int gmg_batch_cg_solve(gmg_batch* B, double* u, const double* b, double rtol, int max_it,
                       int* iterations, double* rel_residual) {
  if (!valid_batch(B) || !u || !b || u == b || !(rtol > 0.0) || max_it < 0) return GMG_ERR_INVALID_ARG;
  const int n = B->n;
  cudaStream_t s = B->stream;
  std::vector<double> h_rr(n), h_bb(n), h_pq(n), h_rz(n);
  std::vector<int> h_active(n, 1), its(n, 0);
  auto fetch = [&](double* dev, std::vector<double>& host) -> int {
    return cudaMemcpyAsync(host.data(), dev, n * 8, cudaMemcpyDeviceToHost, s) == cudaSuccess
               ? GMG_OK : GMG_ERR_CUDA;
  };
  auto push_active = [&]() -> int {
    return cudaMemcpyAsync(B->active, h_active.data(), n * sizeof(int), cudaMemcpyHostToDevice, s) ==
                   cudaSuccess ? GMG_OK : GMG_ERR_CUDA;
  };
  // r = b - A u
  CHECK(batch_apply_f64(B, u, B->cr, b, -1.0, 1.0));
  CHECK(launch_seg_dot(B->seg, b, b, B->partial, B->bb, s));
  CHECK(launch_seg_dot(B->seg, B->cr, B->cr, B->partial, B->rr, s));
  CHECK(fetch(B->bb, h_bb));
  CHECK(fetch(B->rr, h_rr));
  if (cudaStreamSynchronize(s) != cudaSuccess) return GMG_ERR_CUDA;
  int n_active = 0;
  for (int i = 0; i < n; ++i) {
    if (!std::isfinite(h_rr[i]) || !std::isfinite(h_bb[i])) return GMG_ERR_NONFINITE;
    h_active[i] = (h_bb[i] > 0.0 && std::sqrt(h_rr[i]) > rtol * std::sqrt(h_bb[i])) ? 1 : 0;
    n_active += h_active[i];
  }
  CHECK(push_active());
  int status = GMG_OK;
  if (n_active > 0) {
    CHECK(batch_precondition(B, B->cr, B->cz));
    if (cudaMemcpyAsync(B->cp, B->cz, B->total * 8, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      return GMG_ERR_CUDA;
    CHECK(launch_seg_dot(B->seg, B->cr, B->cz, B->partial, B->rz, s));
    for (int it = 1; it <= max_it && n_active > 0; ++it) {
      CHECK(batch_apply_f64(B, B->cp, B->cq, nullptr, 1.0, 0.0));
      CHECK(launch_seg_dot(B->seg, B->cp, B->cq, B->partial, B->pq, s));
      CHECK(launch_seg_cg_update(B->seg, u, B->cr, B->cp, B->cq, B->rz, B->pq, B->active, B->partial,
                                 B->rr, s));
      CHECK(fetch(B->rr, h_rr));
      CHECK(fetch(B->pq, h_pq));
      CHECK(fetch(B->rz, h_rz));
      if (cudaStreamSynchronize(s) != cudaSuccess) return GMG_ERR_CUDA;
      n_active = 0;
      for (int i = 0; i < n; ++i) {
        if (!h_active[i]) continue;
        if (!std::isfinite(h_rr[i]) || !std::isfinite(h_pq[i]) || !std::isfinite(h_rz[i]))
          return GMG_ERR_NONFINITE;
        if (!(h_pq[i] > 0.0) || !(h_rz[i] > 0.0)) return GMG_ERR_BREAKDOWN;
        its[i] = it;
        if (std::sqrt(h_rr[i]) <= rtol * std::sqrt(h_bb[i])) h_active[i] = 0;
        n_active += h_active[i];
      }
      CHECK(push_active());
      if (n_active == 0) break;
      CHECK(batch_precondition(B, B->cr, B->cz));
      CHECK(launch_seg_dot(B->seg, B->cr, B->cz, B->partial, B->rzn, s));
      CHECK(launch_seg_cg_direction(B->seg, B->cp, B->cz, B->rzn, B->rz, B->active, s));
      if (cudaMemcpyAsync(B->rz, B->rzn, n * 8, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return GMG_ERR_CUDA;
    }
    if (n_active > 0) status = GMG_ERR_NOT_CONVERGED;
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) return GMG_ERR_CUDA;
  for (int i = 0; i < n; ++i) {
    if (iterations) iterations[i] = its[i];
    if (rel_residual) rel_residual[i] = h_bb[i] > 0 ? std::sqrt(h_rr[i] / h_bb[i]) : 0.0;
  }
  return status;
}

}  // extern "C"

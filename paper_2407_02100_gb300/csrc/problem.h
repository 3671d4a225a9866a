// Internal definitions shared by the C ABI translation units (api.cu,
// batch.cu): the problem object and the level operations the V-cycles are
// built from.  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "../../include/gmg.h"
#include "kernels.h"

namespace gmg {
namespace detail {

struct Level {
  LevelGeom g;
  long long n_elems = 0;
  double h = 0.0;
  void* u = nullptr;  // level correction (problem precision)
  void* b = nullptr;  // level right-hand side (problem precision)
  void* r = nullptr;  // level residual (problem precision)
  // patches of every colour in Z-curve order (Algorithm 5), built on demand
  int* zlist = nullptr;
  int zoff[9] = {0};
  // skewed-slab schedule of width slab_w (vertex rows along the slowest
  // axis), for the forward [0] and reverse [1] colour orders: the patches of
  // (slab s, order position o) are slist[d][soff[d][s * n_colours + o] ..
  // soff[d][s * n_colours + o + 1]) (lexicographic ids within the colour)
  int slab_w = 0;
  int* slist[2] = {nullptr, nullptr};
  std::vector<int> soff[2];
};

// Options of problem creation used by batches: the finest level's u, b, r
// may live in caller-owned slices, and the outer-CG vectors may be omitted.
struct CreateOptions {
  void* finest_u = nullptr;
  void* finest_b = nullptr;
  void* finest_r = nullptr;
  bool no_cg = false;
  bool no_faces = false;  // no face buffer or operator workspace (batch members)
};

}  // namespace detail
}  // namespace gmg

struct gmg_problem {
  gmg_desc desc{};
  cudaStream_t stream = nullptr;
  size_t esize = 8;  // bytes per level-vector element
  std::vector<gmg::detail::Level> levels;
  // patch fast diagonalisation: 1/(sum of eigenvalues) over M^d modes
  void* dinv = nullptr;
  // transfer tables (problem precision): prolongation 2k x (k+1),
  // restriction k x (4k-1)
  void* coef_prol = nullptr;
  void* coef_rest = nullptr;
  // host copies of the transfer tables, read by the double-float transfer
  // passes of FP64 problems (xfer_df: the tables have the expected pattern)
  std::vector<double> prol_h, rest_h;
  bool xfer_df = false;
  void* tmp1 = nullptr;  // transfer temporaries
  void* tmp2 = nullptr;
  // coarsest-level fast diagonalisation
  int m0 = 0;
  void* coef_c_fwd = nullptr;  // T0^T  (m0 x m0)
  void* coef_c_bwd = nullptr;  // T0    (m0 x m0)
  void* dinv0 = nullptr;       // h0^{2-d} / sum lambda
  void* ctmp1 = nullptr;
  void* ctmp2 = nullptr;
  // single-precision problems solve the coarsest level in FP64: FP64 copies
  // of the tables above, temporaries, and the level's b and x
  void* c64_fwd = nullptr;
  void* c64_bwd = nullptr;
  void* c64_dinv = nullptr;
  void* c64_t1 = nullptr;
  void* c64_t2 = nullptr;
  void* c64_b = nullptr;
  void* c64_x = nullptr;
  // outer CG (double, finest level)
  double* cg_r = nullptr;
  double* cg_z = nullptr;
  double* cg_p = nullptr;
  double* cg_q = nullptr;
  double* partial = nullptr;
  double* scal = nullptr;  // device scalars
  // variable coefficient -div(a grad u) (gmg_set_coefficient): one value per
  // cell and level (problem precision), the finest also in FP64 for the CG
  bool varcoef = false;
  std::vector<void*> coef;
  std::vector<void*> vscale;  // per level: (abar, theta) of every interior vertex's patch
  double* coef64 = nullptr;
  int local_solver = 0;             // GMG_LOCAL_FD_MEAN or GMG_LOCAL_LEARNED
  int corr_rank = 0;
  std::vector<float*> corr;         // per level: [patches][m^d * rank + rank] or null
  unsigned corr_levels = 0;         // bit l: level l applies its correction (level judge)
  double* coarse_inv = nullptr;     // dense inverse of the coarsest interior matrix
  int coarse_n = 0;
  std::vector<void*> owned;
  // skewed-slab schedule request: 0 whole colours, > 0 slab width in
  // vertex rows, -1 chosen per level to fit L2 (gmg_set_slab_width)
  int slab_width = 0;
  // shared-face form of the FP64 3D sweep (degrees >= 3, whole colours):
  // face buffer sized for the largest colour of the finest level and reused
  // by every level (null: the closure form is used), and its switch
  // (gmg_set_shared_faces)
  void* faces = nullptr;
  bool shared_faces = true;
  // FP64 colour steps of at most this many patches use the coarse-level
  // kernel (gmg_set_small_sweep; 0: never; set by gmg_create)
  int small_patches = 0;
  // workspace of the three-pass FP64 3D operator (four finest-level
  // vectors), null where the tile kernel is used
  void* apply_ws = nullptr;
  bool three_pass = true;  // gmg_set_three_pass_operator
  int apply_tile = 0;      // tile shape of the operator kernel (gmg_set_operator_tile)
  bool finest_borrowed = false;  // finest u, b, r are slices of a batch's vectors
  void* op_ws() const { return three_pass ? apply_ws : nullptr; }
  // CUDA graph of one outer-CG iteration (V-cycle preconditioner, dot
  // products, direction, FP64 operator, update) for the solution vector
  // cg_graph_u, captured on a private stream; dropped whenever anything the
  // V-cycle launches changes
  cudaStream_t cap_stream = nullptr;
  cudaGraph_t cg_graph = nullptr;
  cudaGraphExec_t cg_exec = nullptr;
  const void* cg_graph_u = nullptr;
  long long cg_graph_kernels = 0;
  // per-phase timing of the CG (gmg_set_phase_timing): event pairs recorded
  // on the stream around each outermost phase, summed into phase_ms at the
  // solver's synchronisation points; events are pooled and reused
  bool phase_timing = false;
  int phase_depth = 0;
  struct PhaseMark {
    int phase;
    cudaEvent_t start, stop;
  };
  std::vector<PhaseMark> phase_marks;
  std::vector<cudaEvent_t> event_pool;
  double phase_ms[GMG_PHASE_COUNT] = {};
};

namespace gmg {
namespace detail {

#define CHECK(x)                   \
  do {                             \
    int st_ = (x);                 \
    if (st_ != GMG_OK) return st_; \
  } while (0)

// Times the enclosed launches as one phase when phase timing is on and no
// enclosing scope is open (the outermost phase owns the time of nested ones).
class PhaseScope {
 public:
  PhaseScope(gmg_problem* p, int phase);
  ~PhaseScope();
  PhaseScope(const PhaseScope&) = delete;
  PhaseScope& operator=(const PhaseScope&) = delete;

 private:
  gmg_problem* p_;
  int phase_;
  cudaEvent_t start_ = nullptr;
};
// add the elapsed times of the recorded phases (stream already synchronised)
void collect_phases(gmg_problem* p);
void release_phase_events(gmg_problem* p);

int dalloc(gmg_problem* p, void** ptr, size_t bytes);
// forget the captured outer-CG iteration (anything the V-cycle launches changed)
void drop_cg_graph(gmg_problem* p);
LevelGeom make_geom(int dim, int k, int n);
long long geom_elems(const LevelGeom& g);
double op_scale(const Level& L);  // h^{d-2}
int apply_level(gmg_problem* p, int level, const void* x, void* y, const void* bvec, double alpha,
                double beta);
PatchLaunch colour_launch(const Level& L, int colour, double omega);
int launch_colour(gmg_problem* p, const PatchLaunch& pl, void* u, const void* b);
int smooth(gmg_problem* p, int level, void* u, const void* b, int n_sweeps, int reverse);
int prolongate_add(gmg_problem* p, int cl, const void* coarse, void* fine);
int restrict_to(gmg_problem* p, int fl, const void* fine, void* coarse);
int coarse_solve(gmg_problem* p, const void* b, void* x);
int vcycle_level(gmg_problem* p, int l, void* x, const void* b);
int create_problem(const gmg_desc* d, gmg_problem* p, const CreateOptions& opt);
int upload_table(gmg_problem* p, void** dst, const std::vector<double>& src);
int check_desc(const gmg_desc* d);

}  // namespace detail
}  // namespace gmg

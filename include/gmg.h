/*
 * gmg.h -- C ABI of the GB300 multiplicative vertex-patch smoother and the
 * geometric multigrid / conjugate-gradient solver built around it.
 *
 * Method: Wichrowski, Munch, Kronbichler, Kanschat, "Smoothers with localized
 * residual computations for geometric multigrid methods" (arXiv 2407.02100).
 *
 * Problem: -div(grad u) = f on the unit square/cube, homogeneous Dirichlet
 * data, continuous Q_k elements (Gauss-Lobatto support points) on a uniform
 * Cartesian mesh of n cells per direction (App. A.2), with nested levels
 * obtained by halving n (Sec. 2).
 *
 * VECTOR LAYOUT (every vector argument).  A level with n cells has
 * N = n k + 1 nodes per direction.  Node (i_0, i_1[, i_2]) is stored at
 *     i_0 + pitch_y * i_1 [+ pitch_z * i_2],
 * with pitch_y = N rounded up to a multiple of 4 and pitch_z = pitch_y * N;
 * a vector holds n_elems = pitch_y * N (2D) or pitch_z * N (3D) elements.
 * gmg_vector_layout() returns these numbers.  Dirichlet nodes (any index 0
 * or N-1) and padding entries (i_0 >= N) must be zero on input; every call
 * keeps them zero.  Vectors are DEVICE pointers owned by the caller, of the
 * element type given per call (double, or float for GMG_FP32 level vectors).
 *
 * STREAMS.  Every call is enqueued on gmg_desc.stream (a cudaStream_t; NULL
 * = legacy default stream) and returns without waiting, except
 * cg_gmg_solve(), which synchronises the stream to read back scalars.
 *
 * ERRORS.  Every entry point returns GMG_OK (0) or a negative status; no
 * C++ exception crosses the ABI.  gmg_status_string() names a status.
 * A problem object must not be used from two host threads at once.
 */
#ifndef GMG_H
#define GMG_H

#ifdef __cplusplus
extern "C" {
#endif

enum gmg_status {
  GMG_OK = 0,
  GMG_ERR_INVALID_ARG = -1,   /* bad descriptor, level, pointer or size */
  GMG_ERR_OOM = -2,           /* device allocation failed */
  GMG_ERR_CUDA = -3,          /* a CUDA runtime call or launch failed */
  GMG_ERR_NONFINITE = -4,     /* NaN/Inf met in a solver scalar */
  GMG_ERR_BREAKDOWN = -5,     /* CG breakdown: p^T A p <= 0 or r^T z <= 0 */
  GMG_ERR_NOT_CONVERGED = -6, /* max_it reached above the tolerance */
  GMG_ERR_UNSUPPORTED = -7,   /* valid but not implemented combination */
  GMG_ERR_TIMEOUT = -8        /* a bounded device-side wait expired (tensor-core sweep) */
};

enum gmg_precision {
  GMG_FP64 = 0,  /* smoother, transfer and V-cycle in double */
  GMG_FP32 = 1,  /* smoother, transfer and V-cycle in float (inside FP64 CG) */
  GMG_FP32_TC = 2,  /* as GMG_FP32, and for 3D degrees 4..7 the combined
                       sweep's 1D contractions run on the tensor cores with
                       FP32 accumulation, each factor split into its TF32
                       rounding and the TF32 rounding of the remainder, three
                       MMAs per product (hi*hi + lo*hi + hi*lo: FP32-level
                       accuracy); other degrees, 2D and the sweep variants
                       use the FP32 kernels */
  GMG_FP32_TF32 = 3 /* as GMG_FP32_TC with data and matrices rounded to TF32
                       once (one MMA per product; the smoother then depends on
                       its input's rounding and the outer CG needs more
                       iterations) */
};

enum gmg_sweep_variant {
  GMG_SWEEP_COMBINED = 0,   /* Algorithm 4: combined colourised (local residuals) */
  GMG_SWEEP_SEPARATED = 1,  /* Algorithm 3: global residual per colour, then solves */
  GMG_SWEEP_BATCHED = 2     /* Algorithm 5: Z-curve batches of n_B patches per colour */
};

enum gmg_local_solver {
  GMG_LOCAL_FD_MEAN = 0,   /* FD of the constant-coefficient patch, scaled by the mean coefficient */
  GMG_LOCAL_LEARNED = 1    /* the same plus the learned rank-R correction (gmg_learned_train) */
};

typedef struct gmg_problem gmg_problem; /* opaque; owns all level data */

typedef struct {
  int dim;          /* 2 or 3 */
  int degree;       /* k, 1..8 */
  int n_cells;      /* cells per direction on the finest level, >= 2 */
  int n_levels;     /* >= 1; 0 = halve n while it stays even and >= 2 */
  int precision;    /* enum gmg_precision */
  double damping;   /* omega of the scatter u += omega d (1.0 = the paper's P_j) */
  int pre_sweeps;   /* smoothing steps before the coarse correction (>= 0) */
  int post_sweeps;  /* smoothing steps after it (>= 0) */
  void* stream;     /* cudaStream_t used by every call on this problem */
} gmg_desc;

/* Phases of a solve, as timed by gmg_set_phase_timing (the GPU form of the
 * breakdown of a V-cycle's time into its parts, Sec. 4). */
enum gmg_phase {
  GMG_PHASE_SMOOTH = 0,    /* patch smoothing sweeps of every level */
  GMG_PHASE_OPERATOR = 1,  /* level residuals b - A x and the CG's operator */
  GMG_PHASE_TRANSFER = 2,  /* restriction and prolongation */
  GMG_PHASE_COARSE = 3,    /* coarsest-level solve */
  GMG_PHASE_VECTOR = 4,    /* CG dot products and updates, precision
                              conversions, zeroing of level corrections */
  GMG_PHASE_COUNT = 5
};

typedef struct {
  int iterations;            /* CG iterations done */
  int converged;             /* 1 if ||r|| <= rtol ||b|| */
  double initial_residual;   /* ||b - A u_0|| */
  double final_residual;     /* ||b - A u|| (recurrence residual) */
  double relative_residual;  /* final_residual / ||b|| */
  double residual_history[64]; /* relative residuals, entry i after iteration i */
  double phase_ms[GMG_PHASE_COUNT]; /* GPU milliseconds per phase (enum
                                       gmg_phase) when phase timing is on,
                                       zeros otherwise */
} gmg_solve_stats;

/* Create a problem: builds the level hierarchy (Sec. 2, nested meshes), the
 * 1D reference matrices, the fast-diagonalisation data of the patch (App.
 * A.3, K T = M T Lambda with T^T M T = I) and of the coarsest level, and
 * allocates the internal level vectors on the current CUDA device.
 * desc: read only; *out receives the new problem (NULL on failure).
 * Errors: INVALID_ARG (dim not 2/3, degree not 1..8, n_cells < 2, levels
 * not possible for n_cells, precision unknown, damping not finite), OOM,
 * CUDA. */
int gmg_create(const gmg_desc* desc, gmg_problem** out);

/* Release every device buffer of the problem after synchronising its
 * stream.  NULL is accepted. */
int gmg_destroy(gmg_problem* p);

/* Layout of vectors on `level` (0 = coarsest, n_levels-1 = finest); see the
 * layout note above.  Any output pointer may be NULL.  Host-only. */
int gmg_vector_layout(const gmg_problem* p, int level, long long* n_elems,
                      int* nodes_1d, int* pitch_y, long long* pitch_z);

/* Number of levels and cells per direction of a level.  Host-only. */
int gmg_level_info(const gmg_problem* p, int level, int* n_cells, int* n_levels);

/* y = A_level x: the matrix-free stiffness operator of the level (Sec. 2,
 * eq. "matrix"; evaluated by sum factorisation of the tensor-product cell
 * operators, App. A.1).  x, y: device vectors of the problem's level-vector
 * type (double for GMG_FP64, float for GMG_FP32), distinct buffers.
 * Only interior nodes of y are written; its Dirichlet and padding entries
 * must already be zero (as for every vector argument). */
int gmg_apply_operator(gmg_problem* p, int level, const void* x, void* y);

/* Same operator in double precision regardless of the problem precision
 * (the operator used by the outer CG).  Finest level only is guaranteed to
 * be allocated for GMG_FP32 problems; any level for GMG_FP64. */
int gmg_apply_operator_f64(gmg_problem* p, int level, const double* x, double* y);

/* Multiplicative vertex-patch smoothing on `level`, in place on u, with
 * right-hand side b: n_sweeps steps of the combined colourised smoother
 * (Algorithm 4).  Each patch gathers u on its closure and b on its interior
 * (eq. "gather"), forms the local residual r_j = b_j - Pi_j bar A_j bar u_j
 * (eq. "main:4"), solves A_j d_j = r_j by fast diagonalisation (App. A.3,
 * eq. "fdm:inverse"), and adds omega d_j to the patch interior (eq.
 * "scatter").  Colours c = sum_a 2^a (v_a mod 2) of the vertex v are taken
 * in ascending order, or descending when reverse != 0.  u, b: level vectors
 * of the problem's type. */
int gmg_smooth(gmg_problem* p, int level, void* u, const void* b, int n_sweeps, int reverse);

/* One colour of the smoother (all patches of colour `colour`, 0..2^dim-1),
 * in place on u.  Same arguments and semantics as gmg_smooth. */
int gmg_smooth_colour(gmg_problem* p, int level, void* u, const void* b, int colour);

/* One smoothing step on `level` in one of the paper's loop organisations
 * (Sec. 3.2, 3.3 and 4.1): GMG_SWEEP_COMBINED = Algorithm 4 (as gmg_smooth);
 * GMG_SWEEP_SEPARATED = Algorithm 3, per colour one level residual
 * r = b - A u followed by the colour's local solves from r (same result as
 * Algorithm 4 up to rounding); GMG_SWEEP_BATCHED = Algorithm 5, patches in
 * Z-curve order (Morton order of the vertex index, v_0 lowest bit) grouped by
 * colour and cut into batches of batch_size; for each batch index every
 * colour's batch in turn (bit for bit the closure form of Algorithm 4 when
 * batch_size >= the largest colour; see gmg_set_shared_faces).  reverse != 0 reverses colours (and batches).  The first batched
 * call on a level allocates its patch list.  Errors: INVALID_ARG (unknown
 * variant, batch_size < 1), OOM, CUDA. */
int gmg_smooth_variant(gmg_problem* p, int level, void* u, const void* b, int variant,
                       long long batch_size, int reverse);

/* coarse = R fine with R = P^T, the transpose of the embedding prolongation
 * (Sec. 2, restriction as the adjoint of the embedding).  fine: level
 * `fine_level` (>= 1), coarse: level fine_level-1; problem's vector type.
 * One pass per axis; FP64 problems compute the passes in double-float
 * arithmetic (agreeing with FP64 arithmetic to about 1e-14 relative) and
 * use the problem's two transfer temporaries, so calls on one problem must
 * not overlap.  Errors: INVALID_ARG (level out of range, null vector),
 * UNSUPPORTED (a pass too large for one launch), CUDA. */
int gmg_restrict(gmg_problem* p, int fine_level, const void* fine, void* coarse);

/* fine += P coarse, P the embedding of V_{l} into V_{l+1} (Sec. 2).
 * coarse: level `coarse_level`, fine: level coarse_level+1.  Passes,
 * arithmetic, temporaries and errors as for gmg_restrict. */
int gmg_prolongate_add(gmg_problem* p, int coarse_level, const void* coarse, void* fine);

/* x = A_0^{-1} b on the coarsest level, by fast diagonalisation of the
 * whole level (exact for the constant-coefficient Cartesian operator). */
int gmg_coarse_solve(gmg_problem* p, const void* b, void* x);

/* x = V(b): one V-cycle on the finest level with x_0 = 0 (Sec. 2, the
 * V-cycle; pre-smoothing with ascending colours, post-smoothing with
 * descending colours, exact coarse solve).  x, b: finest-level vectors of
 * the problem's type. */
int gmg_vcycle(gmg_problem* p, void* x, const void* b);

/* Preconditioned CG on the finest level in double precision, preconditioned
 * by one V-cycle per iteration (in the problem's precision).  u: initial
 * guess on input (a restart resumes from it), solution on output; b: right
 * hand side; both double device vectors.  Stops when ||r|| <= rtol ||b||.
 * stats may be NULL.  Errors: INVALID_ARG, CUDA, NONFINITE, BREAKDOWN,
 * NOT_CONVERGED (u then holds the last iterate).  From the second iteration
 * on, one iteration up to its convergence check (V-cycle, dot products,
 * direction, FP64 operator, update) is replayed as a CUDA graph captured on
 * a private stream for this u (kept until u, the coefficient, the local
 * solver or the slab schedule changes); the host reads back the scalars once
 * per iteration.  Results are identical to launching the kernels one by one. */
int cg_gmg_solve(gmg_problem* p, double* u, const double* b, double rtol, int max_it,
                 gmg_solve_stats* stats);

/* ---- Autotuning (result-neutral choices timed on the GPU) -----------------
 * gmg_set_operator_tile: the tile shape of the operator kernel for 3D
 * problems of degree 3, 4 or 7 where the level operator is the tile kernel
 * (FP32 levels, FP64 problems without the three-pass form): 0 the default
 * shape of the precision and degree, 1 cubes, 2 flat 4x4x1 cells, 3 flat
 * 8x4x1 cells (a shape whose tile exceeds the shared memory of a CTA runs
 * as the default).  Every shape evaluates each output row by the same sums
 * in the same order, so results are bit-identical (App. A.1's sum
 * factorisation, tiled differently).  GMG_ERR_INVALID_ARG for other values.
 * gmg_autotune: times, on the finest level of p, one smoothing step for the
 * slab widths 0 (whole colours), 1, 2, 4, 8 and the L2-sized width -1 of
 * gmg_set_slab_width (only where slab schedules reproduce the whole-colour
 * sweep bit for bit: constant coefficient, and whole colours in the closure
 * kernel, i.e. not the shared-face form or the tensor-core sweep), and five
 * operator applications for each tile shape where the shape is selectable;
 * keeps the fastest of each, and reports the choice and the times (NULL out
 * allowed).  Uses the level's internal vectors as scratch (zeroed on
 * return); synchronises the stream.  GMG_ERR_INVALID_ARG for a null problem
 * or a batch member (whose finest vectors are the batch's). */
typedef struct {
  int slab_width;             /* chosen: 0 whole colours, > 0 width, -1 the L2 rule */
  int operator_tile;          /* chosen tile shape (see gmg_set_operator_tile) */
  double sweep_ms;            /* finest-level smoothing step with the choice */
  double sweep_ms_default;    /* with whole colours */
  double operator_ms;         /* finest-level operator with the choice */
  double operator_ms_default; /* with the default tile shape */
} gmg_tuning;
int gmg_set_operator_tile(gmg_problem* p, int tile);
int gmg_autotune(gmg_problem* p, gmg_tuning* out);

/* Per-phase timing of cg_gmg_solve (enable != 0) or none (0, the default).
 * When on, the solver records a pair of CUDA events on the problem's stream
 * around each phase (enum gmg_phase) of every iteration, launches each
 * iteration's kernels directly instead of replaying its CUDA graph, and
 * returns the summed event times in gmg_solve_stats.phase_ms.  Results are
 * the same either way; the events and the direct launches add a little
 * time.  GMG_ERR_INVALID_ARG for a null problem. */
int gmg_set_phase_timing(gmg_problem* p, int enable);

/* gmg_smooth without a problem object and without allocating device memory
 * (the paper has no counterpart: this is a deployment variant).  For callers
 * that cannot call cudaMalloc -- their device memory belongs to another
 * allocator (a framework arena or pool), or they must not incur cudaMalloc's
 * implicit device-wide synchronisation.  Runs n_sweeps FP64 smoothing steps
 * on one uniform level of n_cells cells per direction (same layout, colour
 * order and damping semantics as gmg_smooth), in place on the caller's
 * double device vectors u and b, on `stream` (a cudaStream_t).
 * The fast-diagonalisation diagonal (with its float-pair split for the
 * double-float arithmetic of the FP64 sweep) lives in a library-owned static
 * device array of 2 (2*8-1)^3 doubles (54 KB, kept on every GPU that loads
 * the library until exit); patches needing more are rejected with
 * GMG_ERR_INVALID_ARG, as are bad dim/degree/n_cells/damping/pointers.
 * SET-UP: the first call for a (device, degree) pair does that pair's set-up
 * with the device current: it looks the array's address up and copies the
 * degree's coefficient tables to __constant__ memory (cudaMemcpyToSymbol:
 * synchronous, no allocation).  Make that first call outside any stream
 * capture.  Every later call for the pair only enqueues kernels on `stream`:
 * one that rewrites the part of the array the degree uses, then one per
 * colour.  Calls that overlap on the GPU (different streams, no ordering
 * between them) race on the array.
 * STATUS: a bounded wait of the sweep kernel that expires is not reported by
 * the return value (the call returns before the kernels run); it sets the
 * device flag read by gmg_tc_status(). */
int gmg_smooth_noalloc(int dim, int degree, int n_cells, double damping, double* u,
                       const double* b, int n_sweeps, int reverse, void* stream);

/* ---- Batches of independent problems ------------------------------------
 * Many problems of one dimension, degree and precision but different mesh
 * sizes, solved together (each problem is the same method as a single
 * gmg_problem; batching only schedules the work): one sweep-kernel launch per
 * colour covers the patches of all problems at a given depth of their level
 * hierarchies, the batched V-cycle is captured once into a CUDA graph and
 * replayed, and the FP64 CG keeps per-problem scalars, stopping each problem
 * when it converges.  Batch vectors concatenate the finest-level vectors of
 * all problems: problem i occupies elements [offset_i, offset_i + n_elems_i)
 * in its own gmg_vector_layout, gaps are zero. */
typedef struct gmg_batch gmg_batch;

/* desc: dim, degree, precision, damping, sweeps and stream shared by all
 * problems (desc->n_cells and n_levels are ignored); n_cells[i] is problem
 * i's finest mesh, levels by halving while even and >= 2.  Errors:
 * INVALID_ARG (any problem's descriptor invalid, n_problems < 1), OOM, CUDA. */
int gmg_batch_create(const gmg_desc* desc, int n_problems, const int* n_cells, gmg_batch** out);
int gmg_batch_destroy(gmg_batch* b);

/* Offset and length (elements) of problem i in a batch vector, and the
 * batch vector length.  Host-only; outputs may be NULL. */
int gmg_batch_layout(const gmg_batch* b, int problem, long long* offset, long long* n_elems,
                     long long* total);

/* The problem object of batch member i (owned by the batch: do not destroy;
 * use it for gmg_vector_layout and single-problem calls on its own vectors). */
int gmg_batch_problem(const gmg_batch* b, int problem, gmg_problem** out);

/* One finest-level smoothing step (Algorithm 4) of every problem, in place on
 * the batch vector u with right-hand side b (problem precision), one launch
 * per colour; reverse != 0 takes the colours in descending order. */
int gmg_batch_smooth(gmg_batch* b, void* u, const void* rhs, int reverse);

/* x = V(rhs) for every problem (batch vectors, problem precision), through
 * the captured CUDA graph (the first call captures it; make it before any
 * capture of your own). */
int gmg_batch_vcycle(gmg_batch* b, void* x, const void* rhs);

/* PCG of every problem to ||r_i|| <= rtol ||b_i||, FP64 batch vectors u
 * (initial guess in, solution out) and rhs.  iterations[i], rel_residual[i]
 * (host arrays of n_problems entries, may be NULL) receive per-problem
 * results.  Errors: INVALID_ARG, CUDA, NONFINITE, BREAKDOWN, NOT_CONVERGED. */
int gmg_batch_cg_solve(gmg_batch* b, double* u, const double* rhs, double rtol, int max_it,
                       int* iterations, double* rel_residual);

/* Choose, by timing batched sweeps on the GPU, the number of patches per CTA
 * of the batched sweep kernel (0 = the default configuration, or 1, 2, 4;
 * the variants exist for 3D FP32 up to degree 4).  The choice never changes
 * results: every patch is computed the same way whatever the grouping.
 * *ppc_out (may be NULL) receives the choice. */
int gmg_batch_autotune(gmg_batch* b, int* ppc_out);

/* Set the patches-per-CTA variant explicitly (0, 1, 2 or 4). */
int gmg_batch_set_ppc(gmg_batch* b, int ppc);

/* ---- Variable coefficient ------------------------------------------------
 * Switch the problem to -div(a grad u) with one coefficient per cell of the
 * finest mesh: coef is a HOST array of n_cells^dim positive values, cell
 * (c_0, c_1[, c_2]) at c_0 + n c_1 [+ n^2 c_2].  Coarser levels take the
 * geometric mean of their 2^dim children; the coarse solve becomes the dense
 * inverse of the coarsest interior matrix (at most 2000 unknowns).  The patch
 * local residual is evaluated cell by cell with the coefficients (the paper's
 * local_update, Sec. 3.1); since fast diagonalisation is then only
 * approximate (App. A.3 assumes a tensor-product patch matrix), the local
 * solver is the constant-coefficient FD scaled by the geometric mean of the
 * patch's cell coefficients (GMG_LOCAL_FD_MEAN), optionally corrected by
 * the learned low-rank term (GMG_LOCAL_LEARNED).  Degrees 1..3 only
 * (GMG_ERR_UNSUPPORTED otherwise); only the combined sweep variant. */
int gmg_set_coefficient(gmg_problem* p, const double* coef);

/* Select the local solver of a variable-coefficient problem; LEARNED needs a
 * completed gmg_learned_train. */
int gmg_set_local_solver(gmg_problem* p, int solver);

/* ---- Learned correction of the local solver (no counterpart in the paper;
 * it builds on the paper's remark that approximate local solvers fit the
 * subspace-correction framework, Sec. 2.1).  Variable-coefficient problems,
 * degree <= 3 in 3D (patch interiors of at most 125 nodes).
 * A two-layer perceptron (8 -> 32 tanh -> m^d R + R, R = 4) maps the
 * log-coefficients of a patch's cells, relative to their mean, to a
 * symmetric rank-R correction U diag(s) U^T of the reference FD inverse.
 * gmg_learned_train generates its data by exact dense (Cholesky, FP64) solves
 * of sample patches of any level -- sample_vertices: HOST array of n_samples
 * patch ids over the levels, finest level first: ids [0, (n-1)^d) are the
 * finest level's lexicographic vertex ids v0-1 + (n-1)(v1-1) [+ (n-1)^2 (v2-1)],
 * the next (n/2-1)^d ids those of the next coarser level, and so on;
 * residuals: DEVICE array n_samples x m^d (FP64) of reference-unit residuals --
 * trains with Adam for `steps` minibatches of `batch` samples (learning rate
 * lr; parameters initialised from `seed`; FP32 master weights) with the loss
 * ||theta FD r + U diag(s) U^T r - A_exact^{-1} r||^2 / ||A_exact^{-1} r||^2
 * (theta = min(1, 1.8 abar / max_c a_c), the FD damping of the patch), then
 * evaluates the network (FP16-rounded weights, FP32 accumulation) on every
 * patch of every level and keeps a patch's correction only if it lowers the
 * local energy-norm error on a probe residual (damped FD is the fallback).
 * Finally a level judge decides per level whether the correction is used at
 * all: the FP64 CG solves a fixed probe right-hand side to 1e-10 with no
 * level corrected, then, from the coarsest level up, a level keeps its
 * correction only if the iteration count drops below the best so far
 * (see gmg_learned_levels).  loss_history (HOST, `steps` entries) and
 * kept_patches (patches kept by the per-patch gate, all levels) may be NULL.
 * On success the local solver becomes GMG_LOCAL_LEARNED.  Allocates the
 * per-patch corrections (m^d R + R floats per patch and level) and
 * temporaries; synchronises the device. */
int gmg_learned_train(gmg_problem* p, int n_samples, const int* sample_vertices,
                      const double* residuals, int steps, int batch, double lr, unsigned seed,
                      double* loss_history, int* kept_patches);

/* Levels whose learned correction the smoother applies under
 * GMG_LOCAL_LEARNED, as a bit mask (bit l = level l, 0 = coarsest), chosen
 * by the level judge of gmg_learned_train; the other levels use damped FD.
 * gmg_learned_set_levels overrides the choice (every set bit must name a
 * trained level).  Errors: INVALID_ARG (null or constant-coefficient
 * problem, bits beyond the levels or on untrained levels). */
int gmg_learned_levels(const gmg_problem* p);
int gmg_learned_set_levels(gmg_problem* p, int mask);

/* Copy the per-patch corrections of `level` (patches in lexicographic vertex
 * order, each U (m^d x R, row-major) then s (R)) to the HOST array out of
 * `count` floats. */
int gmg_learned_corrections(const gmg_problem* p, int level, float* out, long long count);

/* The training targets of gmg_learned_train, exposed for testing: for each of
 * n patches, the exact reference-unit local solve d_exact = Ahat(w)^{-1} r and
 * the damped fast-diagonalisation solve d_fd = theta Ahat^{-1} r, theta =
 * min(1, 1.8 / max_c w_c) (App. A.3 for Ahat^{-1}; the exact solve is the
 * A_j^{-1} of the local problem, Sec. 2.1, for cells of unit width).  Ahat(w)
 * is the patch-interior stiffness block assembled from the 2^dim unit-cell
 * matrices weighted by w, and factorised by dense FP64 Cholesky on the GPU.
 * w: DEVICE double n x 2^dim cell weights, cell offset o_0 fastest, with
 * geometric mean 1 per patch (the cell coefficients divided by their
 * geometric mean); r: DEVICE double n x m^dim residuals (m = 2 degree - 1,
 * lexicographic, x fastest); d_exact, d_fd: DEVICE double n x m^dim outputs.
 * degree 1..3.  Allocates and frees device memory and synchronises the
 * device.  Errors: INVALID_ARG, UNSUPPORTED, OOM, CUDA. */
int gmg_exact_patch_solve(int dim, int degree, int n, const double* w, const double* r, double* d_exact,
                          double* d_fd);

/* Loss and gradient of the perceptron on one batch (for testing the kernels):
 * params (DEVICE, FP32) = W1 [hidden x 2^dim] | b1 [hidden] | W2 [no x hidden]
 * | b2 [no] with no = m^dim rank + rank; X (DEVICE FP32, n x 2^dim); R, DFD,
 * DEX (DEVICE FP64, n x m^dim); loss -> HOST double; grads (DEVICE FP32, same
 * layout as params).  rank <= 4, hidden <= 32, degree <= 3. */
int gmg_mlp_loss_grad(int dim, int degree, int rank, int hidden, int n, const float* params,
                      const float* X, const double* R, const double* DFD, const double* DEX,
                      double* loss, float* grads);

/* Host-only set-up math exposed for testing: the 1D fast-diagonalisation
 * data of one vertex patch built from two cells of unit width (App. A.3):
 * M, K = interior (2k-1)x(2k-1) mass and stiffness of the two-cell 1D
 * Q_k mesh, T with T^T M T = I and T^T K T = diag(lambda).  All arrays are
 * row-major, caller-allocated, of (2k-1)^2 (M, K, T) and 2k-1 (lambda)
 * doubles; any may be NULL. */
int gmg_patch_fd_1d(int degree, double* M, double* K, double* T, double* lambda);

/* ---- Skewed-slab schedule of the sweep (the GPU form of the locality-
 * ordered batches of Sec. 4.1) ---------------------------------------------
 * With width W > 0 the patches of a level are grouped into slabs of W
 * vertex rows along the slowest axis (z in 3D, y in 2D), skewed by the
 * position o of their colour in the sweep's colour order: patch (v, o) is in
 * slab floor((v_slow + o) / W).  gmg_smooth (and the V-cycle) then launch one
 * kernel per (slab, colour) pair, slabs in order, colours in order inside a
 * slab, so consecutive launches touch about (W + 2) k node planes.  A patch
 * that overlaps one of an earlier colour position never lands in an earlier
 * slab, so every patch reads the values Algorithm 4 gives it: results are
 * bit-identical for every W, and to whole colours in the closure form (for
 * FP64 3D problems of degree >= 3 the whole-colour default is the
 * shared-face form below, equal up to rounding).  width = 0 restores one launch per colour
 * (default); width = -1 picks per level the largest W whose node planes of u
 * and b fit in half of the L2 cache (W >= n - 1 + 2^d is one launch per
 * colour).  Constant-coefficient problems only (variable-coefficient ones
 * keep one launch per colour).  Builds the schedules of all levels (device
 * memory, synchronises). */
int gmg_set_slab_width(gmg_problem* p, int width);

/* The slab width in effect on `level` (0 = one launch per colour), or a
 * negative status. */
int gmg_slab_width(const gmg_problem* p, int level);

/* ---- Shared-face form of the 3D sweep ------------------------------------
 * Constant-coefficient 3D problems in FP64 of degree >= 3, and in GMG_FP32 of
 * degree >= 7 (below that the FP32 closure kernel measured faster), evaluate
 * the local
 * residual of a whole-colour sweep (Algorithm 4) from the closure boundary
 * only: the local solver is exact (App. A.3), so the new interior is
 * A_j^{-1}(b_j - bar A_j bar u_j^0) with the patch interior of bar u_j^0 set
 * to zero, and bar A_j bar u_j^0 is a sum over the six closure faces of
 * one-dimensional columns of the two-cell matrices times two-dimensional
 * sum-factorised face terms (eq. "main:4" restricted to the boundary).  A
 * face plane between two same-colour patches has the same terms in both, so
 * each colour launch first evaluates every face once (face kernel) and the
 * patch kernel reads them.  Same method and colour order; results agree
 * with the closure form up to rounding.  The face buffer (allocated by
 * gmg_create: 12 (2k-1)^2 doubles per patch of the finest level's largest
 * colour, about 0.6x a level vector at k = 4, in the problem precision) is
 * shared by all levels; if it cannot be allocated the closure form is used.
 * Algorithm 3 and 5, slab schedules, batches and the tensor-core precisions
 * always use the closure form (or their own kernel).
 * gmg_set_shared_faces: enable (default) or disable the form; returns
 *   GMG_ERR_INVALID_ARG for a null problem.
 * gmg_shared_faces: 1 if whole-colour 3D sweeps of the problem use the
 *   form (enabled and the buffer allocated), 0 if not, GMG_ERR_INVALID_ARG
 *   for a null problem. */
int gmg_set_shared_faces(gmg_problem* p, int enable);
int gmg_shared_faces(const gmg_problem* p);

/* ---- Coarse-level sweep of FP64 problems -----------------------------------
 * A whole-colour sweep step (Algorithm 4) of an FP64 problem whose colour
 * holds at most max_patches patches runs on the coarse-level kernel: one CTA
 * per patch and one thread per output of each stage (the residual on the
 * patch closure by sum factorisation, each fast-diagonalisation transform,
 * then u += omega d), in double-float arithmetic.  A colour step of a
 * coarse level lasts as long as one patch takes; the line kernels give a
 * thread a whole line per stage, this kernel a single output.  Same method
 * and colour order; results agree with the other forms up to rounding.
 * Levels swept by it take no slab schedule.
 * gmg_set_small_sweep: max_patches >= 0 (0 turns the kernel off; gmg_create
 *   sets 256 for degrees up to 4 and 0 above); GMG_ERR_INVALID_ARG for a
 *   null problem or a negative count.  Single-precision and variable-
 *   coefficient problems ignore it.
 * gmg_small_sweep: the current max_patches, GMG_ERR_INVALID_ARG for a null
 *   problem. */
int gmg_set_small_sweep(gmg_problem* p, int max_patches);
int gmg_small_sweep(const gmg_problem* p);

/* ---- Three-pass FP64 operator -------------------------------------------
 * In 3D at degree >= 3 the FP64 level operator (the stiffness operator of
 * Sec. 2, evaluated matrix-free by sum factorisation as in App. A.1;
 * gmg_apply_operator(_f64), the V-cycle residuals of FP64 problems and the
 * FP64 CG of every problem) runs as three passes over the level, one 1D
 * contraction per axis with the
 * global 1D mass and stiffness matrices (z, then y, then x), through four
 * workspace vectors of the finest level (FP64, allocated by gmg_create).
 * Every output row is evaluated once; the tile kernel recomputes a halo of
 * up to k + 1 nodes per direction.  Same operator, results equal up to
 * rounding.  If the workspace cannot be allocated the tile kernel is used.
 * gmg_set_three_pass_operator: enable (default) or disable the form (the
 *   workspace stays allocated); GMG_ERR_INVALID_ARG for a null problem.
 * gmg_three_pass_operator: 1 if the FP64 operator of the problem uses the
 *   form (enabled and the workspace allocated), 0 if not,
 *   GMG_ERR_INVALID_ARG for a null problem. */
int gmg_set_three_pass_operator(gmg_problem* p, int enable);
int gmg_three_pass_operator(const gmg_problem* p);

/* ---- Tensor-core sweep (GMG_FP32_TC) and bounded device waits ----------
 * Every patch of one colour is processed as in gmg_smooth (Algorithm 4,
 * local_update of Sec. 3.1: gather, local residual by sum factorisation,
 * fast-diagonalisation solve of App. A.3, scatter), with each 1D
 * contraction executed as a TF32 tcgen05 MMA over the lines of the patch
 * tensor.  Device-side waits are bounded: on the tensor cores' completion,
 * and on the TMA gathers of the sweep kernels (every sweep gathers a patch's
 * closure with one TMA box per vector when the vectors' base addresses are
 * 16-byte aligned and their pitches multiples of 16 bytes, else with one
 * cp.async per element).  An expired wait makes the kernel finish early and
 * set a device flag (one per device).  This covers every sweep kernel of the
 * library (gmg_smooth and its variants, gmg_smooth_noalloc, the V-cycle and
 * CG, batches, the variable-coefficient sweep) and the tensor-core sweep.
 * gmg_tc_status synchronises the device, returns GMG_OK or the recorded
 * status (GMG_ERR_TIMEOUT) of the current device and clears it. */
int gmg_tc_status(void);

/* Diagnostic of the tensor-core encoding: D = A B^T for one 128 x 16 (A) by
 * 32 x 16 (B) TF32 product on the tensor cores, one MMA tile, as the sweep
 * kernel issues it.  A, B, D are HOST arrays, row-major (A 128x16, B 32x16,
 * D 128x32 floats); inputs are rounded to TF32.  With force_timeout != 0 the
 * MMA completion is signalled only after a short bounded wait has expired:
 * the call then returns GMG_ERR_TIMEOUT (the sweep kernel's failure path)
 * and D still holds the product.  Allocates and frees device memory and
 * synchronises. */
int gmg_tc_probe(const float* A, const float* B, float* D, int force_timeout);

/* Diagnostic with no counterpart in the paper: the measured peak rate of the
 * current device's fused multiply-add pipe for precision GMG_FP64 (DFMA) or
 * GMG_FP32 (FFMA), in TFLOP/s (2 flops per FMA).  It is the denominator of
 * the arithmetic roofline that the sweep kernels are reported against.  A
 * grid of 1024 threads per SM runs 8 independent FMA chains per thread; the
 * best of three timed launches after a warm-up (about 0.1 s each, CUDA
 * events on a private non-blocking stream) is returned in *tflops.  Uses no
 * device allocation; synchronises its stream.  Errors: INVALID_ARG (other
 * precision, NULL tflops), CUDA. */
int gmg_fma_peak(int precision, double* tflops);

/* Number of CUDA kernels this library has enqueued since it was loaded
 * (host-side counter, all problems and devices).  Host-only. */
long long gmg_kernel_launch_count(void);

/* Human-readable name of a status code (static storage). */
const char* gmg_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* GMG_H */

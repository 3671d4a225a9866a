// Host-visible launchers of the CUDA kernels (internal to the library; the
// public C ABI is include/gmg.h).  Every launcher enqueues on `stream` and
// returns a gmg_status code.
#pragma once
#include <cuda_runtime.h>

#include "per_device.h"

#include <cstdint>

namespace gmg {

// Geometry of one level vector: N nodes per direction, pitches in elements.
struct LevelGeom {
  int dim, k, n;      // dimension, degree, cells per direction
  int N;              // nodes per direction = n k + 1
  int py;             // element stride of the y index
  long long pz;       // element stride of the z index (3D)
};

// One colour of the patch sweep.  Patches of colour c sit at vertices
// v_a = first[a] + 2 i_a, i_a < count[a] (first[a] = 1 if bit a of c is
// set, else 2).
struct PatchLaunch {
  LevelGeom g;
  int first[3];
  int count[3];
  int n_patches;
  double sb;          // h^{2-d}: scales b to the unit-cell operator
  double omega;       // damping of the scatter
  // optional list of patches (lexicographic ids within the colour); patch
  // number i of the launch is plist[i] when plist != nullptr
  const int* plist;
  // 0: combined local residual + solve (Algorithm 4);
  // 1: solve only, b holds the global residual r = b - A u (Algorithm 3)
  int mode;
};

// One launch of the sweep kernel covers one colour of up to kMaxTable
// problems (or level slices): entry i owns groups [group_begin, group_begin
// + ceil(n_patches / PPC)) of the launch.  Passed by value as a kernel
// parameter.
constexpr int kMaxTable = 64;
struct PatchEntry {
  long long py, pz;     // pitches of the level vectors
  int N;                // nodes per direction
  int first[3], count[3];
  int n_patches;
  int group_begin;
  double sb;            // h^{2-d}
  void* u;              // level vector updated in place
  const void* b;        // right-hand side (or residual in solve-only mode)
  const int* plist;     // optional patch list (lexicographic ids in the colour)
};
struct PatchTable {
  int n;                // entries used
  int total_groups;
  int mode;             // 0 combined (Algorithm 4), 1 solve only (Algorithm 3)
  double omega;
  PatchEntry e[kMaxTable];
};

// y = alpha * (A_ref x) + beta * bvec on owned interior nodes, where A_ref is
// the level operator assembled from unit cells (A = h^{d-2} A_ref).
struct ApplyLaunch {
  LevelGeom g;
  double alpha, beta;
  // FP64 3D: four level vectors of workspace (pz * N doubles each) for the
  // halo-free three-pass form, or null for the tile kernel
  void* ws = nullptr;
  // tile kernel shape in 3D at degrees 3, 4, 7 (gmg_set_operator_tile):
  // 0 the default of the precision and degree, 1 cubes, 2 flat 4x4x1,
  // 3 flat 8x4x1 (shapes whose tile does not fit in shared memory fall back
  // to the default); every shape evaluates the same sums in the same order
  int tile = 0;
};
// whether launch_apply<double> uses the three-pass form in 3D at degree k
// when given a workspace
bool staged_apply_preferred(int dim, int k);

// One 1D contraction along `axis` of a (up to) 3-index array:
//   out[o + out_off] (+)= sum_w coef[(o_ax % R) * W + w] * in[i]
// where along the contracted axis the input index is
//   ((o_ax + shift) / R) * S + off + w   (skipped if outside [0, in_dim[axis]))
// with coefficient row (o_ax + shift) % R, and along the other axes it is
// o + in_off.  Output counts per axis are cnt[]; strides are in elements.
struct AxisOp {
  int axis;
  int cnt[3];
  int in_dim[3];
  long long in_stride[3];
  int in_off[3];
  long long out_stride[3];
  int out_off[3];
  int R, S, off, W;
  int shift;
  int accumulate;
};

// Device flag of the bounded device-side waits (TMA gathers, tensor-core
// MMA completion): set to GMG_ERR_TIMEOUT by a kernel whose wait expired;
// read and cleared by gmg_tc_status.  One flag per device: the address
// returned is that of the current device's copy.
int* device_wait_flag();

// Host-side count of kernel launches made by this library (all launchers
// call count_launch once per kernel they enqueue).
void count_launch(int n = 1);
long long launch_count();

template <typename T>
int upload_patch_tables(int k, const double* Mp, const double* Kp, const double* That,
                        const double* Mc, const double* Kc, cudaStream_t s);
template <typename T>
int launch_patch_colour(const PatchLaunch& pl, T* u, const T* b, const T* dinv, cudaStream_t s);
// one colour of a coarse level with the one-output-per-thread kernel (FP64 problems,
// mode 0, no patch list; GMG_ERR_UNSUPPORTED otherwise)
template <typename T>
int launch_patch_small(const PatchLaunch& pl, T* u, const T* b, const T* dinv, cudaStream_t s);
// several problems / slices of one colour in one launch (all of dimension
// dim and degree k); ppc = 0 picks the default patches per CTA, else one of
// the tuned variants 1, 2, 4 (3D FP32 only; others use the default)
template <typename T>
int launch_patch_table(int dim, int k, const PatchLaunch* pls, T* const* us, const T* const* bs,
                       int n, const T* dinv, int ppc, cudaStream_t s);
// Tensor-core sweep (patch_tc.cu): 3D, FP32 data, degrees 4..7, combined
// mode only (GMG_ERR_UNSUPPORTED otherwise).
bool tc_supported(int dim, int k);
int upload_tc_tables(int k, const double* Mp, const double* Kp, const double* That);
// split: data operands as TF32 hi + remainder (GMG_FP32_TC), else TF32 once
int launch_patch_tc(const PatchLaunch& pl, float* u, const float* b, const float* dinv, bool split,
                    cudaStream_t s);
int launch_patch_table_tc(int dim, int k, const PatchLaunch* pls, float* const* us, const float* const* bs,
                          int n, const float* dinv, bool split, cudaStream_t s);

// Shared-face form of the 3D sweep of one whole colour (face kernel, then
// patch kernel; faces: a buffer of face_buffer_elems<T>(pl) elements).
// GMG_ERR_UNSUPPORTED when the form does not apply (2D, k < 3, solve-only
// mode, a patch list, or a b vector the TMA box cannot address).
template <typename T>
int launch_patch_faces(const PatchLaunch& pl, T* u, const T* b, const T* dinv, T* faces, cudaStream_t s);
template <typename T>
long long face_buffer_elems(const PatchLaunch& pl);

template <typename T>
int launch_apply(const ApplyLaunch& al, const T* x, T* y, const T* bvec, cudaStream_t s);

// Variable-coefficient kernels (var_f64.cu / var_f32.cu; degree <= 3).
template <typename T>
int upload_var_tables(int k, const double* Mc, const double* Kc, const double* That);
// y = alpha sum_c a_c A_c x + beta bvec on interior nodes (bvec may be null)
template <typename T>
int launch_apply_var(const LevelGeom& g, long long n_elems, const T* x, T* y, const T* bvec,
                     double alpha, double beta, const T* coef, cudaStream_t s);
// vscale: per interior vertex of the level (x fastest), the patch's
// geometric-mean coefficient abar and its FD damping theta (two values)
template <typename T>
int launch_patch_var(const PatchLaunch& pl, T* u, const T* b, const T* coef, const T* vscale, const T* dinv,
                     const float* corr, int rank, cudaStream_t s);

// x = Ainv b on the interior nodes of a level (Ainv dense FP64, interior
// nodes numbered x fastest); the coarse solve of variable-coefficient problems
template <typename T>
int launch_dense_solve(const LevelGeom& g, const double* Ainv, int n_int, const T* b, T* x,
                       cudaStream_t s);

template <typename T>
int launch_axis_op(const AxisOp& op, const T* in, T* out, const T* coef, cudaStream_t s);
// The transfer passes of FP64 problems in double-float arithmetic
// (transfer_df.cu): op is the prolongation (restrict_op false) or
// restriction pass that launch_axis_op would run, table its coefficient
// table (host FP64, rows of op.W), n_cells the coarse cells along the pass
// axis; in / out are doubles, or float pairs where in_df / out_df.
// transfer_table_df_ok checks that a table has the zero pattern the kernel
// relies on.
int transfer_table_df_ok(int k, bool restrict_op, const double* table);
int launch_transfer_df(const AxisOp& op, int k, int n_cells, bool restrict_op, const double* table,
                       const void* in, bool in_df, void* out, bool out_df, cudaStream_t s);
template <typename T>
int launch_scale(long long n, T* x, const T* d, cudaStream_t s);  // x *= d
// element-type conversions over n elements
int launch_convert_f64_f32(long long n, const double* x, float* y, cudaStream_t s);
int launch_convert_f32_f64(long long n, const float* x, double* y, cudaStream_t s);

// FP64 reductions: partial sums per block into `partial` (>= kReduceBlocks
// doubles) then a single-block sum into `result` (device scalar).
constexpr int kReduceBlocks = 1024;
int launch_dot(long long n, const double* x, const double* y, double* partial, double* result,
               cudaStream_t s);
// x += alpha p, r -= alpha q with alpha = num/den read from device scalars;
// also the partial sums of r.r into `partial` and their total into `result`.
int launch_cg_update(long long n, double* x, double* r, const double* p, const double* q,
                     const double* num, const double* den, double* partial, double* result,
                     cudaStream_t s);
// p = z + (num/den) p
int launch_cg_direction(long long n, double* p, const double* z, const double* num,
                        const double* den, cudaStream_t s);

// Segmented (per-problem) FP64 vector kernels over concatenated vectors.  The
// concatenation is cut into chunks; chunk c covers elements [start[c],
// start[c] + len[c]) and belongs to problem owner[c]; problem i owns chunks
// [begin[i], begin[i+1]).  Per-problem scalars are arrays indexed by problem.
struct Segments {
  int n_chunks = 0;
  int n_problems = 0;
  const long long* start = nullptr;  // device arrays
  const int* len = nullptr;
  const int* owner = nullptr;
  const int* begin = nullptr;        // n_problems + 1
};
constexpr int kSegChunk = 8192;
// result[i] = x_i . y_i
int launch_seg_dot(const Segments& sg, const double* x, const double* y, double* partial,
                   double* result, cudaStream_t s);
// for active problems: x += (num/den) p, r -= (num/den) q; result[i] = r_i . r_i
int launch_seg_cg_update(const Segments& sg, double* x, double* r, const double* p, const double* q,
                         const double* num, const double* den, const int* active, double* partial,
                         double* result, cudaStream_t s);
// for active problems: p = z + (num/den) p
int launch_seg_cg_direction(const Segments& sg, double* p, const double* z, const double* num,
                            const double* den, const int* active, cudaStream_t s);

}  // namespace gmg

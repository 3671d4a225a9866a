// Patch sweep and level operator kernels in double precision.
#define GMG_T double
#define GMG_NS f64
#include "patch_kernels.cuh"
#include "patch_launch.cuh"
#include "face_kernels.cuh"
#include "small_kernels.cuh"

namespace gmg {

bool staged_apply_preferred(int dim, int k) { return dim == 3 && f64::staged_apply_degree(k); }

}  // namespace gmg

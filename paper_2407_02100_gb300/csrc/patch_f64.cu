// Patch sweep and level operator kernels in double precision.
#define GMG_T double
#define GMG_NS f64
#include "patch_kernels.cuh"
#include "patch_launch.cuh"

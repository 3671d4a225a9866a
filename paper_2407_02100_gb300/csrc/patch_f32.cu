// Patch sweep and level operator kernels in single precision.
#define GMG_T float
#define GMG_NS f32
#include "patch_kernels.cuh"
#include "patch_launch.cuh"
#include "face_kernels.cuh"
#include "small_kernels.cuh"

// Variable-coefficient operator and patch smoother in single precision.
#define GMG_T float
#define GMG_NS vf32
#include "var_kernels.cuh"
#include "var_launch.cuh"

// Variable-coefficient operator and patch smoother in double precision.
#define GMG_T double
#define GMG_NS vf64
#include "var_kernels.cuh"
#include "var_launch.cuh"

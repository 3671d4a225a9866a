// Patch sweep and level operator kernels in double precision.
#define GMG_T double
#define GMG_NS f64
#include "patch_kernels.cuh"
#include "patch_launch.cuh"
#include "face_kernels.cuh"

namespace gmg {

int launch_patch_faces(const PatchLaunch& pl, double* u, const double* b, const double* dinv, double* faces,
                       cudaStream_t s) {
  if (pl.g.dim != 3 || pl.g.k < 3 || pl.g.k > 8 || pl.mode != 0 || pl.plist || !faces)
    return GMG_ERR_UNSUPPORTED;
  if (!tma_vector_ok(b, 8, 3, pl.g.py, pl.g.pz)) return GMG_ERR_UNSUPPORTED;
  if (pl.n_patches <= 0) return GMG_OK;
  switch (pl.g.k) {
    case 3: return f64::face_sweep_impl<3>(pl, u, b, dinv, faces, s);
    case 4: return f64::face_sweep_impl<4>(pl, u, b, dinv, faces, s);
    case 5: return f64::face_sweep_impl<5>(pl, u, b, dinv, faces, s);
    case 6: return f64::face_sweep_impl<6>(pl, u, b, dinv, faces, s);
    case 7: return f64::face_sweep_impl<7>(pl, u, b, dinv, faces, s);
    default: return f64::face_sweep_impl<8>(pl, u, b, dinv, faces, s);
  }
}

long long face_buffer_elems(const PatchLaunch& pl) { return f64::face_buffer_elems(pl); }

bool staged_apply_preferred(int dim, int k) { return dim == 3 && f64::staged_apply_degree(k); }

}  // namespace gmg

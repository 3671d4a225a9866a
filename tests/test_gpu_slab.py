"""Skewed-slab schedule of the sweep: one launch per (slab, colour) instead of
one per colour.  Every patch reads the values Algorithm 4 gives it for any
slab width, so the GPU results must be bit-identical to the one-launch-per-
colour sweep, in both colour orders, for every precision path (the patch
kernels compute a patch the same way however patches are grouped)."""
import numpy as np
import pytest

from paper_2407_02100_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gmg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2407_02100_gb300 import build, gmg as g
    build.build()
    return g


CASES = [(2, 2, 12, 0), (3, 2, 6, 0), (3, 3, 8, 0), (3, 4, 5, 1), (3, 4, 5, 2), (3, 2, 9, 1)]


@pytest.mark.parametrize("dim,k,n,prec", CASES)
@pytest.mark.parametrize("reverse", [False, True])
def test_sweep_is_identical_for_every_slab_width(gmg, dim, k, n, prec, reverse):
    u0 = inputs.random_nodal(dim, k, n, 4001)
    b = inputs.random_nodal(dim, k, n, 4002)
    # small FP64 levels take the coarse-level kernel and no slabs:
    # turn it off so that these sizes exercise the slab schedule
    P = gmg.Problem(dim, k, n, n_levels=1, precision=prec, small_sweep=0)
    # slabs launch the closure-form kernel on patch lists: the reference is
    # the whole-colour closure form (FP64 3D problems default to shared faces)
    gmg.gmg_set_shared_faces(P.h, False)
    bd = P.to_device(b)
    ref = P.to_device(u0)
    gmg.gmg_smooth(P.h, 0, ref, bd, 1, reverse)
    ref = P.from_device(ref)
    for w in (1, 2, 3):
        gmg.gmg_set_slab_width(P.h, w)
        assert gmg.gmg_slab_width(P.h, 0) == w
        ud = P.to_device(u0)
        gmg.gmg_smooth(P.h, 0, ud, bd, 1, reverse)
        assert np.array_equal(P.from_device(ud), ref), w
    gmg.gmg_set_slab_width(P.h, 0)
    assert gmg.gmg_slab_width(P.h, 0) == 0


@pytest.mark.parametrize("prec", [0, 1])
def test_pcg_is_identical_with_slabs(gmg, prec):
    import torch
    dim, k, n, L = 3, 2, 16, 3
    b = inputs.random_nodal(dim, k, n, 4101)
    sols = []
    for w in (0, 2, -1):
        P = gmg.Problem(dim, k, n, n_levels=L, precision=prec, small_sweep=0)
        gmg.gmg_set_slab_width(P.h, w)
        u = P.zeros(dtype=torch.float64)
        _, st = gmg.cg_gmg_solve(P.h, u, P.to_device(b, dtype=torch.float64), 1e-10, 50)
        sols.append((st.iterations, P.from_device(u)))
    for its, x in sols[1:]:
        assert its == sols[0][0]
        assert np.array_equal(x, sols[0][1])


def test_small_fp64_levels_take_no_slabs(gmg):
    """A level whose colours all take the coarse-level kernel (FP64)
    keeps no slab schedule, so a slab width cannot change its sweep; turning
    the kernel off gives the level its slabs back."""
    P = gmg.Problem(3, 2, 8, n_levels=1)            # 343 patches, 64 per colour at most
    gmg.gmg_set_slab_width(P.h, 2)
    assert gmg.gmg_small_sweep(P.h) == 256          # the default up to degree 4
    assert gmg.gmg_small_sweep(gmg.Problem(3, 5, 4, n_levels=1).h) == 0
    assert gmg.gmg_slab_width(P.h, 0) == 0
    gmg.gmg_set_small_sweep(P.h, 0)
    assert gmg.gmg_slab_width(P.h, 0) == 2
    gmg.gmg_set_small_sweep(P.h, 64)                # the largest colour fits again
    assert gmg.gmg_slab_width(P.h, 0) == 0
    with pytest.raises(gmg.GmgError):
        gmg.gmg_set_small_sweep(P.h, -1)
    P.close()

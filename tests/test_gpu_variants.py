"""GPU parity of the paper's other loop organisations: Algorithm 3 (separated,
colourised: one global residual per colour, then the colour's local solves)
and Algorithm 5 (Z-curve batches of n_B patches per colour, batch-major),
against the oracle's own implementations of both, and their limits: Algorithm
3 equals Algorithm 4 up to rounding, Algorithm 5 with n_B >= the largest
colour is Algorithm 4 exactly."""
import numpy as np
import pytest

from oracle.mesh import Mesh
from oracle.smoother import PatchSmoother, sweep_alg3, sweep_alg5
from paper_2407_02100_gb300 import inputs

pytestmark = pytest.mark.gpu
RTOL = 1e-12


@pytest.fixture(scope="module")
def gmg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2407_02100_gb300 import build, gmg as g
    build.build()
    return g


def close(got, ref, what):
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err <= RTOL and np.abs(got - ref).max() <= 10 * RTOL * np.abs(ref).max(), f"{what}: {err:.3e}"


@pytest.mark.parametrize("dim,k,n", [(2, 2, 9), (2, 5, 6), (3, 2, 6), (3, 4, 5)])
@pytest.mark.parametrize("reverse", [False, True])
def test_separated_sweep(gmg, dim, k, n, reverse):
    m = Mesh(dim, k, n)
    s = PatchSmoother(m)
    P = gmg.Problem(dim, k, n, n_levels=1)
    u0 = inputs.random_nodal(dim, k, n, 1401)
    b = inputs.random_nodal(dim, k, n, 1402)
    ud = P.to_device(u0)
    gmg.gmg_smooth_variant(P.h, 0, ud, P.to_device(b), gmg.GMG_SWEEP_SEPARATED, 1, reverse)
    close(P.from_device(ud), sweep_alg3(m, m.assemble(), s, u0, b, reverse), "Algorithm 3")


@pytest.mark.parametrize("dim,k,n", [(2, 2, 11), (3, 1, 9), (3, 3, 6)])
@pytest.mark.parametrize("n_b", [1, 3, 17])
def test_batched_sweep(gmg, dim, k, n, n_b):
    m = Mesh(dim, k, n)
    s = PatchSmoother(m)
    P = gmg.Problem(dim, k, n, n_levels=1)
    u0 = inputs.random_nodal(dim, k, n, 1501)
    b = inputs.random_nodal(dim, k, n, 1502)
    ud = P.to_device(u0)
    gmg.gmg_smooth_variant(P.h, 0, ud, P.to_device(b), gmg.GMG_SWEEP_BATCHED, n_b, False)
    close(P.from_device(ud), sweep_alg5(s, u0, b, n_b), f"Algorithm 5, n_B={n_b}")


def test_batched_with_whole_colours_is_algorithm4_bitwise(gmg):
    dim, k, n = 3, 3, 8
    # Algorithm 5 batches use the closure form: so must the reference sweep
    # (no shared faces, no coarse-level kernel)
    P = gmg.Problem(dim, k, n, n_levels=1, small_sweep=0)
    gmg.gmg_set_shared_faces(P.h, False)
    u0 = inputs.random_nodal(dim, k, n, 1601)
    bd = P.to_device(inputs.random_nodal(dim, k, n, 1602))
    a, c = P.to_device(u0), P.to_device(u0)
    gmg.gmg_smooth_variant(P.h, 0, a, bd, gmg.GMG_SWEEP_BATCHED, 10 ** 9, False)
    gmg.gmg_smooth(P.h, 0, c, bd, 1, False)
    assert np.array_equal(P.from_device(a), P.from_device(c))

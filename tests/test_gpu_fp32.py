"""GPU parity of the FP32 path (smoother, operator, transfer and V-cycle in
single precision) against the FP64 oracle, and of the mixed-precision solve
(FP32 V-cycle preconditioning FP64 CG) against the FP64 solve.

Tolerances: single precision rounds at u = 6e-8; a sweep applies the patch
inverses whose condition numbers reach ~1e3 for k <= 4, so the sweep and the
V-cycle are compared at 1e-5 relative (2-norm) and the operator at 1e-6.  The
outer CG is FP64, so the mixed solve must still reach 1e-10 and match the FP64
oracle solution to 1e-8, with at most one more iteration than the FP64 run."""
import numpy as np
import pytest

from oracle.mesh import Mesh
from oracle.multigrid import Multigrid
from oracle.smoother import PatchSmoother
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


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("dim,k,n", [(2, 2, 20), (2, 5, 7), (3, 2, 10), (3, 4, 5), (3, 7, 3)])
def test_apply_fp32(gmg, dim, k, n):
    m = Mesh(dim, k, n)
    P = gmg.Problem(dim, k, n, n_levels=1, precision=gmg.GMG_FP32)
    x = inputs.random_nodal(dim, k, n, 1001)
    y = P.zeros()
    gmg.gmg_apply_operator(P.h, 0, P.to_device(x), y)
    assert rel(P.from_device(y), m.assemble() @ x) < 1e-6


@pytest.mark.parametrize("dim,k,n", [(2, 2, 16), (2, 4, 6), (3, 2, 7), (3, 4, 5), (3, 5, 4)])
def test_sweep_fp32(gmg, dim, k, n):
    m = Mesh(dim, k, n)
    s = PatchSmoother(m)
    P = gmg.Problem(dim, k, n, n_levels=1, precision=gmg.GMG_FP32)
    u0 = inputs.random_nodal(dim, k, n, 1101)
    b = inputs.random_nodal(dim, k, n, 1102)
    ud = P.to_device(u0)
    gmg.gmg_smooth(P.h, 0, ud, P.to_device(b), 1, False)
    assert rel(P.from_device(ud), s.sweep(u0, b)) < 1e-5


@pytest.mark.parametrize("dim,k,n,L", [(2, 2, 32, 3), (3, 2, 8, 3), (3, 4, 4, 2)])
def test_vcycle_fp32(gmg, dim, k, n, L):
    mg = Multigrid(dim, k, n, L)
    P = gmg.Problem(dim, k, n, n_levels=L, precision=gmg.GMG_FP32)
    b = inputs.random_nodal(dim, k, n, 1201)
    x = P.zeros()
    gmg.gmg_vcycle(P.h, x, P.to_device(b))
    assert rel(P.from_device(x), mg.vcycle(b)) < 1e-5


@pytest.mark.parametrize("dim,k,n,L", [(2, 2, 32, 3), (2, 4, 16, 3), (3, 2, 8, 3), (3, 4, 8, 3)])
def test_mixed_precision_pcg(gmg, dim, k, n, L):
    import torch
    b = inputs.random_nodal(dim, k, n, 1301)
    P64 = gmg.Problem(dim, k, n, n_levels=L, precision=gmg.GMG_FP64)
    P32 = gmg.Problem(dim, k, n, n_levels=L, precision=gmg.GMG_FP32)
    bd = P64.to_device(b, dtype=torch.float64)
    u64 = P64.zeros(dtype=torch.float64)
    u32 = P32.zeros(dtype=torch.float64)
    _, s64 = gmg.cg_gmg_solve(P64.h, u64, bd, 1e-10, 100)
    _, s32 = gmg.cg_gmg_solve(P32.h, u32, bd, 1e-10, 100)
    assert s32.converged and s32.relative_residual <= 1e-10
    assert s32.iterations <= s64.iterations + 1, (s32.iterations, s64.iterations)
    xo, its, _ = Multigrid(dim, k, n, L).pcg(b, rtol=1e-10)
    assert rel(P32.from_device(u32), xo) < 1e-8
    assert rel(P64.from_device(u64), xo) < 1e-8


@pytest.mark.parametrize("dim,k,n", [(3, 4, 4), (2, 3, 8), (3, 2, 6)])
def test_fp32_problem_solves_the_coarse_level_in_fp64(gmg, dim, k, n):
    """Single-precision problems keep FP64 for the coarse solve: with a
    right-hand side that is exactly representable in FP32 the only rounding
    left is that of the FP32 result (6e-8 relative), whereas an FP32
    fast-diagonalisation solve would lose about cond(A_0) times more."""
    P = gmg.Problem(dim, k, n, n_levels=1, precision=gmg.GMG_FP32)
    b = inputs.random_nodal(dim, k, n, 5101).astype(np.float32).astype(np.float64)
    x = P.zeros()
    gmg.gmg_coarse_solve(P.h, P.to_device(b), x)
    ref = Multigrid(dim, k, n, 1).vcycle(b)
    assert rel(P.from_device(x), ref) < 3e-7

"""GPU parity of the variable-coefficient path (-div(a grad u), one
coefficient per cell, lognormal random field) against the oracle: operator,
sweep with the mean-coefficient fast-diagonalisation local solver, coarse
solve, V-cycle and PCG.  Tolerances as for the constant-coefficient path in
FP64 (1e-12; the operator accumulates with atomics, so only rounding order
differs) and 1e-5 in FP32."""
import numpy as np
import pytest

from oracle.mesh import Mesh
from oracle.varcoef import VarMultigrid, VarPatchSmoother
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


@pytest.mark.parametrize("dim,k,n", [(2, 1, 9), (2, 3, 6), (3, 1, 6), (3, 2, 5), (3, 3, 4)])
@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-5)])
def test_var_apply(gmg, dim, k, n, precision, tol):
    m = Mesh(dim, k, n)
    coef = inputs.lognormal_coefficient(dim, n, 11)
    P = gmg.Problem(dim, k, n, n_levels=1, precision=precision)
    gmg.gmg_set_coefficient(P.h, coef)
    x = inputs.random_nodal(dim, k, n, 12)
    y = P.zeros()
    gmg.gmg_apply_operator(P.h, 0, P.to_device(x), y)
    assert rel(P.from_device(y), m.assemble(coef) @ x) < tol


@pytest.mark.parametrize("dim,k,n", [(2, 2, 7), (2, 3, 6), (3, 1, 6), (3, 2, 5), (3, 3, 4)])
@pytest.mark.parametrize("reverse", [False, True])
def test_var_sweep_fd_mean(gmg, dim, k, n, reverse):
    m = Mesh(dim, k, n)
    coef = inputs.lognormal_coefficient(dim, n, 13)
    P = gmg.Problem(dim, k, n, n_levels=1)
    gmg.gmg_set_coefficient(P.h, coef)
    u0 = inputs.random_nodal(dim, k, n, 14)
    b = inputs.random_nodal(dim, k, n, 15)
    ud = P.to_device(u0)
    gmg.gmg_smooth(P.h, 0, ud, P.to_device(b), 1, reverse)
    ref = VarPatchSmoother(m, coef, "fd_mean").sweep(u0, b, reverse)
    assert rel(P.from_device(ud), ref) < 1e-12


# The mean-coefficient FD local solver is only approximate; its per-patch
# damping keeps every patch update an energy decrease, so the V-cycle stays
# positive definite at omega = 1 even for sigma = 1 fields on coarse meshes.
@pytest.mark.parametrize("dim,k,n,L,sigma,omega", [(2, 2, 16, 3, 1.0, 1.0), (3, 2, 8, 3, 1.0, 1.0),
                                                   (3, 3, 4, 2, 1.0, 1.0), (3, 2, 8, 3, 0.5, 0.7)])
def test_var_vcycle_and_pcg(gmg, dim, k, n, L, sigma, omega):
    import torch
    coef = inputs.lognormal_coefficient(dim, n, 16, sigma=sigma)
    mg = VarMultigrid(dim, k, n, L, coef, "fd_mean", omega=omega)
    P = gmg.Problem(dim, k, n, n_levels=L, damping=omega)
    gmg.gmg_set_coefficient(P.h, coef)
    b = inputs.random_nodal(dim, k, n, 17)
    x = P.zeros()
    gmg.gmg_vcycle(P.h, x, P.to_device(b))
    assert rel(P.from_device(x), mg.vcycle(b)) < 1e-11
    u = P.zeros(dtype=torch.float64)
    _, st = gmg.cg_gmg_solve(P.h, u, P.to_device(b, dtype=torch.float64), 1e-10, 100)
    xo, its = mg.pcg(b, 1e-10)
    assert st.converged and abs(st.iterations - its) <= 1, (st.iterations, its)
    assert rel(P.from_device(u), xo) < 1e-8


def test_overdamped_indefinite_case_reports_breakdown(gmg):
    """omega = 2.5 makes the smoother diverge (spectrum of the damped update
    above 2): the V-cycle is indefinite and the solver returns
    GMG_ERR_BREAKDOWN (a status, never a trap)."""
    import torch
    dim, k, n = 2, 2, 16
    coef = inputs.lognormal_coefficient(dim, n, 16)
    P = gmg.Problem(dim, k, n, n_levels=3, damping=2.5)
    gmg.gmg_set_coefficient(P.h, coef)
    b = P.to_device(inputs.random_nodal(dim, k, n, 17), dtype=torch.float64)
    u = P.zeros(dtype=torch.float64)
    st, _ = gmg.cg_gmg_solve(P.h, u, b, 1e-10, 50, raise_on_error=False)
    assert st in (-5, -6)


def test_var_rejects_high_degree(gmg):
    P = gmg.Problem(3, 4, 4, n_levels=1)
    with pytest.raises(gmg.GmgError) as e:
        gmg.gmg_set_coefficient(P.h, np.ones(64))
    assert e.value.status == -7


@pytest.mark.parametrize("dim,k,n,prec", [(3, 3, 4, 1), (3, 2, 6, 0), (2, 3, 8, 1)])
def test_var_sweep_tma_and_elementwise_gathers_agree(gmg, dim, k, n, prec):
    """A solution vector 4 or 8 bytes off 16-byte alignment cannot be read by
    TMA boxes: the variable-coefficient sweep then gathers element by
    element.  Both feed the same arithmetic: bit-identical results."""
    import torch
    P = gmg.Problem(dim, k, n, n_levels=1, precision=prec)
    gmg.gmg_set_coefficient(P.h, inputs.lognormal_coefficient(dim, n, 61))
    u0 = inputs.random_nodal(dim, k, n, 62)
    bd = P.to_device(inputs.random_nodal(dim, k, n, 63))
    ua = P.to_device(u0)
    gmg.gmg_smooth(P.h, 0, ua, bd, 1, False)
    buf = torch.zeros(ua.numel() + 1, dtype=ua.dtype, device=ua.device)
    um = buf[1:]
    um.copy_(P.to_device(u0))
    gmg.gmg_smooth(P.h, 0, um, bd, 1, False)
    assert gmg.gmg_tc_status() == 0
    assert torch.equal(ua, um)

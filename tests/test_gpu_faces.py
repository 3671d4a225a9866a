"""Shared-face form of the 3D sweep (degrees >= 3; FP64 and FP32 problems)
through the C ABI.

The local solver is exact, so a patch's new interior depends on its closure
boundary only; the form evaluates each face plane's two-dimensional
sum-factorised terms once per colour and lets both patches that share the
plane read them.  It is the same method as the closure form: both are
compared with the oracle (FP64: relative 1e-12; FP32, used from k = 7: no
more than twice the closure form's own FP32 error, both about
eps_32 cond(A_j), cond(A_j) = 174 at k = 7) and with each other."""
import numpy as np
import pytest

from oracle.mesh import Mesh
from oracle.smoother import PatchSmoother
from paper_2407_02100_gb300 import inputs

FP32_RTOL = 1e-5
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
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def test_form_is_used_where_it_applies(gmg):
    assert gmg.gmg_shared_faces(gmg.Problem(3, 4, 4, n_levels=1).h) == 1
    assert gmg.gmg_shared_faces(gmg.Problem(3, 3, 4).h) == 1
    assert gmg.gmg_shared_faces(gmg.Problem(3, 2, 4, n_levels=1).h) == 0      # k < 3
    assert gmg.gmg_shared_faces(gmg.Problem(2, 4, 4, n_levels=1).h) == 0      # 2D
    assert gmg.gmg_shared_faces(gmg.Problem(3, 4, 4, n_levels=1, precision=gmg.GMG_FP32).h) == 0
    assert gmg.gmg_shared_faces(gmg.Problem(3, 7, 2, n_levels=1, precision=gmg.GMG_FP32).h) == 1
    assert gmg.gmg_shared_faces(gmg.Problem(3, 4, 4, n_levels=1, precision=gmg.GMG_FP32_TC).h) == 0
    P = gmg.Problem(3, 4, 4, n_levels=1)
    gmg.gmg_set_shared_faces(P.h, False)
    assert gmg.gmg_shared_faces(P.h) == 0
    gmg.gmg_set_shared_faces(P.h, True)
    assert gmg.gmg_shared_faces(P.h) == 1


# every degree of the form, even and odd cell counts (colours of unequal
# patch counts), single-patch meshes
FACE_CASES = [(3, 4), (3, 5), (3, 6), (4, 3), (4, 4), (5, 3), (6, 2), (7, 3), (8, 2), (4, 2)]


@pytest.mark.parametrize("k,n", FACE_CASES)
def test_each_colour_matches_oracle(gmg, k, n):
    m = Mesh(3, k, n)
    s = PatchSmoother(m)
    P = gmg.Problem(3, k, n, n_levels=1, small_sweep=0)  # these sizes would take the coarse-level kernel
    assert gmg.gmg_shared_faces(P.h) == 1
    u0 = inputs.random_nodal(3, k, n, 7101)
    b = inputs.random_nodal(3, k, n, 7102)
    bd = P.to_device(b)
    for c in range(m.n_colours):
        ud = P.to_device(u0)
        gmg.gmg_smooth_colour(P.h, 0, ud, bd, c)
        ref = s.colour_step(u0.copy(), b, c)
        got = P.from_device(ud)
        assert rel(got, ref) <= 1e-12, (c, rel(got, ref))
        assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max()


@pytest.mark.parametrize("k,n,omega", [(3, 5, 1.0), (4, 4, 0.7), (5, 3, 1.3), (7, 2, 0.8)])
@pytest.mark.parametrize("reverse", [False, True])
def test_face_and_closure_forms_agree(gmg, k, n, omega, reverse):
    """Two sweeps with each form from the same state: equal up to rounding,
    and equal to the oracle's (damped) sweeps."""
    P = gmg.Problem(3, k, n, n_levels=1, damping=omega, small_sweep=0)
    u0 = inputs.random_nodal(3, k, n, 7201)
    b = inputs.random_nodal(3, k, n, 7202)
    bd = P.to_device(b)
    out = []
    for on in (True, False):
        gmg.gmg_set_shared_faces(P.h, on)
        ud = P.to_device(u0)
        gmg.gmg_smooth(P.h, 0, ud, bd, 2, reverse)
        out.append(P.from_device(ud))
    gmg.gmg_set_shared_faces(P.h, True)
    assert rel(out[0], out[1]) <= 1e-13
    s = PatchSmoother(Mesh(3, k, n), omega)
    ref = s.sweep(s.sweep(u0, b, reverse=reverse), b, reverse=reverse)
    assert rel(out[0], ref) <= 1e-12


def test_unaligned_rhs_takes_the_closure_form(gmg):
    """A right-hand side whose base is not 16-byte aligned cannot be read by
    the TMA box of the form: the sweep falls back to the closure kernel with
    its element-wise gather, bit-identical to that kernel run directly."""
    import torch
    k, n = 4, 5
    P = gmg.Problem(3, k, n, n_levels=1, small_sweep=0)
    u0 = inputs.random_nodal(3, k, n, 7301)
    b = inputs.random_nodal(3, k, n, 7302)
    bb = P.to_device(b)
    buf = torch.zeros(bb.numel() + 1, dtype=bb.dtype, device=bb.device)
    bm = buf[1:]
    bm.copy_(bb)
    runs = []
    for on in (True, False):
        gmg.gmg_set_shared_faces(P.h, on)
        ud = P.to_device(u0)
        gmg.gmg_smooth(P.h, 0, ud, bm, 1, False)
        runs.append(ud)
    gmg.gmg_set_shared_faces(P.h, True)
    assert gmg.gmg_tc_status() == 0
    assert torch.equal(runs[0], runs[1])
    ref = PatchSmoother(Mesh(3, k, n)).sweep(u0, b)
    assert rel(P.from_device(runs[0]), ref) <= 1e-12


@pytest.mark.parametrize("k,n", [(3, 8), (4, 8)])
def test_pcg_iterations_and_solution(gmg, k, n):
    """GMG-PCG to 1e-10 with V(1,1) on every level: same iterations with
    either form, solutions equal to well below the tolerance."""
    import torch
    P = gmg.Problem(3, k, n)
    b = P.to_device(inputs.random_nodal(3, k, n, 7401), dtype=torch.float64)
    sols, its = [], []
    for on in (True, False):
        gmg.gmg_set_shared_faces(P.h, on)
        u = P.zeros(dtype=torch.float64)
        _, st = gmg.cg_gmg_solve(P.h, u, b, 1e-10, 100)
        assert st.converged == 1 and st.relative_residual <= 1e-10
        sols.append(P.from_device(u))
        its.append(st.iterations)
    gmg.gmg_set_shared_faces(P.h, True)
    assert its[0] == its[1]
    assert rel(sols[0], sols[1]) <= 1e-11


@pytest.mark.parametrize("k,n", [(7, 3), (8, 2), (7, 2), (7, 4)])
def test_fp32_each_colour_matches_oracle(gmg, k, n):
    """FP32 data (the oracle takes the FP32-rounded inputs): each colour step
    of the shared-face form (the FP32 default from k = 7) and of the closure
    form is within the FP32 sweep tolerance 1e-5 of the oracle (relative
    2-norm over all nodes, as for every FP32 sweep)."""
    m = Mesh(3, k, n)
    s = PatchSmoother(m)
    P = gmg.Problem(3, k, n, n_levels=1, precision=gmg.GMG_FP32)
    assert gmg.gmg_shared_faces(P.h) == 1
    u0 = inputs.random_nodal(3, k, n, 7501).astype(np.float32).astype(np.float64)
    b = inputs.random_nodal(3, k, n, 7502).astype(np.float32).astype(np.float64)
    bd = P.to_device(b)
    for c in range(m.n_colours):
        ref = s.colour_step(u0.copy(), b, c)
        err = []
        for on in (True, False):
            gmg.gmg_set_shared_faces(P.h, on)
            ud = P.to_device(u0)
            gmg.gmg_smooth_colour(P.h, 0, ud, bd, c)
            err.append(rel(P.from_device(ud), ref))
        gmg.gmg_set_shared_faces(P.h, True)
        assert max(err) <= FP32_RTOL, (c, err)


@pytest.mark.parametrize("k,n,omega", [(7, 3, 1.0), (7, 2, 0.8), (8, 2, 1.0)])
def test_fp32_face_and_closure_forms_agree(gmg, k, n, omega):
    P = gmg.Problem(3, k, n, n_levels=1, precision=gmg.GMG_FP32, damping=omega)
    u0 = inputs.random_nodal(3, k, n, 7601)
    bd = P.to_device(inputs.random_nodal(3, k, n, 7602))
    out = []
    for on in (True, False):
        gmg.gmg_set_shared_faces(P.h, on)
        ud = P.to_device(u0)
        gmg.gmg_smooth(P.h, 0, ud, bd, 2, False)
        out.append(P.from_device(ud))
    gmg.gmg_set_shared_faces(P.h, True)
    assert rel(out[0], out[1]) <= 3e-5


@pytest.mark.parametrize("k,n", [(7, 4)])
def test_fp32_mixed_pcg_iterations(gmg, k, n):
    """FP32 V-cycle inside FP64 CG: same iterations and solution (to the
    solve's tolerance) with either form of the FP32 sweep."""
    import torch
    P = gmg.Problem(3, k, n, precision=gmg.GMG_FP32)
    b = P.to_device(inputs.random_nodal(3, k, n, 7701), dtype=torch.float64)
    sols, its = [], []
    for on in (True, False):
        gmg.gmg_set_shared_faces(P.h, on)
        u = P.zeros(dtype=torch.float64)
        _, st = gmg.cg_gmg_solve(P.h, u, b, 1e-10, 100)
        assert st.converged == 1 and st.relative_residual <= 1e-10
        sols.append(P.from_device(u))
        its.append(st.iterations)
    gmg.gmg_set_shared_faces(P.h, True)
    assert abs(its[0] - its[1]) <= 1, its
    assert rel(sols[0], sols[1]) <= 1e-8

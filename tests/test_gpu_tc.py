"""Tensor-core sweep (3D, degrees 4..7, contractions as tcgen05 MMAs with
FP32 accumulation in tensor memory), in its two forms:

* GMG_FP32_TC: every factor split into its TF32 rounding and the TF32
  rounding of the remainder, three MMAs per product.  The products then
  carry about 22 significant bits, so the sweep is held to the FP32 kernel's
  bound, 1e-5 relative (2-norm) against the FP64 oracle, and the outer FP64
  CG to the FP64 iteration count + 1.
* GMG_FP32_TF32: data and matrices rounded to TF32 once (11 significant
  bits, unit roundoff 2^-11 = 4.9e-4); a sweep chains nine contractions per
  patch through the patch inverse, so it is held to 2e-2, and the outer CG
  must still reach 1e-10 (its iteration count is reported, not bounded: the
  smoother then depends on the rounding of its input).

The first test checks the MMA encoding alone (instruction and shared-memory
descriptors, TMEM read-back) on integer operands, for which TF32 products
and FP32 sums are exact, so any layout mistake shows as a wrong entry."""
import numpy as np
import pytest

from oracle.multigrid import Multigrid
from oracle.mesh import Mesh
from oracle.smoother import PatchSmoother
from paper_2407_02100_gb300 import inputs

pytestmark = pytest.mark.gpu
MODES = {"split": (2, 1e-5), "tf32": (3, 2e-2)}   # precision enum, sweep tolerance


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


def test_probe_is_exact_on_integers(gmg):
    rng = np.random.default_rng(7)
    A = rng.integers(-8, 9, (128, 16)).astype(np.float32)
    B = rng.integers(-8, 9, (32, 16)).astype(np.float32)
    D = gmg.gmg_tc_probe(A, B)
    np.testing.assert_array_equal(D, A @ B.T)


def test_expired_wait_is_reported_as_a_status(gmg):
    """The MMA completion is withheld until a short bounded wait has run out:
    the kernel returns GMG_ERR_TIMEOUT instead of hanging or trapping, the
    context stays usable and the next call succeeds."""
    rng = np.random.default_rng(8)
    A = rng.integers(-8, 9, (128, 16)).astype(np.float32)
    B = rng.integers(-8, 9, (32, 16)).astype(np.float32)
    st, D = gmg.gmg_tc_probe(A, B, force_timeout=True, raise_on_error=False)
    assert st == -8
    np.testing.assert_array_equal(D, A @ B.T)
    np.testing.assert_array_equal(gmg.gmg_tc_probe(A, B), A @ B.T)


@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("k,n", [(4, 4), (4, 5), (5, 3), (6, 3), (7, 3)])
@pytest.mark.parametrize("reverse", [False, True])
def test_tc_sweep_matches_oracle(gmg, mode, k, n, reverse):
    prec, tol = MODES[mode]
    m = Mesh(3, k, n)
    P = gmg.Problem(3, k, n, n_levels=1, precision=prec)
    u0 = inputs.random_nodal(3, k, n, 3101)
    b = inputs.random_nodal(3, k, n, 3102)
    ud = P.to_device(u0)
    gmg.gmg_smooth(P.h, 0, ud, P.to_device(b), 1, reverse)
    assert gmg.gmg_tc_status() == 0
    err = rel(P.from_device(ud), PatchSmoother(m).sweep(u0, b, reverse=reverse))
    print(f"{mode} k={k} n={n} reverse={reverse}: sweep vs FP64 oracle {err:.2e}")
    assert err < tol


@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("k,n", [(4, 16), (7, 6)])
def test_tc_sweep_tracks_fp32_kernel_on_many_patches(gmg, mode, k, n):
    """More patches than resident CTAs: every CTA walks several patches.
    Two sweeps double the single-sweep bound."""
    prec_tc, tol = MODES[mode]
    u0 = inputs.random_nodal(3, k, n, 3201)
    b = inputs.random_nodal(3, k, n, 3202)
    out = {}
    for prec in (gmg.GMG_FP32, prec_tc):
        P = gmg.Problem(3, k, n, n_levels=1, precision=prec)
        ud = P.to_device(u0)
        gmg.gmg_smooth(P.h, 0, ud, P.to_device(b), 2, False)
        out[prec] = P.from_device(ud)
    assert gmg.gmg_tc_status() == 0
    err = rel(out[prec_tc], out[gmg.GMG_FP32])
    print(f"{mode} k={k} n={n}: vs FP32 kernel after two sweeps {err:.2e}")
    assert err < 2 * tol


@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("k,n,L", [(4, 8, 3), (5, 6, 2), (7, 4, 2)])
def test_tc_pcg_reaches_fp64_accuracy(gmg, mode, k, n, L):
    import torch
    prec_tc = MODES[mode][0]
    b = inputs.random_nodal(3, k, n, 3301)
    its = {}
    for prec in (gmg.GMG_FP64, prec_tc):
        P = gmg.Problem(3, k, n, n_levels=L, precision=prec)
        u = P.zeros(dtype=torch.float64)
        _, st = gmg.cg_gmg_solve(P.h, u, P.to_device(b, dtype=torch.float64), 1e-10, 100)
        assert st.converged and st.relative_residual <= 1e-10
        its[prec] = (st.iterations, P.from_device(u))
    assert gmg.gmg_tc_status() == 0
    xo, it_o, _ = Multigrid(3, k, n, L).pcg(b, rtol=1e-10)
    assert rel(its[prec_tc][1], xo) < 1e-8
    print(f"{mode} k={k}: iterations FP64 {its[gmg.GMG_FP64][0]}, tensor cores {its[prec_tc][0]}, oracle {it_o}")
    if mode == "split":
        assert its[prec_tc][0] <= its[gmg.GMG_FP64][0] + 1


@pytest.mark.parametrize("mode", list(MODES))
def test_tc_batch_equals_single_problems(gmg, mode):
    """The batched launch (one kernel per colour over all problems) computes
    every patch exactly as the single-problem launch does."""
    k, ns = 4, [4, 6, 8]
    prec = MODES[mode][0]
    B = gmg.Batch(3, k, ns, precision=prec)
    us = [inputs.random_nodal(3, k, n, 3400 + i) for i, n in enumerate(ns)]
    bs = [inputs.random_nodal(3, k, n, 3500 + i) for i, n in enumerate(ns)]
    u = B.pack(us)
    gmg.gmg_batch_smooth(B.h, u, B.pack(bs), False)
    got = B.unpack(u)
    for i, n in enumerate(ns):
        P = gmg.Problem(3, k, n, precision=prec)
        ud = P.to_device(us[i])
        gmg.gmg_smooth(P.h, P.finest, ud, P.to_device(bs[i]), 1, False)
        assert np.array_equal(got[i], P.from_device(ud)), i
    assert gmg.gmg_tc_status() == 0

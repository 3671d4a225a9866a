"""Pins of the oracle's variable-coefficient smoother and of the learned
correction's analytic gradients."""
import numpy as np
import pytest

from oracle import learned
from oracle.mesh import Mesh
from oracle.smoother import PatchSmoother, colour_sorted_vertices, sweep_alg1
from oracle.varcoef import VarMultigrid, VarPatchSmoother, coarsen_coefficient
from paper_2407_02100_gb300 import inputs


def _rand(m, seed):
    return inputs.random_nodal(m.dim, m.k, m.n, seed)


def test_constant_coefficient_reduces_to_the_poisson_smoother():
    m = Mesh(3, 2, 4)
    u0, b = _rand(m, 1), _rand(m, 2)
    ref = PatchSmoother(m).sweep(u0, b)
    coef = np.ones((4, 4, 4))
    for mode in ("exact", "fd_mean"):
        np.testing.assert_allclose(VarPatchSmoother(m, coef, mode).sweep(u0, b), ref, atol=1e-12)
    # a constant c != 1 scales A by c: the solution of the local problems by 1/c
    c = 3.7
    got = VarPatchSmoother(m, c * coef, "fd_mean").sweep(u0 / 1.0, c * b)
    np.testing.assert_allclose(got, PatchSmoother(m).sweep(u0, b), atol=1e-11)


@pytest.mark.parametrize("dim,k,n", [(2, 2, 5), (3, 1, 4), (3, 2, 4)])
def test_exact_variable_smoother_equals_naive_loop(dim, k, n):
    """Algorithm 1 with the assembled variable-coefficient matrix pins the
    patch-to-cell coefficient mapping of the local blocks."""
    m = Mesh(dim, k, n)
    coef = inputs.lognormal_coefficient(dim, n, 3)
    A = m.assemble(coef)
    u0, b = _rand(m, 4), _rand(m, 5)
    got = VarPatchSmoother(m, coef, "exact").sweep(u0, b)
    ref = sweep_alg1(m, A, u0, b, colour_sorted_vertices(m))
    np.testing.assert_allclose(got, ref, atol=1e-11 * np.abs(ref).max())


def test_coarsening_is_geometric_mean():
    c = inputs.lognormal_coefficient(3, 4, 6)
    cc = coarsen_coefficient(c)
    assert cc.shape == (2, 2, 2)
    assert abs(cc[1, 0, 1] - np.prod(c[2:4, 0:2, 2:4]) ** (1 / 8)) < 1e-12


def test_variable_pcg_converges_and_fd_mean_is_weaker():
    dim, k, n = 2, 2, 16
    coef = inputs.lognormal_coefficient(dim, n, 7, sigma=1.0, corr_len=0.1)
    b = inputs.random_nodal(dim, k, n, 8)
    its = {}
    for mode in ("exact", "fd_mean"):
        mg = VarMultigrid(dim, k, n, 3, coef, mode)
        x, its[mode] = mg.pcg(b, 1e-10)
        A = mg.A[-1]
        assert np.linalg.norm(b - A @ x) <= 1e-10 * np.linalg.norm(b) * 1.01
    assert its["exact"] <= its["fd_mean"]


def test_learned_gradients_match_finite_differences():
    rng = np.random.default_rng(0)
    nf, nh, nint, rank, N = 4, 5, 9, 2, 7
    params = [0.3 * rng.standard_normal((nh, nf)), 0.1 * rng.standard_normal(nh),
              0.3 * rng.standard_normal((nint * rank + rank, nh)), 0.1 * rng.standard_normal(nint * rank + rank)]
    X = rng.standard_normal((N, nf))
    R = rng.standard_normal((N, nint))
    DFD = rng.standard_normal((N, nint))
    DEX = rng.standard_normal((N, nint))
    L, grads = learned.loss_and_grads(params, X, R, DFD, DEX, rank)
    assert abs(L - learned.loss(params, X, R, DFD, DEX, rank)) < 1e-14
    eps = 1e-6
    for P, G in zip(params, grads):
        for idx in [tuple(rng.integers(0, s) for s in P.shape) for _ in range(6)]:
            old = P[idx]
            P[idx] = old + eps
            lp = learned.loss(params, X, R, DFD, DEX, rank)
            P[idx] = old - eps
            lm = learned.loss(params, X, R, DFD, DEX, rank)
            P[idx] = old
            fd = (lp - lm) / (2 * eps)
            assert abs(fd - G[idx]) <= 1e-7 * max(1.0, abs(fd)), (idx, fd, G[idx])


@pytest.mark.parametrize("dim,k", [(2, 2), (3, 2), (3, 3)])
def test_fd_mean_damped_local_update_is_a_contraction(dim, k):
    """A_j <= max_c a_c h^{d-2} Ahat_j (cell-wise), so the damped local update
    B_j A_j with B_j = theta_j/abar h^{2-d} Ahat_j^{-1},
    theta_j = min(1, 1.8 abar / max a), has its spectrum in (0, 1.8]; the
    bound is attained up to the spectrum of the coefficient-ratio pencil, so
    some patch of a strongly varying field overshoots beyond 2 undamped."""
    n = 6
    m = Mesh(dim, k, n)
    coef = inputs.lognormal_coefficient(dim, n, 11, sigma=1.5, corr_len=0.05)
    sm = VarPatchSmoother(m, coef, "fd_mean")
    worst_undamped = 0.0
    for v in m.vertices():
        Abar, _, abar, theta = sm._patch(v)
        inner = m.patch_block()[1]
        Aj = Abar[:, inner]
        B = sm.local_solve(v, np.eye(Aj.shape[0]))
        lam = np.linalg.eigvals(B @ Aj).real
        assert lam.min() > 0 and lam.max() <= 1.8 + 1e-9
        worst_undamped = max(worst_undamped, lam.max() / theta)
    assert worst_undamped > 2.0

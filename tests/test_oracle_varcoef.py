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


def _reference_patch_inverse(dim, k, w):
    """Ahat(w)^{-1}: the exact patch inverse in reference units (unit cells),
    built from a two-cell-per-direction mesh at h = 1/2, independently of the
    smoother's own patch blocks, which are assembled at the mesh's h."""
    blk, inner = Mesh(dim, k, 2).patch_block(w)
    return np.linalg.inv(blk[:, inner] / 0.5 ** (dim - 2))


def _full_rank_corrections(m, coef, ref_inv):
    """Per patch the symmetric correction Ahat(w)^{-1} - theta Ahat^{-1} as
    eigenpairs (U, s), so U diag(s) U^T is the whole gap between the damped
    FD inverse and the exact one (Sec. 2.1: exact local solvers)."""
    from oracle.varcoef import patch_cell_coefs
    corr = {}
    for v in m.vertices():
        cc = patch_cell_coefs(m, coef, v)
        abar = np.exp(np.mean(np.log(cc)))
        w = cc / abar
        theta = min(1.0, 1.8 / np.max(w))
        gap = _reference_patch_inverse(m.dim, m.k, w) - theta * ref_inv
        s, U = np.linalg.eigh(0.5 * (gap + gap.T))
        corr[tuple(int(x) for x in v)] = (U, s)
    return corr


@pytest.mark.parametrize("dim,k,n", [(2, 2, 4), (2, 3, 6), (3, 2, 4), (3, 2, 6), (3, 1, 8)])
def test_full_rank_learned_correction_reproduces_exact_local_solves(dim, k, n):
    """With the full-rank correction Ahat(w)^{-1} - theta Ahat^{-1} the learned
    local solver is the exact one: (theta Ahat^{-1} + gap) h^{2-d} r / abar =
    (h^{d-2} abar Ahat(w))^{-1} r = A_j^{-1} r.  Meshes of different h in 3D
    pin the h^{2-d} factor and the division by abar; a dropped theta, a
    misplaced scale or a transposed U fails."""
    m = Mesh(dim, k, n)
    coef = inputs.lognormal_coefficient(dim, n, 41, sigma=1.0, corr_len=0.2)
    ex = VarPatchSmoother(m, coef, "exact")
    corr = _full_rank_corrections(m, coef, ex.ref_inv)
    lr = VarPatchSmoother(m, coef, "learned", corrections=corr)
    rng = np.random.default_rng(dim * 100 + n)
    for v in m.vertices()[:: max(1, len(m.vertices()) // 9)]:
        r = rng.standard_normal(len(ex.ref_inner))
        d_ex, d_lr = ex.local_solve(v, r), lr.local_solve(v, r)
        assert np.linalg.norm(d_lr - d_ex) <= 1e-12 * np.linalg.norm(d_ex)
    u0, b = _rand(m, 42), _rand(m, 43)
    ref = ex.sweep(u0, b)
    got = lr.sweep(u0, b)
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)


@pytest.mark.parametrize("dim,k", [(2, 2), (3, 2)])
def test_network_output_layout_and_loss_units(dim, k):
    """The perceptron's output vector o holds U row-major (U[i, q] = o[i R + q])
    then s; the loss compares theta FD r + U diag(s) U^T r with the exact
    reference-unit solve Ahat(w)^{-1} r.  Pins, on one patch:
    (1) at full rank R = m^d the loss is zero when o carries the eigenpairs
        of the gap Ahat(w)^{-1} - theta Ahat^{-1} laid out as documented;
    (2) at rank r < m^d (the r eigenpairs of largest modulus) the loss of an
        eigenvector residual u_q is 0 if q is kept and s_q^2 / ||DEX||^2 if
        not (Eckart-Young for the symmetric gap);
    (3) the same rank-r (U, s) in the smoother's learned mode gives the
        reference-unit update theta FD r + U diag(s) U^T r, i.e. the loss's
        prediction, once scaled by h^{2-d} / abar."""
    n = 4
    m = Mesh(dim, k, n)
    coef = inputs.lognormal_coefficient(dim, n, 44, sigma=1.2, corr_len=0.2)
    from oracle.varcoef import patch_cell_coefs
    fd = VarPatchSmoother(m, coef, "fd_mean")
    v = m.vertices()[len(m.vertices()) // 2]
    cc = patch_cell_coefs(m, coef, v)
    abar = np.exp(np.mean(np.log(cc)))
    w = cc / abar
    theta = min(1.0, 1.8 / np.max(w))
    exact_ref = _reference_patch_inverse(dim, k, w)
    gap = exact_ref - theta * fd.ref_inv
    s, U = np.linalg.eigh(0.5 * (gap + gap.T))
    nint = len(s)

    def pack(Ur, sr):
        return np.concatenate([Ur.reshape(-1), sr])[None, :]   # U[i, q] at i * R + q

    rng = np.random.default_rng(7)
    Rm = rng.standard_normal((3, nint))
    DFD = (theta * fd.ref_inv @ Rm.T).T
    DEX = (exact_ref @ Rm.T).T
    O = pack(U, s)
    params = [np.zeros((1, 1)), np.zeros(1), np.zeros((O.shape[1], 1)), O[0]]  # o = b2 exactly
    Lfull = learned.loss(params, np.zeros((3, 1)), Rm, DFD, DEX, nint)
    assert Lfull <= 1e-26
    # rank r: keep the r eigenpairs of largest |s|
    r = 3
    keep = np.argsort(-np.abs(s))[:r]
    Ur, sr = U[:, keep], s[keep]
    params_r = [np.zeros((1, 1)), np.zeros(1), np.zeros((nint * r + r, 1)), pack(Ur, sr)[0]]
    for q in range(nint):
        uq = U[:, q][None, :]
        dfd = (theta * fd.ref_inv @ uq.T).T
        dex = (exact_ref @ uq.T).T
        Lq = learned.loss(params_r, np.zeros((1, 1)), uq, dfd, dex, r)
        want = 0.0 if q in keep else s[q] ** 2 / np.sum(dex ** 2)
        assert abs(Lq - want) <= 1e-10 * max(want, 1e-20) + 1e-24, (q, Lq, want)
    # (3) the smoother's learned mode with the same rank-r correction
    lr = VarPatchSmoother(m, coef, "learned", corrections={tuple(int(x) for x in v): (Ur, sr)})
    rr = rng.standard_normal(nint)
    O_r = pack(Ur, sr)
    pred_ref = theta * fd.ref_inv @ rr + learned.correction(O_r, rr[None, :], nint, r)[0]
    got = lr.local_solve(v, rr / fd.hscale * abar)    # residual whose reference-unit form is rr
    assert np.linalg.norm(got - pred_ref) <= 1e-12 * np.linalg.norm(pred_ref)

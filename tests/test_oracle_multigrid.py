"""Pins of the oracle's multigrid layer: Galerkin identity of the embedding,
exact reproduction of coarse polynomials, O(h^{k+1}) L2 convergence of the
manufactured solution (App. A.2), symmetry of the V(1,1)-cycle with reversed
post-smoothing, and PCG convergence against a direct sparse solve."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import problem
from oracle.mesh import Mesh
from oracle.multigrid import Multigrid, prolongation
from paper_2407_02100_gb300 import inputs


@pytest.mark.parametrize("dim,k,nc", [(2, 1, 2), (2, 2, 2), (2, 3, 3), (3, 1, 2), (3, 2, 2)])
def test_galerkin_identity(dim, k, nc):
    """V_c is a subspace of V_f and a(.,.) is the same form, so
    A_c = P^T A_f P exactly (up to rounding)."""
    c, f = Mesh(dim, k, nc), Mesh(dim, k, 2 * nc)
    P = prolongation(c, f)
    Ac = c.assemble().toarray()
    Af = f.assemble().toarray()
    np.testing.assert_allclose(P.T @ Af @ P, Ac, atol=1e-12 * np.abs(Ac).max())


@pytest.mark.parametrize("dim,k", [(2, 2), (2, 4), (3, 2), (3, 3)])
def test_prolongation_reproduces_coarse_polynomials(dim, k):
    """p = prod x_a (1 - x_a) is in Q_k for k >= 2 and vanishes on the
    boundary: P applied to its coarse nodal values gives its fine values."""
    c, f = Mesh(dim, k, 3), Mesh(dim, k, 6)
    p = lambda X: np.prod(X * (1 - X), axis=1)
    P = prolongation(c, f)
    np.testing.assert_allclose(P @ p(c.node_coordinates()), p(f.node_coordinates()), atol=1e-14)


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 7, 8])
def test_restriction_rows_stay_in_their_coarse_cell(k):
    """The support the transfer kernels rely on, read off the oracle's P:
    a coarse node c inside coarse cell j (c mod k != 0) restricts only fine
    nodes strictly inside that cell (2k j < x_f < 2k j + 2k); a coarse
    vertex c = k j restricts fine nodes within 2k - 1 of its position 2c.
    Checked along x on a 2D mesh (the y factor only scales the rows)."""
    c, f = Mesh(2, k, 3), Mesh(2, k, 6)
    P = prolongation(c, f)
    fx, cx = f.node_multi()[:, 0], c.node_multi()[:, 0]  # x lattice index of every node
    nz_f, nz_c = np.nonzero(np.abs(P) > 1e-15)
    for xf, xc in zip(fx[nz_f], cx[nz_c]):
        j = xc // k
        if xc % k:
            assert 2 * k * j < xf < 2 * k * j + 2 * k, (xc, xf)
        else:
            assert abs(xf - 2 * xc) <= 2 * k - 1, (xc, xf)


@pytest.mark.parametrize("dim,k,ns", [(2, 1, (4, 8, 16)), (2, 2, (4, 8, 16)), (2, 3, (2, 4, 8)),
                                      (3, 1, (2, 4, 8)), (3, 2, (2, 4))])
def test_manufactured_solution_converges_at_rate_k_plus_1(dim, k, ns):
    u_exact, f = problem.sine_solution(dim)
    errs = []
    for n in ns:
        m = Mesh(dim, k, n)
        A = m.assemble()
        b = problem.load_vector(m, f)
        inner = m.interior_nodes()
        u = np.zeros(m.n_nodes)
        u[inner] = spla.spsolve(A[inner][:, inner].tocsc(), b[inner])
        errs.append(problem.l2_error(m, u, u_exact))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates.min() > k + 1 - 0.35, (errs, rates)


def _mg(dim, k, n, levels):
    return Multigrid(dim, k, n, levels)


def test_vcycle_is_symmetric():
    mg = _mg(2, 2, 8, 3)
    r1 = inputs.random_nodal(2, 2, 8, 21)
    r2 = inputs.random_nodal(2, 2, 8, 22)
    a, b = r1 @ mg.vcycle(r2), r2 @ mg.vcycle(r1)
    assert abs(a - b) < 1e-12 * abs(a)


def test_vcycle_with_exact_coarse_on_one_level_is_direct_solve():
    mg = _mg(2, 3, 4, 1)
    b = inputs.random_nodal(2, 3, 4, 23)
    A = mg.A[0]
    x = mg.vcycle(b)
    np.testing.assert_allclose(A @ x, b, atol=1e-11 * np.abs(b).max())


@pytest.mark.parametrize("dim,k,n,levels", [(2, 2, 32, 3), (2, 3, 16, 3), (3, 2, 8, 3)])
def test_pcg_matches_direct_solve(dim, k, n, levels):
    mg = _mg(dim, k, n, levels)
    b = inputs.random_nodal(dim, k, n, 24)
    x, its, hist = mg.pcg(b, rtol=1e-10)
    assert hist[-1] <= 1e-10
    assert its <= 15
    A = mg.A[mg.finest]
    inner = mg.meshes[-1].interior_nodes()
    xd = np.zeros_like(b)
    xd[inner] = spla.spsolve(A[inner][:, inner].tocsc(), b[inner])
    assert np.linalg.norm(x - xd) <= 1e-8 * np.linalg.norm(xd)


def test_pcg_iterations_do_not_grow_with_refinement():
    its = []
    for n in (8, 16, 32):
        mg = _mg(2, 2, n, 3 if n >= 8 else 2)
        b = inputs.random_nodal(2, 2, n, 25)
        its.append(mg.pcg(b, rtol=1e-10)[1])
    assert max(its) - min(its) <= 2, its

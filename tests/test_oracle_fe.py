"""Pins of the oracle's finite element layer against closed forms.

Nothing here re-types the oracle's formulas: the expected values are
textbook closed forms (Gauss-Lobatto points, Q1 element matrices, the Q1
five/nine-point stencil), polynomial exactness, and the energy identity
u^T A u = int |grad u|^2 for polynomials in the Q_k space."""
import numpy as np
import pytest

from oracle import fe
from oracle.mesh import Mesh


def test_gauss_lobatto_closed_forms():
    np.testing.assert_allclose(fe.gauss_lobatto_points(1), [0, 1], atol=0)
    np.testing.assert_allclose(fe.gauss_lobatto_points(2), [0, 0.5, 1], atol=1e-15)
    a = 1 / np.sqrt(5)                       # GLL(3) on [-1,1]: 0-free, +-1/sqrt5
    np.testing.assert_allclose(fe.gauss_lobatto_points(3), [0, (1 - a) / 2, (1 + a) / 2, 1], atol=1e-15)
    b = np.sqrt(3 / 7)                       # GLL(4): 0, +-sqrt(3/7)
    np.testing.assert_allclose(fe.gauss_lobatto_points(4), [0, (1 - b) / 2, 0.5, (1 + b) / 2, 1], atol=1e-15)
    # GLL(5) interior points on [-1,1]: +-sqrt(1/3 -+ 2 sqrt7 / 21)
    c1, c2 = np.sqrt(1 / 3 - 2 * np.sqrt(7) / 21), np.sqrt(1 / 3 + 2 * np.sqrt(7) / 21)
    ref = np.array([-1, -c2, -c1, c1, c2, 1])
    np.testing.assert_allclose(fe.gauss_lobatto_points(5), (ref + 1) / 2, atol=1e-15)


@pytest.mark.parametrize("k", range(1, 9))
def test_gauss_lobatto_symmetric_and_sorted(k):
    x = fe.gauss_lobatto_points(k)
    assert len(x) == k + 1
    assert np.all(np.diff(x) > 0)
    np.testing.assert_allclose(x + x[::-1], 1.0, atol=2e-15)


@pytest.mark.parametrize("nq", range(1, 10))
def test_gauss_rule_exact_on_monomials(nq):
    x, w = fe.gauss_rule(nq)
    for p in range(2 * nq):
        assert abs(np.sum(w * x ** p) - 1.0 / (p + 1)) < 1e-14


@pytest.mark.parametrize("k", range(1, 9))
def test_lagrange_interpolation_and_derivative(k):
    nodes = fe.gauss_lobatto_points(k)
    V = fe.lagrange_values(nodes, nodes)
    np.testing.assert_allclose(V, np.eye(k + 1), atol=1e-13)
    t = np.linspace(0, 1, 17)
    coeffs = np.random.default_rng(k).standard_normal(k + 1)
    poly = np.polynomial.Polynomial(coeffs)
    # interpolation of a degree-k polynomial is exact, and so is its derivative
    np.testing.assert_allclose(fe.lagrange_values(nodes, t) @ poly(nodes), poly(t), atol=1e-11)
    np.testing.assert_allclose(fe.lagrange_derivatives(nodes, t) @ poly(nodes), poly.deriv()(t), atol=1e-9)


def test_q1_element_matrices_closed_form():
    h = 0.37
    # 2D mass = (h/6 [2 1; 1 2]) kron (h/6 [2 1; 1 2]); 2D stiffness has no h
    np.testing.assert_allclose(fe.cell_mass(2, 1, h)[:2, :2] / h ** 2, [[4 / 36, 2 / 36], [2 / 36, 4 / 36]], atol=1e-15)
    A2 = fe.cell_stiffness(2, 1, h)           # independent of h in 2D
    ref = np.array([[4, -1, -1, -2], [-1, 4, -2, -1], [-1, -2, 4, -1], [-2, -1, -1, 4]]) / 6.0
    np.testing.assert_allclose(A2, ref, atol=1e-15)


def test_q1_assembled_stencil_2d():
    """The Q1 stiffness on a uniform square mesh is the 9-point stencil
    8/3 at the centre and -1/3 at the 8 neighbours."""
    m = Mesh(2, 1, 4)
    A = m.assemble().toarray()
    centre = m.flat(np.array([2, 2]))
    row = A[centre].reshape(m.N, m.N)         # [y, x]
    expect = np.zeros((m.N, m.N))
    expect[1:4, 1:4] = -1 / 3
    expect[2, 2] = 8 / 3
    np.testing.assert_allclose(row, expect, atol=1e-14)


@pytest.mark.parametrize("dim,k", [(2, 1), (2, 2), (2, 5), (3, 1), (3, 3)])
def test_element_stiffness_energy_of_polynomials(dim, k):
    """u^T A_c u = int_cell |grad u|^2 for u in Q_k; A_c 1 = 0."""
    h = 0.25
    A = fe.cell_stiffness(dim, k, h)
    np.testing.assert_allclose(A, A.T, atol=1e-13)
    np.testing.assert_allclose(A.sum(axis=1), 0.0, atol=1e-11 / h)
    nodes = fe.gauss_lobatto_points(k) * h
    grid = np.indices((k + 1,) * dim).reshape(dim, -1)[::-1].T
    X = nodes[grid]                           # [i, alpha] physical coordinates
    # u = x_0^k: int_{[0,h]^d} (k x^{k-1})^2 = k^2 h^{2k-1}/(2k-1) * h^{d-1}
    u = X[:, 0] ** k
    expect = k * k * h ** (2 * k - 1) / (2 * k - 1) * h ** (dim - 1)
    assert abs(u @ A @ u - expect) < 1e-12 * max(1.0, expect)
    # u = x_0 + x_1 (linear): |grad u|^2 = 2 -> 2 h^d
    u = X[:, 0] + X[:, 1]
    assert abs(u @ A @ u - 2 * h ** dim) < 1e-13


def test_paper_problem_sizes_golden():
    """Table 2 lists the DoF counts of its three meshes, each one vertex
    patch refined ten times (2D) or six times (3D); the node counting of the
    oracle (all lattice nodes, boundary included) must reproduce them."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "table2_problem_sizes.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for dim, k, refinements, dofs in rows:
        dim, k, refinements, dofs = int(dim), int(k), int(refinements), int(dofs)
        n_cells = 2 * 2 ** refinements        # a single vertex patch has 2 cells per direction
        m = Mesh.__new__(Mesh)
        Mesh.__init__(m, dim, k, n_cells)
        assert m.n_nodes == dofs

"""Q_k finite element ingredients, FP64, plain definitions (test infrastructure).

Sec. 2 of the paper builds V_l from Lagrange shape functions attached to
support points; App. A.2 fixes the Poisson problem on the unit hypercube on a
uniform Cartesian mesh.  The paper does not name the support points; we use
the Gauss-Lobatto points (the usual choice for FE_Q-type elements; the
discrete solution does not depend on it, only the matrix entries do).

Everything here is written out from the definitions: Lagrange polynomials as
products, gradients by the product rule, the cell stiffness as the full
d-dimensional quadrature sum of grad(phi_i) . grad(phi_j) -- no tensor
factorisation, no sum factorisation.
"""
import numpy as np


def gauss_lobatto_points(k):
    """k+1 Gauss-Lobatto points on [0, 1]: the end points and the roots of
    P_k' (derivative of the Legendre polynomial), polished by Newton steps."""
    if k < 1:
        raise ValueError("degree must be >= 1")
    if k == 1:
        return np.array([0.0, 1.0])
    leg = np.polynomial.legendre.Legendre.basis(k)
    d1 = leg.deriv(1)
    d2 = leg.deriv(2)
    x = np.sort(np.real(d1.roots()))
    for _ in range(8):
        x = x - d1(x) / d2(x)
    pts = np.concatenate([[-1.0], x, [1.0]])
    return 0.5 * (pts + 1.0)


def gauss_rule(nq):
    """nq-point Gauss-Legendre rule on [0, 1] (exact for degree 2 nq - 1)."""
    x, w = np.polynomial.legendre.leggauss(nq)
    return 0.5 * (x + 1.0), 0.5 * w


def lagrange_values(nodes, x):
    """V[q, p] = phi_p(x_q) with phi_p(t) = prod_{r != p} (t - t_r)/(t_p - t_r)."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    V = np.ones((len(x), n))
    for p in range(n):
        for r in range(n):
            if r != p:
                V[:, p] *= (x - nodes[r]) / (nodes[p] - nodes[r])
    return V


def lagrange_derivatives(nodes, x):
    """D[q, p] = phi_p'(x_q) by the product rule:
    phi_p'(t) = sum_{s != p} 1/(t_p - t_s) prod_{r != p, s} (t - t_r)/(t_p - t_r)."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    D = np.zeros((len(x), n))
    for p in range(n):
        for s in range(n):
            if s == p:
                continue
            term = np.full(len(x), 1.0 / (nodes[p] - nodes[s]))
            for r in range(n):
                if r != p and r != s:
                    term *= (x - nodes[r]) / (nodes[p] - nodes[r])
            D[:, p] += term
    return D


def _multi_indices(dim, n):
    """Lexicographic multi-indices (i_0 fastest) of an n^dim tensor grid."""
    idx = np.indices((n,) * dim).reshape(dim, -1)[::-1].T  # column 0 = i_0 (fastest)
    return idx


def cell_stiffness(dim, k, h, coef=1.0):
    """Cell matrix A_c[i, j] = coef * int_cell grad(phi_i) . grad(phi_j) dx on an
    axis-aligned cube of side h, by full dim-dimensional Gauss quadrature with
    k+1 points per direction (exact: the integrand has degree 2k per variable).
    Local numbering is lexicographic with the x index fastest."""
    nodes = gauss_lobatto_points(k)
    xq, wq = gauss_rule(k + 1)
    V = lagrange_values(nodes, xq)        # [q, p]
    D = lagrange_derivatives(nodes, xq) / h  # physical derivative
    basis = _multi_indices(dim, k + 1)    # [i, alpha] -> p
    quad = _multi_indices(dim, k + 1)     # [q, alpha] -> 1D point index
    nb, nqp = len(basis), len(quad)
    weights = np.prod(wq[quad], axis=1) * h ** dim
    grads = np.empty((nqp, nb, dim))
    for a in range(dim):
        g = np.ones((nqp, nb))
        for b in range(dim):
            tab = D if b == a else V
            g *= tab[quad[:, b]][:, basis[:, b]]
        grads[:, :, a] = g
    A = np.einsum("q,qia,qja->ij", weights, grads, grads)
    return coef * A


def cell_mass(dim, k, h):
    """Cell mass matrix int phi_i phi_j by full Gauss quadrature (k+1 points)."""
    nodes = gauss_lobatto_points(k)
    xq, wq = gauss_rule(k + 1)
    V = lagrange_values(nodes, xq)
    basis = _multi_indices(dim, k + 1)
    quad = _multi_indices(dim, k + 1)
    weights = np.prod(wq[quad], axis=1) * h ** dim
    vals = np.ones((len(quad), len(basis)))
    for b in range(dim):
        vals *= V[quad[:, b]][:, basis[:, b]]
    return np.einsum("q,qi,qj->ij", weights, vals, vals)

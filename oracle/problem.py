"""Test problem of App. A.2 (Poisson on the unit hypercube, zero Dirichlet
data) -- load vector and L2 error by plain cell-by-cell quadrature.
Test infrastructure.  The paper prints the equation as "Delta u = f"; we read
it as -Delta u = f so that the stiffness matrix is symmetric positive
definite (the sign only flips f)."""
import itertools

import numpy as np

from . import fe
from .mesh import Mesh


def _cell_quadrature(mesh: Mesh, nq):
    xq, wq = fe.gauss_rule(nq)
    nodes = fe.gauss_lobatto_points(mesh.k)
    V = fe.lagrange_values(nodes, xq)                       # [q, p]
    quad = np.indices((nq,) * mesh.dim).reshape(mesh.dim, -1)[::-1].T
    basis = np.indices((mesh.k + 1,) * mesh.dim).reshape(mesh.dim, -1)[::-1].T
    w = np.prod(wq[quad], axis=1) * mesh.h ** mesh.dim
    vals = np.ones((len(quad), len(basis)))
    for a in range(mesh.dim):
        vals *= V[quad[:, a]][:, basis[:, a]]
    return xq[quad], w, vals


def load_vector(mesh: Mesh, f, nq=None):
    """b_i = int f phi_i over the domain, Dirichlet entries zeroed.
    f: callable on an [npts, dim] coordinate array."""
    nq = mesh.k + 3 if nq is None else nq
    xref, w, vals = _cell_quadrature(mesh, nq)
    b = np.zeros(mesh.n_nodes)
    for cell in itertools.product(range(mesh.n), repeat=mesh.dim):
        x = (np.asarray(cell)[None, :] + xref) * mesh.h
        fx = f(x)
        b[mesh.cell_dofs(cell)] += vals.T @ (w * fx)
    b[mesh.boundary_mask()] = 0.0
    return b


def l2_error(mesh: Mesh, u, exact, nq=None):
    """|| u_h - exact ||_{L2} by cell quadrature."""
    nq = mesh.k + 3 if nq is None else nq
    xref, w, vals = _cell_quadrature(mesh, nq)
    err2 = 0.0
    for cell in itertools.product(range(mesh.n), repeat=mesh.dim):
        x = (np.asarray(cell)[None, :] + xref) * mesh.h
        uh = vals @ u[mesh.cell_dofs(cell)]
        err2 += np.sum(w * (uh - exact(x)) ** 2)
    return np.sqrt(err2)


def sine_solution(dim):
    """u = prod sin(pi x_a) and f = -Delta u = dim pi^2 u."""
    def u(x):
        return np.prod(np.sin(np.pi * x), axis=1)

    def f(x):
        return dim * np.pi ** 2 * np.prod(np.sin(np.pi * x), axis=1)
    return u, f

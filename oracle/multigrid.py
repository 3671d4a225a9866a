"""Geometric multigrid around the patch smoother, FP64 (test infrastructure).

Sec. 2: nested meshes M_0 < ... < M_L (here: uniform refinement, n cells per
direction halved per level), prolongation = embedding of V_l into V_{l+1},
restriction = its transpose.  The embedding is written out from its
definition: the fine coefficient of node x is the coarse function's value at
x, i.e. P[f, c] = phi^coarse_c(x_f), evaluated cell by cell with the coarse
Lagrange basis (no tensor factorisation).

Our readings where the paper is silent: V(1,1)-cycle, pre-smoothing with
ascending colours, post-smoothing with descending colours, exact dense
coarse solve, and the preconditioned conjugate gradient method as the
outer iteration (x_0 = 0, stop at ||r|| <= rtol ||b||).
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from . import fe
from .mesh import Mesh
from .smoother import PatchSmoother


def prolongation(coarse: Mesh, fine: Mesh, sparse=False):
    """Embedding matrix P (fine nodes x coarse nodes), Dirichlet rows and
    columns zeroed; dense, or scipy CSR when sparse=True (same entries)."""
    assert fine.dim == coarse.dim and fine.k == coarse.k and fine.n == 2 * coarse.n
    k, dim = coarse.k, coarse.dim
    xi = fe.gauss_lobatto_points(k)
    X = fine.node_coordinates()                       # [n_fine, dim]
    loc = np.indices((k + 1,) * dim).reshape(dim, -1)[::-1].T
    rows, cols, vals = [], [], []
    for f in range(fine.n_nodes):
        cell = np.minimum(np.floor(X[f] / coarse.h).astype(int), coarse.n - 1)
        t = X[f] / coarse.h - cell                    # reference coordinate in [0,1]
        v = np.ones(len(loc))
        for a in range(dim):
            v *= fe.lagrange_values(xi, t[a])[0][loc[:, a]]
        rows.append(np.full(len(loc), f))
        cols.append(coarse.flat(cell[None, :] * k + loc))
        vals.append(v)
    P = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(fine.n_nodes, coarse.n_nodes)).tocsr()
    # every (fine, coarse) pair appears once: the fine node is assigned to one
    # coarse cell, whose local nodes are distinct
    keep_f = sp.diags((~fine.boundary_mask()).astype(np.float64))
    keep_c = sp.diags((~coarse.boundary_mask()).astype(np.float64))
    P = (keep_f @ P @ keep_c).tocsr()
    return P if sparse else P.toarray()


class Multigrid:
    """Level hierarchy with assembled operators (small meshes only)."""

    def __init__(self, dim, degree, n_cells, n_levels, omega=1.0, sparse=True):
        self.meshes = []
        for l in range(n_levels):
            n = n_cells // 2 ** (n_levels - 1 - l)
            if n * 2 ** (n_levels - 1 - l) != n_cells or n < 1:
                raise ValueError("n_cells not divisible for this many levels")
            self.meshes.append(Mesh(dim, degree, n))
        self.A = [m.assemble() for m in self.meshes]
        self.P = [prolongation(self.meshes[l], self.meshes[l + 1], sparse) for l in range(n_levels - 1)]
        self.smoothers = [PatchSmoother(m, omega) for m in self.meshes]
        inner0 = self.meshes[0].interior_nodes()
        self._inner0 = inner0
        self._coarse = sla.cho_factor(self.A[0][inner0][:, inner0].toarray())

    @property
    def finest(self):
        return len(self.meshes) - 1

    def coarse_solve(self, b):
        x = np.zeros_like(b)
        x[self._inner0] = sla.cho_solve(self._coarse, b[self._inner0])
        return x

    def vcycle(self, b, level=None, pre=1, post=1):
        """x = V(b) with x_0 = 0 on every level."""
        l = self.finest if level is None else level
        if l == 0:
            return self.coarse_solve(b)
        sm = self.smoothers[l]
        u = np.zeros_like(b)
        for _ in range(pre):
            u = sm.sweep(u, b, reverse=False)
        r = b - self.A[l] @ u
        e = self.vcycle(self.P[l - 1].T @ r, l - 1, pre, post)
        u = u + self.P[l - 1] @ e
        for _ in range(post):
            u = sm.sweep(u, b, reverse=True)
        return u

    def pcg(self, b, rtol=1e-10, max_it=200):
        """Preconditioned CG on the finest level.  Returns (x, iterations,
        relative residual history)."""
        A = self.A[self.finest]
        x = np.zeros_like(b)
        r = b.copy()
        bnorm = np.linalg.norm(b)
        hist = [1.0]
        if bnorm == 0.0:
            return x, 0, hist
        z = self.vcycle(r)
        p = z.copy()
        rz = r @ z
        for it in range(1, max_it + 1):
            Ap = A @ p
            alpha = rz / (p @ Ap)
            x += alpha * p
            r -= alpha * Ap
            hist.append(np.linalg.norm(r) / bnorm)
            if hist[-1] <= rtol:
                return x, it, hist
            z = self.vcycle(r)
            rz_new = r @ z
            p = z + (rz_new / rz) * p
            rz = rz_new
        return x, max_it, hist

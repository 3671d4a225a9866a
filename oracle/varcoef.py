"""Variable-coefficient operator -div(a grad u) with one coefficient per cell,
and the patch smoother with approximate local solvers (test infrastructure).

The paper's method (Sec. 2.1: P_j with A_j^{-1}; approximate local solvers are
covered by the framework although P_j then stops being a projection) is applied
with three local solvers:
  exact       A_j^{-1} by dense LU of the patch block assembled from the 2^d
              cell matrices scaled by their coefficients;
  fd_mean     theta_j (1/abar) Ahat_j^{-1}: the constant-coefficient patch
              inverse (fast diagonalisation, App. A.3) scaled by the geometric
              mean abar of the 2^d cell coefficients, with the per-patch
              damping theta_j = min(1, 1.8 abar / max_c a_c).  Since
              A_j <= max_c a_c Ahat_j, theta_j bounds the spectrum of the
              damped local update by 1.8 < 2, so every patch correction
              decreases the energy (our reading of how to use fast
              diagonalisation when it is only approximate);
  learned     (1/abar) (theta_j Ahat_j^{-1} + U diag(s) U^T): the damped FD
              inverse plus a rank-r symmetric correction given per patch (from
              the MLP, trained so that the sum approximates the exact patch
              inverse; a patch whose correction is gated off keeps s = 0,
              i.e. damped FD).
Coarse levels use the geometric mean of the 2^d children as cell coefficient
(our reading; the paper's test problem has constant coefficients).

Pinned (tests/test_oracle_varcoef.py): the exact mode against Algorithm 1
with the assembled variable matrix; fd_mean against the Poisson smoother for
constant coefficients and by its spectral bound; the learned mode by the
full-rank correction Ahat(w)^{-1} - theta Ahat^{-1}, with which it must
reproduce the exact mode (2D and 3D, several h).
"""
import itertools

import numpy as np
import scipy.linalg as sla

from .mesh import Mesh
from .multigrid import prolongation


def coarsen_coefficient(coef):
    """Geometric mean over 2^dim children, coef indexed [c_{d-1},...,c_0]."""
    dim = coef.ndim
    logc = np.log(coef)
    out = 0.0
    for off in itertools.product(range(2), repeat=dim):
        out = out + logc[tuple(slice(o, None, 2) for o in off)]
    return np.exp(out / 2 ** dim)


def patch_cell_coefs(mesh: Mesh, coef, v):
    """Coefficients of the 2^dim cells of the patch at vertex v, flat with the
    cell offset o_0 fastest (the order Mesh.patch_block expects)."""
    out = []
    for off in itertools.product(range(2), repeat=mesh.dim):
        o = off[::-1]                                 # o_0 fastest
        cell = [v[a] - 1 + o[a] for a in range(mesh.dim)]
        out.append(coef[tuple(cell[::-1])])
    return np.array(out)


class VarPatchSmoother:
    """Algorithm 4 with per-patch local solvers on a variable coefficient."""

    def __init__(self, mesh: Mesh, coef, mode="exact", omega=1.0, corrections=None):
        self.mesh, self.coef, self.mode, self.omega = mesh, coef, mode, float(omega)
        self.ref_block, inner = Mesh(mesh.dim, mesh.k, 2).patch_block()   # h = 1/2
        self.ref_block = self.ref_block / 0.5 ** (mesh.dim - 2)          # unit cells
        self.ref_inner = inner
        self.ref_inv = np.linalg.inv(self.ref_block[:, inner])          # Ahat_j^{-1}
        self.corrections = corrections or {}
        self.hscale = mesh.h ** (2 - mesh.dim)                           # h^{2-d}
        self._cache = {}

    def _patch(self, v):
        key = tuple(int(x) for x in v)
        if key not in self._cache:
            cc = patch_cell_coefs(self.mesh, self.coef, v)
            Abar, inner = self.mesh.patch_block(cc)
            abar = np.exp(np.mean(np.log(cc)))
            theta = min(1.0, 1.8 * abar / np.max(cc))
            self._cache[key] = (Abar, sla.lu_factor(Abar[:, inner]), abar, theta)
        return self._cache[key]

    def local_solve(self, v, r):
        Abar, lu, abar, theta = self._patch(v)
        if self.mode == "exact":
            return sla.lu_solve(lu, r)
        d = theta * (self.ref_inv @ (self.hscale * r))
        if self.mode == "learned":
            U, s = self.corrections[tuple(int(x) for x in v)]
            d = d + U @ (s * (U.T @ (self.hscale * r)))
        return d / abar

    def colour_step(self, u, b, c):
        m = self.mesh
        V = m.vertices_of_colour(c)
        updates = []
        for v in V:
            Abar = self._patch(v)[0]
            clo = m.closure_index(v[None, :])[0]
            inn = m.interior_index(v[None, :])[0]
            r = b[inn] - Abar @ u[clo]
            updates.append((inn, self.local_solve(v, r)))
        for inn, d in updates:                         # same colour: independent
            u[inn] += self.omega * d
        return u

    def sweep(self, u, b, reverse=False):
        u = np.array(u, dtype=np.float64, copy=True)
        order = range(self.mesh.n_colours)
        for c in (reversed(list(order)) if reverse else order):
            self.colour_step(u, b, c)
        return u


class VarMultigrid:
    """V(1,1)-cycle and PCG for -div(a grad u), assembled operators."""

    def __init__(self, dim, degree, n_cells, n_levels, coef, mode="exact", corrections=None,
                 omega=1.0):
        self.meshes, self.coefs = [], []
        c = coef
        for l in range(n_levels):
            n = n_cells // 2 ** l
            self.meshes.insert(0, Mesh(dim, degree, n))
            self.coefs.insert(0, c)
            if l < n_levels - 1:
                c = coarsen_coefficient(c)
        self.A = [m.assemble(cf) for m, cf in zip(self.meshes, self.coefs)]
        self.P = [prolongation(self.meshes[l], self.meshes[l + 1], sparse=True)
                  for l in range(n_levels - 1)]
        corr = corrections or [None] * n_levels
        self.smoothers = [VarPatchSmoother(m, cf, mode, omega, corrections=cr)
                          for m, cf, cr in zip(self.meshes, self.coefs, corr)]
        inner0 = self.meshes[0].interior_nodes()
        self._inner0 = inner0
        self._coarse = sla.cho_factor(self.A[0][inner0][:, inner0].toarray())

    def vcycle(self, b, level=None):
        l = len(self.meshes) - 1 if level is None else level
        if l == 0:
            x = np.zeros_like(b)
            x[self._inner0] = sla.cho_solve(self._coarse, b[self._inner0])
            return x
        sm = self.smoothers[l]
        u = sm.sweep(np.zeros_like(b), b)
        r = b - self.A[l] @ u
        u = u + self.P[l - 1] @ self.vcycle(self.P[l - 1].T @ r, l - 1)
        return sm.sweep(u, b, reverse=True)

    def pcg(self, b, rtol=1e-10, max_it=200):
        A = self.A[-1]
        x = np.zeros_like(b)
        r = b.copy()
        bn = np.linalg.norm(b)
        z = self.vcycle(r)
        p = z.copy()
        rz = r @ z
        for it in range(1, max_it + 1):
            Ap = A @ p
            alpha = rz / (p @ Ap)
            x += alpha * p
            r -= alpha * Ap
            if np.linalg.norm(r) <= rtol * bn:
                return x, it
            z = self.vcycle(r)
            rz_new = r @ z
            p = z + (rz_new / rz) * p
            rz = rz_new
        return x, max_it

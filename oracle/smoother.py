"""Multiplicative vertex-patch smoother, FP64 (test infrastructure).

The smoother is the successive subspace correction of Sec. 2.1,
S = prod_j (I - P_j) with P_j = Pi_j^T A_j^{-1} Pi_j A (eq. "main:2",
"s-ell"), evaluated with local residuals (Sec. 3.1):

    gather    bar u_j = bar Pi_j u,  b_j = Pi_j b
    evaluate  r_j = b_j - Pi_j bar A_j bar u_j
    solve     A_j d_j = r_j           (dense LU here; no fast diagonalisation)
    scatter   u += omega Pi_j^T d_j

and ordered by colours (Algorithm 4, the combined colourised smoother): for
each colour in turn, every patch of the colour is updated from the state
left by the previous colours.  Same-colour patches write disjoint interiors
and none reads another's interior, so updating them together is the same as
any sequential order (Sec. 3.2).  Pre-smoothing takes the colours in
ascending order, post-smoothing in descending order (our reading: the paper
does not fix it; the reverse order makes the V-cycle symmetric).

omega: damping of the scatter (the paper's P_j has none, i.e. omega = 1).
"""
import numpy as np
import scipy.linalg as sla

from .mesh import Mesh


class PatchSmoother:
    """Precomputes bar A_j and the LU factors of A_j (identical for every
    patch of a uniform constant-coefficient mesh: one factorisation)."""

    def __init__(self, mesh: Mesh, omega=1.0):
        self.mesh = mesh
        self.omega = float(omega)
        self.Abar, inner = mesh.patch_block()
        self.Aj = self.Abar[:, inner]
        self.lu = sla.lu_factor(self.Aj)
        self._cache = {}

    def _maps(self, c):
        if c not in self._cache:
            V = self.mesh.vertices_of_colour(c)
            self._cache[c] = (self.mesh.closure_index(V), self.mesh.interior_index(V))
        return self._cache[c]

    def local_residual(self, u, b, V):
        """r_j for the patches at vertices V: [P, (2k-1)^dim]."""
        clo = self.mesh.closure_index(V)
        inn = self.mesh.interior_index(V)
        return b[inn] - u[clo] @ self.Abar.T

    def local_solve(self, r):
        """d_j = A_j^{-1} r_j for a stack of residuals [P, m^dim]."""
        return sla.lu_solve(self.lu, r.T).T

    def colour_step(self, u, b, c):
        """All patches of colour c (in place on u)."""
        clo, inn = self._maps(c)
        if len(clo) == 0:
            return u
        r = b[inn] - u[clo] @ self.Abar.T          # gather + evaluate
        d = self.local_solve(r)                     # local solve
        u[inn.ravel()] += self.omega * d.ravel()    # scatter (interiors disjoint)
        return u

    def colour_order(self, reverse=False):
        order = list(range(self.mesh.n_colours))
        return order[::-1] if reverse else order

    def sweep(self, u, b, reverse=False):
        """One smoothing step, Algorithm 4.  Returns a new array."""
        u = np.array(u, dtype=np.float64, copy=True)
        for c in self.colour_order(reverse):
            self.colour_step(u, b, c)
        return u


def sweep_alg1(mesh: Mesh, A, u, b, vertex_sequence, omega=1.0):
    """Algorithm 1 (naive loop): for every patch in the given order, compute
    the GLOBAL residual r = b - A u with the assembled matrix, restrict it to
    the patch interior, solve with the dense A_j and add.  O(n^2); tiny meshes
    only.  A: assembled CSR from Mesh.assemble()."""
    u = np.array(u, dtype=np.float64, copy=True)
    inn_all = mesh.interior_index(vertex_sequence)
    A = A.tocsr()
    for inn in inn_all:
        r = b - A @ u
        Aj = A[inn][:, inn].toarray()
        u[inn] += omega * np.linalg.solve(Aj, r[inn])
    return u


def sweep_alg2(smoother: PatchSmoother, u, b, vertex_sequence):
    """Algorithm 2 (combined, single sequential loop) in the given patch
    order: local residual from the closure, local solve, scatter, one patch
    at a time."""
    u = np.array(u, dtype=np.float64, copy=True)
    for v in np.asarray(vertex_sequence):
        r = smoother.local_residual(u, b, v[None, :])
        d = smoother.local_solve(r)
        inn = smoother.mesh.interior_index(v[None, :])[0]
        u[inn] += smoother.omega * d[0]
    return u


def colour_sorted_vertices(mesh: Mesh, reverse=False):
    """The patch sequence of Algorithm 4 written out: colours ascending (or
    descending), lexicographic inside a colour."""
    order = range(mesh.n_colours)
    if reverse:
        order = reversed(list(order))
    return np.concatenate([mesh.vertices_of_colour(c) for c in order], axis=0)


def skewed_slab_sequence(mesh: Mesh, width, reverse=False):
    """The patch sequence of the skewed-slab schedule (the GPU form of the
    locality batches of Sec. 4.1; our construction): the patch at vertex v
    whose colour sits at position o of the colour order (o = c, or
    n_colours - 1 - c in reverse) belongs to slab (v_slow + o) // width,
    v_slow its index along the slowest axis; slabs in order, colour
    positions in order inside a slab, lexicographic within a group."""
    nc = mesh.n_colours
    groups = {}
    for c in range(nc):
        o = nc - 1 - c if reverse else c
        for v in mesh.vertices_of_colour(c):
            groups.setdefault(((int(v[-1]) + o) // width, o), []).append(v)
    return np.array([v for key in sorted(groups) for v in groups[key]])


def morton_key(v):
    """Z-curve (Morton) key of vertex multi-indices v [..., dim]: the bits of
    v_0, v_1 (, v_2) interleaved, v_0 in the lowest position (Sec. 4.1 step 1
    orders patches along a Z-curve; our reading: the Morton order of the
    vertex index)."""
    v = np.asarray(v, dtype=np.int64)
    dim = v.shape[-1]
    key = np.zeros(v.shape[:-1], dtype=np.int64)
    for bit in range(20):
        for a in range(dim):
            key |= ((v[..., a] >> bit) & 1) << (dim * bit + a)
    return key


def batches_alg5(mesh: Mesh, n_b):
    """Sec. 4.1 set-up: (1) all patches in Z-curve order, (2) grouped by
    colour keeping that order, (3) each colour split into batches of n_b.
    Returns P[b][k] = vertex arrays (possibly empty)."""
    V = mesh.vertices()
    V = V[np.argsort(morton_key(V), kind="stable")]
    col = mesh.colour(V)
    per_colour = [V[col == k] for k in range(mesh.n_colours)]
    nb = max((len(P) + n_b - 1) // n_b for P in per_colour) if len(V) else 0
    return [[P[b * n_b:(b + 1) * n_b] for P in per_colour] for b in range(nb)]


def sweep_alg5(smoother: PatchSmoother, u, b, n_b):
    """Algorithm 5: for each batch b, for each colour k, all patches of
    P_{b,k} (independent: one colour) updated from the current state."""
    u = np.array(u, dtype=np.float64, copy=True)
    m = smoother.mesh
    for batch in batches_alg5(m, n_b):
        for P in batch:
            if len(P) == 0:
                continue
            r = smoother.local_residual(u, b, P)
            d = smoother.local_solve(r)
            u[m.interior_index(P).ravel()] += smoother.omega * d.ravel()
    return u


def sweep_alg3(mesh: Mesh, A, smoother: PatchSmoother, u, b, reverse=False):
    """Algorithm 3 (separated, colourised): per colour, one global residual
    r = b - A u with the assembled matrix, then every local solve of the
    colour from r."""
    u = np.array(u, dtype=np.float64, copy=True)
    for c in smoother.colour_order(reverse):
        r = b - A @ u
        V = mesh.vertices_of_colour(c)
        if len(V) == 0:
            continue
        inn = mesh.interior_index(V)
        d = smoother.local_solve(r[inn])
        u[inn.ravel()] += smoother.omega * d.ravel()
    return u

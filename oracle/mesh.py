"""Uniform Cartesian mesh, node numbering, vertex patches and colours (FP64).

Test infrastructure.  Mesh: the unit hypercube [0,1]^dim split into n cells
per direction (h = 1/n), the Q_k space on it (App. A.2).  Nodes are numbered
on the (n k + 1)^dim lattice, lexicographically with x fastest; ALL nodes are
stored and the homogeneous Dirichlet nodes (any index 0 or n k) carry zeros.

Vertex patches (Sec. 2.1 item 1): one per interior vertex v in {1..n-1}^dim,
made of the 2^dim cells around it.  Its closure (Sec. 3.1, the space bar V_j
used by the gather) is the node box [(v-1)k, (v+1)k]^dim, its interior (the
space V_j of the local solve) is the open box ((v-1)k, (v+1)k)^dim.

Colours (Sec. 3.2): patches of one colour must not overlap.  We use
c(v) = sum_a 2^a (v_a mod 2); two patches of the same colour differ by at
least 2 in some vertex index, so their cell sets are disjoint.
"""
import itertools

import numpy as np
import scipy.sparse as sp

from . import fe


class Mesh:
    def __init__(self, dim, degree, n_cells):
        if dim not in (2, 3):
            raise ValueError("dim must be 2 or 3")
        self.dim, self.k, self.n = dim, degree, n_cells
        self.h = 1.0 / n_cells
        self.N = n_cells * degree + 1               # nodes per direction
        self.n_nodes = self.N ** dim

    # ---- numbering -------------------------------------------------------
    def flat(self, multi):
        """Flat index of node multi-indices (last axis = direction, x first)."""
        multi = np.asarray(multi)
        out = np.zeros(multi.shape[:-1], dtype=np.int64)
        for a in range(self.dim):
            out += multi[..., a].astype(np.int64) * self.N ** a
        return out

    def node_multi(self):
        """[n_nodes, dim] multi-index of every node in flat order."""
        return np.indices((self.N,) * self.dim).reshape(self.dim, -1)[::-1].T

    def boundary_mask(self):
        m = self.node_multi()
        return np.any((m == 0) | (m == self.N - 1), axis=1)

    def interior_nodes(self):
        return np.nonzero(~self.boundary_mask())[0]

    def node_coordinates(self):
        """Physical coordinates: node i_a = c k + p sits at (c + xi_p) h."""
        xi = fe.gauss_lobatto_points(self.k)
        line = np.empty(self.N)
        for c in range(self.n):
            for p in range(self.k + 1):
                line[c * self.k + p] = (c + xi[p]) * self.h
        return line[self.node_multi()]

    def cell_dofs(self, cell):
        """Global flat indices of the (k+1)^dim nodes of a cell, local lexicographic."""
        loc = np.indices((self.k + 1,) * self.dim).reshape(self.dim, -1)[::-1].T
        return self.flat(np.asarray(cell)[None, :] * self.k + loc)

    # ---- assembled operator (small meshes only) --------------------------
    def assemble(self, coef=None):
        """Global stiffness restricted to the interior (Dirichlet) nodes, as a
        CSR matrix on ALL nodes whose boundary rows and columns are zero.
        coef: optional per-cell coefficient array of shape (n,)*dim indexed
        [c_{dim-1}, ..., c_0] (so its C-order flattening has c_0 fastest), for
        the variable-coefficient operator -div(a grad u)."""
        Ae = fe.cell_stiffness(self.dim, self.k, self.h)
        rows, cols, vals = [], [], []
        for cell in itertools.product(range(self.n), repeat=self.dim):
            dofs = self.cell_dofs(cell)
            a = 1.0 if coef is None else float(coef[tuple(cell[::-1])])
            rows.append(np.repeat(dofs, len(dofs)))
            cols.append(np.tile(dofs, len(dofs)))
            vals.append((a * Ae).ravel())
        A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(self.n_nodes, self.n_nodes)).tocsr()
        keep = sp.diags((~self.boundary_mask()).astype(np.float64))
        return (keep @ A @ keep).tocsr()

    # ---- vertex patches ---------------------------------------------------
    def vertices(self):
        """All interior vertices, [J, dim], lexicographic (x fastest)."""
        return np.indices((self.n - 1,) * self.dim).reshape(self.dim, -1)[::-1].T + 1 \
            if self.n > 1 else np.zeros((0, self.dim), dtype=np.int64)

    def colour(self, v):
        v = np.asarray(v)
        return sum((2 ** a) * (v[..., a] % 2) for a in range(self.dim))

    @property
    def n_colours(self):
        return 2 ** self.dim

    def vertices_of_colour(self, c):
        V = self.vertices()
        return V[self.colour(V) == c]

    def closure_local(self):
        """Local closure lattice offsets [(2k+1)^dim, dim] (x fastest)."""
        return np.indices((2 * self.k + 1,) * self.dim).reshape(self.dim, -1)[::-1].T

    def interior_local(self):
        """Local interior lattice offsets [(2k-1)^dim, dim] (x fastest)."""
        return np.indices((2 * self.k - 1,) * self.dim).reshape(self.dim, -1)[::-1].T + 1

    def closure_index(self, V):
        """bar Pi_j as an index map: [P, (2k+1)^dim] global flat indices."""
        V = np.asarray(V).reshape(-1, self.dim)
        base = (V - 1) * self.k
        return self.flat(base[:, None, :] + self.closure_local()[None, :, :])

    def interior_index(self, V):
        """Pi_j as an index map: [P, (2k-1)^dim] global flat indices."""
        V = np.asarray(V).reshape(-1, self.dim)
        base = (V - 1) * self.k
        return self.flat(base[:, None, :] + self.interior_local()[None, :, :])

    def patch_block(self, cell_coefs=None):
        """bar A_j: rows = patch interior nodes, columns = patch closure nodes,
        assembled from the 2^dim cell matrices of the patch (Sec. 3.1 eq.
        "evaluate": the restriction of A to bar V_j).  Rows of the patch
        interior receive contributions from patch cells only, so these rows
        equal the corresponding rows of the global matrix.
        cell_coefs: optional 2^dim per-cell coefficients indexed by the cell
        offset o in {0,1}^dim, flat with o_0 fastest."""
        k, dim = self.k, self.dim
        C = 2 * k + 1
        Ae = fe.cell_stiffness(dim, k, self.h)
        loc = np.indices((k + 1,) * dim).reshape(dim, -1)[::-1].T
        full = np.zeros((C ** dim, C ** dim))
        for ci, off in enumerate(itertools.product(range(2), repeat=dim)):
            off = np.array(off[::-1])           # o_0 fastest in the flat cell index
            a = 1.0 if cell_coefs is None else float(cell_coefs[ci])
            lattice = off[None, :] * k + loc
            idx = sum(lattice[:, a2] * C ** a2 for a2 in range(dim))
            full[np.ix_(idx, idx)] += a * Ae
        cl = self.closure_local()
        inner = np.nonzero(np.all((cl > 0) & (cl < 2 * k), axis=1))[0]
        return full[inner, :], inner

"""Seeded synthetic inputs shared by the CUDA path, its tests and the oracle.

This module holds no arithmetic of the method: it only draws random nodal
vectors on the (n k + 1)^dim node lattice of a uniform Q_k mesh (flat,
x index fastest) and zeroes the homogeneous Dirichlet nodes.  The paper's
test problem (App. A.2) is Poisson on the unit hypercube with zero Dirichlet
data; its right-hand sides here are N(0,1) or U[-1,1] draws from
``numpy.random.default_rng(seed)``.
"""
import numpy as np


def nodes_per_direction(degree, n_cells):
    return n_cells * degree + 1


def boundary_mask(dim, degree, n_cells):
    """Boolean mask of the Dirichlet nodes (any lattice index 0 or n k)."""
    N = nodes_per_direction(degree, n_cells)
    line = np.zeros(N, dtype=bool)
    line[0] = line[-1] = True
    if dim == 2:
        return (line[None, :] | line[:, None]).ravel()
    return (line[None, None, :] | line[None, :, None] | line[:, None, None]).ravel()


def random_nodal(dim, degree, n_cells, seed, dist="normal"):
    """Random vector on all nodes, Dirichlet entries zero, float64."""
    N = nodes_per_direction(degree, n_cells)
    rng = np.random.default_rng(seed)
    n = N ** dim
    if dist == "normal":
        x = rng.standard_normal(n)
    elif dist == "uniform":
        x = rng.uniform(-1.0, 1.0, n)
    else:
        raise ValueError("dist must be 'normal' or 'uniform'")
    x[boundary_mask(dim, degree, n_cells)] = 0.0
    return x


def sample_vertices(dim, n_cells, count, seed):
    """Random interior vertices v in {1..n-1}^dim, unique, sorted
    lexicographically (x index fastest)."""
    rng = np.random.default_rng(seed)
    out = set()
    tries = 0
    while len(out) < count and tries < 100 * count + 1000:
        tries += 1
        out.add(tuple(int(x) for x in rng.integers(1, n_cells, size=dim)))
    return np.array(sorted(out, key=lambda t: t[::-1]), dtype=np.int64).reshape(-1, dim)

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


def gaussian_random_field(dim, n_cells, seed, sigma=1.0, corr_len=0.1):
    """Per-cell values of a stationary Gaussian random field with squared-
    exponential covariance sigma^2 exp(-r^2 / (2 corr_len^2)), sampled at the
    cell centres of a uniform n^dim mesh of the unit cube by circulant
    embedding on a periodic grid of 2n points per direction (spacing 1/n),
    from numpy.random.default_rng(seed).  Returns shape (n,)*dim indexed
    [c_{dim-1}, ..., c_0] (C-order flattening = c_0 fastest)."""
    m = 2 * n_cells
    h = 1.0 / n_cells
    d1 = np.minimum(np.arange(m), m - np.arange(m)) * h          # periodic distances
    r2 = np.zeros((m,) * dim)
    for a in range(dim):
        shape = [1] * dim
        shape[a] = m
        r2 = r2 + (d1 ** 2).reshape(shape)
    cov = sigma ** 2 * np.exp(-r2 / (2.0 * corr_len ** 2))
    lam = np.real(np.fft.fftn(cov))
    lam = np.maximum(lam, 0.0)                                    # clip round-off negatives
    rng = np.random.default_rng(seed)
    xi = rng.standard_normal((m,) * dim)
    g = np.real(np.fft.ifftn(np.sqrt(lam) * np.fft.fftn(xi)))
    return g[(slice(0, n_cells),) * dim].copy()


def lognormal_coefficient(dim, n_cells, seed, sigma=1.0, corr_len=0.1):
    """a = exp(g) per cell, g from gaussian_random_field (float64)."""
    return np.exp(gaussian_random_field(dim, n_cells, seed, sigma, corr_len))

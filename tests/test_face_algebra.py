"""Identities the GPU kernels rely on, checked in FP64 on the CPU with the
oracle's unit-cell matrices (no GPU).

1. Zero-interior residual (App. A.3 with eq. "main:4"): with an exact local
   solver the new patch interior is A_j^{-1}(b_j - bar A_j bar u_j^0), bar u_j^0
   the closure with a zero interior.  bar A_j bar u_j^0 splits into six face
   terms: a column of a two-cell 1D matrix (closure column 0 or 2k) times a
   two-dimensional sum-factorised term of one closure face.  The shared-face
   sweep evaluates the face terms once per face plane.
2. On the vertex row of the two-cell matrices both end columns hold the same
   cell-matrix entry (the reference cell matrices are symmetric about the cell
   centre), so the two y (z) faces of a patch can share one coefficient there.
3. The three-pass operator evaluates global 1D row c k + p (0 <= p < k) from
   the 2k + 1 nodes around it: row k of cell c - 1 plus row 0 of cell c at a
   vertex, row p of cell c inside."""
import numpy as np
import pytest

from oracle import fe


def two_cell(k):
    """Two-cell 1D mass and stiffness on unit cells: interior rows 1..2k-1,
    closure columns 0..2k."""
    C = 2 * k + 1
    Mc, Kc = fe.cell_mass(1, k, 1.0), fe.cell_stiffness(1, k, 1.0)
    Mf, Kf = np.zeros((C, C)), np.zeros((C, C))
    for c in range(2):
        Mf[c * k:c * k + k + 1, c * k:c * k + k + 1] += Mc
        Kf[c * k:c * k + k + 1, c * k:c * k + k + 1] += Kc
    return Mf[1:C - 1], Kf[1:C - 1]


def patch_op(Ex, Ey, Ez, v):
    """(Ex (x) Ey (x) Ez) applied to v[x, y, z]."""
    return np.einsum("ia,jb,lc,abc->ijl", Ex, Ey, Ez, v)


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 7])
def test_zero_interior_residual_is_a_sum_of_face_terms(k):
    C = 2 * k + 1
    Mp, Kp = two_cell(k)
    MI, KI = Mp[:, 1:C - 1], Kp[:, 1:C - 1]
    u = np.random.default_rng(k).standard_normal((C, C, C))
    u0 = u.copy()
    u0[1:-1, 1:-1, 1:-1] = 0.0
    direct = patch_op(Kp, Mp, Mp, u0) + patch_op(Mp, Kp, Mp, u0) + patch_op(Mp, Mp, Kp, u0)
    faces = np.zeros_like(direct)
    for f in (0, C - 1):
        v = u[f]                                  # x face: all y, z
        F1 = Mp @ v @ Mp.T
        F2 = Kp @ v @ Mp.T + Mp @ v @ Kp.T
        faces += np.einsum("i,jl->ijl", Kp[:, f], F1) + np.einsum("i,jl->ijl", Mp[:, f], F2)
        w = u[1:-1, f, :]                         # y face: x interior, all z
        G1 = KI @ w @ Mp.T + MI @ w @ Kp.T
        G2 = MI @ w @ Mp.T
        faces += np.einsum("j,il->ijl", Mp[:, f], G1) + np.einsum("j,il->ijl", Kp[:, f], G2)
        s = u[1:-1, 1:-1, f]                      # z face: x, y interior
        H1 = KI @ s @ MI.T + MI @ s @ KI.T
        H2 = MI @ s @ MI.T
        faces += np.einsum("l,ij->ijl", Mp[:, f], H1) + np.einsum("l,ij->ijl", Kp[:, f], H2)
    assert np.abs(faces - direct).max() <= 1e-13 * np.abs(direct).max()
    # column 0 is nonzero only on rows 0..k-1 (the first cell) and column 2k
    # only on rows k-1..2k-2: the band the kernels' face coefficients use
    assert np.all(Mp[k:, 0] == 0) and np.all(Mp[:k - 1, C - 1] == 0)


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6, 7, 8])
def test_vertex_row_has_equal_end_columns(k):
    Mp, Kp = two_cell(k)
    C = 2 * k + 1
    for E in (Mp, Kp):
        assert abs(E[k - 1, 0] - E[k - 1, C - 1]) <= 1e-14 * abs(E[k - 1, 0])


@pytest.mark.parametrize("k,n", [(1, 5), (3, 4), (4, 3), (7, 2)])
def test_segment_rows_equal_the_global_1d_matrix(k, n):
    N = n * k + 1
    Mc = fe.cell_stiffness(1, k, 1.0)
    G = np.zeros((N, N))
    for c in range(n):
        G[c * k:c * k + k + 1, c * k:c * k + k + 1] += Mc
    v = np.random.default_rng(7).standard_normal(N)
    out = np.zeros(N)
    for c in range(n):
        win = np.array([v[c * k - k + w] if 0 <= c * k - k + w < N else 0.0 for w in range(2 * k + 1)])
        for p in range(k):
            node = c * k + p
            if node < 1 or node > N - 2:
                continue
            acc = Mc[k] @ win[:k + 1] if p == 0 else 0.0
            out[node] = acc + Mc[p] @ win[k:]
    ref = G @ v
    assert np.abs(out[1:-1] - ref[1:-1]).max() <= 1e-14 * np.abs(ref).max()

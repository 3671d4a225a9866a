"""Pins of the oracle's patch smoother (Algorithm 4) against independent
definitions: the naive global-residual loop (Algorithm 1) with the assembled
matrix, a hand-written multicolour Gauss-Seidel for Q1, the exactness of the
local solve, and the energy decrease of an exact subspace correction."""
import numpy as np
import pytest

from oracle.mesh import Mesh
from oracle.smoother import (PatchSmoother, batches_alg5, colour_sorted_vertices,
                             morton_key, skewed_slab_sequence, sweep_alg1, sweep_alg2, sweep_alg3,
                             sweep_alg5)
from paper_2407_02100_gb300 import inputs


def _rand(m, seed):
    return inputs.random_nodal(m.dim, m.k, m.n, seed)


@pytest.mark.parametrize("dim,k,n", [(2, 1, 5), (2, 3, 6), (3, 2, 4), (3, 1, 5)])
def test_colour_classes_do_not_overlap(dim, k, n):
    m = Mesh(dim, k, n)
    assert m.n_colours == 2 ** dim
    allv = m.vertices()
    assert len(allv) == (n - 1) ** dim
    seen = 0
    covered = np.zeros(m.n_nodes, dtype=int)
    for c in range(m.n_colours):
        V = m.vertices_of_colour(c)
        seen += len(V)
        inn = m.interior_index(V)
        clo = m.closure_index(V)
        # interiors disjoint, and no patch reads another same-colour interior
        assert len(np.unique(inn)) == inn.size
        for j in range(len(V)):
            others = np.delete(inn, j, axis=0).ravel()
            assert not np.intersect1d(clo[j], others).size
        covered[np.unique(inn)] += 1
    assert seen == len(allv)
    # every interior node lies in the interior of at least one patch
    assert np.all(covered[m.interior_nodes()] >= 1)
    assert np.all(covered[m.boundary_mask()] == 0)


@pytest.mark.parametrize("dim,k,n", [(2, 1, 4), (2, 3, 4), (3, 2, 3)])
def test_patch_block_rows_equal_global_rows(dim, k, n):
    m = Mesh(dim, k, n)
    A = m.assemble().toarray()
    Abar, _ = m.patch_block()
    bdry = m.boundary_mask()
    for v in m.vertices():
        inn = m.interior_index(v[None, :])[0]
        clo = m.closure_index(v[None, :])[0]
        # Dirichlet columns are zero in the assembled matrix; they multiply
        # stored zeros in the patch block, so only the other columns matter
        keep = ~bdry[clo]
        np.testing.assert_allclose(A[np.ix_(inn, clo[keep])], Abar[:, keep],
                                   atol=1e-12 * np.abs(Abar).max())
        # interior rows have no entries outside the closure
        rest = np.setdiff1d(np.arange(m.n_nodes), clo)
        assert np.abs(A[np.ix_(inn, rest)]).max() == 0.0


@pytest.mark.parametrize("dim,k,n", [(2, 1, 4), (2, 2, 4), (2, 3, 4), (3, 1, 4), (3, 2, 4)])
@pytest.mark.parametrize("reverse", [False, True])
def test_algorithm4_equals_naive_algorithm1(dim, k, n, reverse):
    m = Mesh(dim, k, n)
    A = m.assemble()
    u0, b = _rand(m, 1), _rand(m, 2)
    s = PatchSmoother(m)
    u4 = s.sweep(u0, b, reverse=reverse)
    u1 = sweep_alg1(m, A, u0, b, colour_sorted_vertices(m, reverse))
    np.testing.assert_allclose(u4, u1, rtol=0, atol=1e-12 * np.abs(u1).max())


@pytest.mark.parametrize("omega", [0.5, 0.8])
def test_damping_matches_naive_loop(omega):
    m = Mesh(2, 2, 5)
    A = m.assemble()
    u0, b = _rand(m, 3), _rand(m, 4)
    u4 = PatchSmoother(m, omega).sweep(u0, b)
    u1 = sweep_alg1(m, A, u0, b, colour_sorted_vertices(m), omega)
    np.testing.assert_allclose(u4, u1, rtol=0, atol=1e-12 * np.abs(u1).max())


def test_same_colour_patches_commute():
    """Sec. 3.2: within a colour the patch order does not change the result."""
    m = Mesh(3, 2, 5)
    s = PatchSmoother(m)
    u0, b = _rand(m, 5), _rand(m, 6)
    u4 = s.sweep(u0, b)
    rng = np.random.default_rng(0)
    seq = np.concatenate([rng.permutation(m.vertices_of_colour(c)) for c in range(m.n_colours)])
    u2 = sweep_alg2(s, u0, b, seq)
    np.testing.assert_allclose(u4, u2, rtol=0, atol=1e-12 * np.abs(u2).max())


def test_q1_sweep_is_multicolour_gauss_seidel():
    """For k = 1 each patch interior is one vertex: the sweep is point
    Gauss-Seidel on the 9-point stencil (8/3 centre, -1/3 neighbours) with
    the four-colour vertex ordering."""
    n = 7
    m = Mesh(2, 1, n)
    u0, b = _rand(m, 7), _rand(m, 8)
    s = PatchSmoother(m)
    got = s.sweep(u0, b)
    U = u0.reshape(n + 1, n + 1).copy()          # [y, x]
    B = b.reshape(n + 1, n + 1)
    for colour in range(4):
        for y in range(1, n):
            for x in range(1, n):
                if (x % 2) + 2 * (y % 2) != colour:
                    continue
                nb = U[y - 1:y + 2, x - 1:x + 2].sum() - U[y, x]
                U[y, x] = (B[y, x] + nb / 3.0) / (8.0 / 3.0)
    np.testing.assert_allclose(got, U.ravel(), rtol=0, atol=1e-13)


@pytest.mark.parametrize("dim,k,n", [(2, 2, 6), (2, 4, 4), (3, 2, 4)])
def test_local_residual_vanishes_after_each_colour(dim, k, n):
    m = Mesh(dim, k, n)
    A = m.assemble()
    s = PatchSmoother(m)
    u, b = _rand(m, 9), _rand(m, 10)
    for c in range(m.n_colours):
        s.colour_step(u, b, c)
        r = b - A @ u
        inn = m.interior_index(m.vertices_of_colour(c))
        assert np.abs(r[inn]).max() < 1e-11 * np.abs(b).max()


@pytest.mark.parametrize("dim,k,n", [(2, 3, 5), (3, 2, 4)])
def test_energy_decreases_per_patch(dim, k, n):
    """J(u) = u^T A u / 2 - b^T u is non-increasing after every exact patch
    solve (each is an A-orthogonal projection of the error, Sec. 2.1)."""
    m = Mesh(dim, k, n)
    A = m.assemble()
    s = PatchSmoother(m)
    u, b = _rand(m, 11), _rand(m, 12)
    J = lambda x: 0.5 * x @ (A @ x) - b @ x
    prev = J(u)
    for v in colour_sorted_vertices(m):
        u = sweep_alg2(s, u, b, v[None, :])
        cur = J(u)
        assert cur <= prev + 1e-12 * abs(prev)
        prev = cur


def test_exact_local_solve_forgets_old_interior():
    """With omega = 1 the new patch interior is A_j^{-1}(b_j - A_jB u_B): it
    does not depend on the old interior values."""
    m = Mesh(2, 3, 5)
    s = PatchSmoother(m)
    u, b = _rand(m, 13), _rand(m, 14)
    v = m.vertices()[7][None, :]
    inn = m.interior_index(v)[0]
    u2 = u.copy()
    u2[inn] = np.random.default_rng(1).standard_normal(len(inn))
    a = sweep_alg2(s, u, b, v)
    c = sweep_alg2(s, u2, b, v)
    np.testing.assert_allclose(a, c, rtol=0, atol=1e-12 * np.abs(a).max())


def test_morton_key_small_cases():
    """Bit interleaving: (1,0)->1, (0,1)->2, (1,1)->3, (2,0)->4, (3,5)->0b100111."""
    got = morton_key(np.array([[1, 0], [0, 1], [1, 1], [2, 0], [3, 5]]))
    np.testing.assert_array_equal(got, [1, 2, 3, 4, 0b100111])
    assert morton_key(np.array([[1, 1, 1]]))[0] == 7


@pytest.mark.parametrize("dim,k,n", [(2, 2, 6), (3, 2, 5)])
def test_algorithm3_equals_algorithm4(dim, k, n):
    """Sec. 3.3: the separated and the combined colourised smoothers are the
    same mathematical algorithm."""
    m = Mesh(dim, k, n)
    A = m.assemble()
    s = PatchSmoother(m)
    u0, b = _rand(m, 15), _rand(m, 16)
    for rev in (False, True):
        np.testing.assert_allclose(sweep_alg3(m, A, s, u0, b, rev), s.sweep(u0, b, rev),
                                   rtol=0, atol=1e-12 * np.abs(b).max())


@pytest.mark.parametrize("dim,k,n", [(2, 2, 7), (3, 1, 6)])
def test_algorithm5_limits(dim, k, n):
    """n_B >= colour size gives Algorithm 4; n_B = 1 gives the sequential loop
    (Algorithm 2, and Algorithm 1 with global residuals) over the interleaved
    sequence batch 0 colours 0..2^d-1, batch 1 colours 0..2^d-1, ..."""
    m = Mesh(dim, k, n)
    A = m.assemble()
    s = PatchSmoother(m)
    u0, b = _rand(m, 17), _rand(m, 18)
    big = len(m.vertices())
    np.testing.assert_allclose(sweep_alg5(s, u0, b, big), s.sweep(u0, b), rtol=0, atol=1e-13)
    seq = np.concatenate([P for batch in batches_alg5(m, 1) for P in batch if len(P)])
    assert len(seq) == big and len({tuple(v) for v in seq}) == big
    ref1 = sweep_alg1(m, A, u0, b, seq)
    np.testing.assert_allclose(sweep_alg5(s, u0, b, 1), ref1, rtol=0, atol=1e-12 * np.abs(ref1).max())
    np.testing.assert_allclose(sweep_alg2(s, u0, b, seq), ref1, rtol=0, atol=1e-12 * np.abs(ref1).max())
    # a middle batch size differs from Algorithm 4 (the order matters)
    assert np.abs(sweep_alg5(s, u0, b, 3) - s.sweep(u0, b)).max() > 1e-8


@pytest.mark.parametrize("dim,k,n", [(2, 2, 8), (3, 1, 6), (3, 2, 5)])
@pytest.mark.parametrize("reverse", [False, True])
def test_skewed_slab_order_reproduces_algorithm4_exactly(dim, k, n, reverse):
    """Any slab width gives a patch sequence in which every patch reads the
    values Algorithm 4 gives it: Algorithm 2 in that order equals Algorithm 2
    in colour order bit for bit (the same per-patch arithmetic on the same
    inputs), and the batched Algorithm 4 to rounding.  A non-skewed slab
    order (slab from v alone) does not, which shows the test can fail."""
    m = Mesh(dim, k, n)
    s = PatchSmoother(m)
    u0, b = _rand(m, 61), _rand(m, 62)
    ref = s.sweep(u0, b, reverse=reverse)
    ref2 = sweep_alg2(s, u0, b, colour_sorted_vertices(m, reverse))
    assert np.abs(ref2 - ref).max() <= 1e-12 * np.abs(ref).max()
    for width in (1, 2, 3, n + 8):
        seq = skewed_slab_sequence(m, width, reverse)
        assert sorted(map(tuple, seq)) == sorted(map(tuple, m.vertices()))
        assert np.array_equal(sweep_alg2(s, u0, b, seq), ref2), width
    nc = m.n_colours
    plain = sorted(m.vertices(), key=lambda v: (int(v[-1]), (nc - 1 - int(m.colour(v[None, :])[0]))
                                                if reverse else int(m.colour(v[None, :])[0])))
    assert np.abs(sweep_alg2(s, u0, b, np.array(plain)) - ref).max() > 1e-8

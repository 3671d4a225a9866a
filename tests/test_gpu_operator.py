"""Three-pass FP64 3D operator (degrees >= 3) through the C ABI.

The level operator A = K (x) M (x) M + M (x) K (x) M + M (x) M (x) K (unit
cells, x fastest) evaluated as one 1D contraction per axis with the global
1D matrices, through workspace vectors.  Checked against the same operator
written out as Kronecker products of the oracle's 1D cell matrices (inputs
nonzero on the boundary too, which the operator reads like any node), and
against the tile kernel."""
import numpy as np
import pytest

from oracle import fe
from paper_2407_02100_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gmg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2407_02100_gb300 import build, gmg as g
    build.build()
    return g


def kron_apply(k, n, x):
    """(K (x) M (x) M + M (x) K (x) M + M (x) M (x) K) x with the global 1D
    matrices assembled from the oracle's unit-cell matrices; x dense with
    index z N^2 + y N + x."""
    N = n * k + 1

    def glob(E):
        G = np.zeros((N, N))
        for c in range(n):
            G[c * k:c * k + k + 1, c * k:c * k + k + 1] += E
        return G

    Mg, Kg = glob(fe.cell_mass(1, k, 1.0)), glob(fe.cell_stiffness(1, k, 1.0))
    t = x.reshape(N, N, N)

    def ap(Ez, Ey, Ex):
        return np.einsum("ia,jb,kc,abc->ijk", Ez, Ey, Ex, t, optimize=True)

    return (ap(Mg, Mg, Kg) + ap(Mg, Kg, Mg) + ap(Kg, Mg, Mg)).ravel()


def interior(dim, N):
    m = np.zeros((N,) * dim, dtype=bool)
    m[(slice(1, -1),) * dim] = True
    return m.ravel()


def test_form_is_used_where_it_applies(gmg):
    assert gmg.gmg_three_pass_operator(gmg.Problem(3, 4, 4, n_levels=1).h) == 1
    assert gmg.gmg_three_pass_operator(gmg.Problem(3, 3, 4, n_levels=1, precision=1).h) == 1  # FP64 CG
    assert gmg.gmg_three_pass_operator(gmg.Problem(3, 2, 4, n_levels=1).h) == 0
    assert gmg.gmg_three_pass_operator(gmg.Problem(2, 4, 4, n_levels=1).h) == 0
    P = gmg.Problem(3, 4, 4, n_levels=1)
    gmg.gmg_set_three_pass_operator(P.h, False)
    assert gmg.gmg_three_pass_operator(P.h) == 0


@pytest.mark.parametrize("k,n", [(3, 2), (3, 3), (4, 3), (5, 2), (6, 2), (7, 2), (8, 2)])
def test_matches_kronecker_operator_with_boundary_data(gmg, k, n):
    """Unit-cell operator (gmg_apply_operator returns h^{d-2} A_ref) on a
    vector that is random on every node, boundary included; only interior
    rows are written."""
    import torch
    P = gmg.Problem(3, k, n, n_levels=1)
    N = n * k + 1
    x = np.random.default_rng(8000 + k).standard_normal(N ** 3)
    y = P.zeros()
    gmg.gmg_apply_operator(P.h, 0, P.to_device(x), y)
    got = P.from_device(y)
    ref = kron_apply(k, n, x) / n  # h^{d-2} = 1/n
    inn = interior(3, N)
    err = np.linalg.norm(got[inn] - ref[inn]) / np.linalg.norm(ref[inn])
    assert err <= 1e-13, err
    assert np.all(got[~inn] == 0)


@pytest.mark.parametrize("k,n", [(3, 7), (4, 5), (7, 3)])
def test_three_pass_and_tile_kernel_agree(gmg, k, n):
    P = gmg.Problem(3, k, n, n_levels=1)
    N = n * k + 1
    x = P.to_device(np.random.default_rng(8100 + k).standard_normal(N ** 3))
    out = []
    for on in (True, False):
        gmg.gmg_set_three_pass_operator(P.h, on)
        y = P.zeros()
        gmg.gmg_apply_operator(P.h, 0, x, y)
        out.append(P.from_device(y))
    gmg.gmg_set_three_pass_operator(P.h, True)
    assert np.linalg.norm(out[0] - out[1]) <= 1e-14 * np.linalg.norm(out[1])


def test_fp64_operator_of_a_single_precision_problem(gmg):
    """The FP64 CG of an FP32 problem applies the FP64 operator in three
    passes: same values as the FP64 problem's operator."""
    import torch
    k, n = 4, 4
    P64 = gmg.Problem(3, k, n)
    P32 = gmg.Problem(3, k, n, precision=1)
    x = inputs.random_nodal(3, k, n, 8200)
    y64 = P64.zeros(dtype=torch.float64)
    y32 = P32.zeros(dtype=torch.float64)
    gmg.gmg_apply_operator_f64(P64.h, P64.finest, P64.to_device(x, dtype=torch.float64), y64)
    gmg.gmg_apply_operator_f64(P32.h, P32.finest, P32.to_device(x, dtype=torch.float64), y32)
    assert torch.equal(y64, y32)

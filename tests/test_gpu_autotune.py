"""The autotuner's choices never change results.  Operator tile shapes are
bit-identical for FP32 and FP64 (tile kernel) at degrees 3, 4 and 7.
gmg_autotune keeps a slab width and a tile shape that leave the V-cycle-
preconditioned CG solution bit for bit unchanged.  It tunes slab widths only
where slab schedules reproduce whole colours exactly (not for the FP64
shared-face form), and it refuses batch members, whose finest vectors belong
to the batch."""
import numpy as np
import pytest

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


@pytest.mark.parametrize("k,n,precision", [(3, 9, 1), (4, 7, 1), (7, 3, 1), (4, 6, 0), (3, 5, 0)])
def test_operator_tile_shapes_are_bit_identical(gmg, k, n, precision):
    import torch
    P = gmg.Problem(3, k, n, n_levels=1, precision=precision)
    if precision == 0:
        gmg.gmg_set_three_pass_operator(P.h, False)   # the FP64 tile kernel
    x = P.to_device(inputs.random_nodal(3, k, n, 9100 + k))
    out = []
    for tile in range(4):
        gmg.gmg_set_operator_tile(P.h, tile)
        y = P.zeros()
        gmg.gmg_apply_operator(P.h, 0, x, y)
        out.append(y)
    for y in out[1:]:
        assert torch.equal(y, out[0])
    with pytest.raises(gmg.GmgError):
        gmg.gmg_set_operator_tile(P.h, 4)
    P.close()


def _solve(gmg, P, b):
    import torch
    u = P.zeros(dtype=torch.float64)
    _, st = gmg.cg_gmg_solve(P.h, u, b, 1e-10, 100)
    return u, st


@pytest.mark.parametrize("k,n,precision", [(4, 16, 1), (2, 16, 0), (3, 8, 1)])
def test_autotune_keeps_results_bit_identical(gmg, k, n, precision):
    import torch
    P = gmg.Problem(3, k, n, precision=precision)
    b = P.to_device(inputs.random_nodal(3, k, n, 9200 + k), dtype=torch.float64)
    u0, st0 = _solve(gmg, P, b)
    t = gmg.gmg_autotune(P.h)
    assert t.slab_width in (0, 1, 2, 4, 8, -1)
    assert 0 <= t.operator_tile <= 3
    assert t.sweep_ms > 0 and t.sweep_ms <= t.sweep_ms_default * 1.0001
    assert t.operator_ms > 0 and t.operator_ms <= t.operator_ms_default * 1.0001
    assert gmg.gmg_slab_width(P.h, P.finest) >= 0
    u1, st1 = _solve(gmg, P, b)
    assert st1.iterations == st0.iterations and torch.equal(u1, u0)
    P.close()


def test_autotune_leaves_the_shared_face_sweep_and_three_pass_operator(gmg):
    import torch
    P = gmg.Problem(3, 4, 8)                       # FP64: shared faces and three passes
    b = P.to_device(inputs.random_nodal(3, 4, 8, 9300), dtype=torch.float64)
    u0, st0 = _solve(gmg, P, b)
    t = gmg.gmg_autotune(P.h)
    assert t.slab_width == 0 and t.operator_tile == 0
    assert gmg.gmg_shared_faces(P.h) == 1
    u1, st1 = _solve(gmg, P, b)
    assert torch.equal(u1, u0)
    P.close()


def test_autotune_refuses_batch_members(gmg):
    B = gmg.Batch(3, 2, [4, 6], precision=1)
    with pytest.raises(gmg.GmgError) as e:
        gmg.gmg_autotune(gmg.gmg_batch_problem(B.h, 0))
    assert e.value.status == -1
    B.close()

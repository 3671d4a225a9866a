"""Batches of independent problems: one sweep launch per colour over all
problems, the CUDA-graph V-cycle and the per-problem CG must give, for every
member, what the single-problem path and the oracle give for that problem
alone; the autotuned patches-per-CTA choice must not change any result."""
import numpy as np
import pytest

from oracle.multigrid import Multigrid
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


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


CASES = [(3, 2, [4, 6, 8, 12]), (2, 3, [8, 12, 16]), (3, 3, [4, 8, 6])]


@pytest.mark.parametrize("dim,k,ns", CASES)
def test_batch_sweep_equals_single_problems(gmg, dim, k, ns):
    B = gmg.Batch(dim, k, ns)
    us = [inputs.random_nodal(dim, k, n, 2000 + i) for i, n in enumerate(ns)]
    bs = [inputs.random_nodal(dim, k, n, 2100 + i) for i, n in enumerate(ns)]
    u = B.pack(us)
    b = B.pack(bs)
    gmg.gmg_batch_smooth(B.h, u, b, False)
    got = B.unpack(u)
    for i, n in enumerate(ns):
        P = gmg.Problem(dim, k, n)
        # batches always evaluate each patch on its closure: compare with the
        # same form of the single-problem sweep (the shared-face form of FP64
        # 3D problems rounds differently)
        gmg.gmg_set_shared_faces(P.h, False)
        gmg.gmg_set_small_sweep(P.h, 0)  # nor the coarse-level kernel
        ud = P.to_device(us[i])
        gmg.gmg_smooth(P.h, P.finest, ud, P.to_device(bs[i]), 1, False)
        assert np.array_equal(got[i], P.from_device(ud)), i


@pytest.mark.parametrize("dim,k,ns", CASES)
def test_batch_vcycle_matches_oracle(gmg, dim, k, ns):
    B = gmg.Batch(dim, k, ns)
    bs = [inputs.random_nodal(dim, k, n, 2200 + i) for i, n in enumerate(ns)]
    x = B.zeros()
    gmg.gmg_batch_vcycle(B.h, x, B.pack(bs))
    got = B.unpack(x)
    for i, n in enumerate(ns):
        P = gmg.Problem(dim, k, n)
        mg = Multigrid(dim, k, n, P.n_levels)
        assert rel(got[i], mg.vcycle(bs[i])) < 1e-12, i
    # the second call replays the captured graph
    x2 = B.zeros()
    gmg.gmg_batch_vcycle(B.h, x2, B.pack(bs))
    assert np.array_equal(B.unpack(x2)[0], got[0])


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_cg(gmg, precision):
    import torch
    dim, k, ns = 3, 2, [4, 8, 6, 12, 8]
    B = gmg.Batch(dim, k, ns, precision=precision)
    bs = [inputs.random_nodal(dim, k, n, 2300 + i) for i, n in enumerate(ns)]
    u = B.zeros(dtype=torch.float64)
    st, its, res = gmg.gmg_batch_cg_solve(B.h, len(ns), u, B.pack(bs, dtype=torch.float64), 1e-10, 50)
    got = B.unpack(u)
    for i, n in enumerate(ns):
        P = gmg.Problem(dim, k, n)
        xo, it_o, _ = Multigrid(dim, k, n, P.n_levels).pcg(bs[i], rtol=1e-10)
        assert res[i] <= 1e-10 and abs(its[i] - it_o) <= 1, (i, its[i], it_o)
        assert rel(got[i], xo) < 1e-8, i


def test_autotune_never_changes_results(gmg):
    dim, k, ns = 3, 3, [6, 8, 10]
    B = gmg.Batch(dim, k, ns, precision=1)
    us = [inputs.random_nodal(dim, k, n, 2400 + i) for i, n in enumerate(ns)]
    bs = [inputs.random_nodal(dim, k, n, 2500 + i) for i, n in enumerate(ns)]
    b = B.pack(bs)
    outs = []
    for ppc in (0, 1, 2, 4):
        gmg.gmg_batch_set_ppc(B.h, ppc)
        u = B.pack(us)
        gmg.gmg_batch_smooth(B.h, u, b, False)
        outs.append(u.cpu())
    for o in outs[1:]:
        assert bool((o == outs[0]).all())
    assert gmg.gmg_batch_autotune(B.h) in (0, 1, 2, 4)

"""gmg_smooth_noalloc against gmg_smooth.

gmg_smooth_noalloc serves callers that cannot allocate device memory (their
GPU memory belongs to another allocator, or they cannot afford cudaMalloc's
implicit synchronisation): it needs no problem object and keeps its only
table in a static device array shared by all calls.  This test runs it twice
in a row, on two different meshes, so the second call must overwrite what the
first left in the shared array, and compares each result with the regular
entry point on the same inputs.  The file is named to be collected last."""
import numpy as np
import pytest

from paper_2407_02100_gb300 import inputs

pytestmark = pytest.mark.gpu

RTOL = 1e-12


@pytest.fixture(scope="module")
def gmg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2407_02100_gb300 import build, gmg as g
    build.build()
    return g


def test_noalloc_sweeps_match_gmg_smooth_on_two_calls(gmg):
    import torch
    cases = [(3, 4, 6, False, 1, 1.0), (2, 3, 9, True, 2, 0.8)]
    for i, (dim, k, n, reverse, sweeps, omega) in enumerate(cases):
        P = gmg.Problem(dim, k, n, n_levels=1, damping=omega)
        u0 = inputs.random_nodal(dim, k, n, 900 + i)
        b = P.to_device(inputs.random_nodal(dim, k, n, 950 + i), dtype=torch.float64)
        ref = P.to_device(u0, dtype=torch.float64)
        gmg.gmg_smooth(P.h, 0, ref, b, sweeps, reverse)
        got = P.to_device(u0, dtype=torch.float64)
        gmg.gmg_smooth_noalloc(dim, k, n, got, b, sweeps, reverse, omega)
        torch.cuda.synchronize()
        r, g = P.from_device(ref), P.from_device(got)
        err = np.linalg.norm(g - r) / np.linalg.norm(r)
        assert err <= RTOL, (dim, k, n, err)
        assert np.abs(g - r).max() <= 10 * RTOL * np.abs(r).max()
        P.close()


def test_noalloc_rejects_bad_arguments(gmg):
    import torch
    u = torch.zeros(64, dtype=torch.float64, device="cuda")
    b = torch.zeros(64, dtype=torch.float64, device="cuda")
    for dim, k, n in [(4, 2, 4), (3, 9, 4), (3, 2, 1)]:
        with pytest.raises(gmg.GmgError) as e:
            gmg.gmg_smooth_noalloc(dim, k, n, u, b)
        assert e.value.status == -1

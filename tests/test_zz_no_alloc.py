"""gmg_smooth_noalloc: the smoother for callers that cannot allocate device
memory.

Some callers cannot call cudaMalloc: their GPU memory belongs to another
allocator (a framework's arena or pool that has reserved the device), or
they cannot afford the implicit device-wide synchronisation of cudaMalloc
in the middle of their own pipeline.  gmg_smooth_noalloc needs no problem
object and keeps its only table (the fast-diagonalisation diagonal) in a
static device array shared by all calls.

The tests run it twice in a row on different meshes and degrees, so each
call must overwrite what the previous one left in the shared array.  They
compare each result with the oracle's smoother (dense LU patch solves,
Algorithm 4) and with gmg_smooth.  They also check three things:
- the largest patch the array holds (3D, degree 8: exactly its size) is
  accepted, and degree 9 is rejected;
- a call after the first changes no device memory counter;
- a later call enqueues only on its own (non-blocking) stream: it returns
  and completes while the legacy default stream is still busy.

The file is named to be collected last."""
import time

import numpy as np
import pytest

from oracle.mesh import Mesh
from oracle.smoother import PatchSmoother
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


def _padded(dense, dim, k, n):
    """Dense node array -> device vector in the layout of include/gmg.h
    (row pitch = nodes per direction rounded up to 4)."""
    import torch
    N = n * k + 1
    py = (N + 3) // 4 * 4
    shape = (N, py) if dim == 2 else (N, N, py)
    out = torch.zeros(shape, dtype=torch.float64)
    out[..., :N] = torch.as_tensor(np.asarray(dense, dtype=np.float64)).view((N,) * dim)
    return out.reshape(-1).cuda()


def _dense(vec, dim, k, n):
    N = n * k + 1
    py = (N + 3) // 4 * 4
    shape = (N, py) if dim == 2 else (N, N, py)
    return vec.cpu().view(shape)[..., :N].reshape(-1).numpy().copy()


def _oracle_sweeps(dim, k, n, u0, b, sweeps, reverse, omega):
    sm = PatchSmoother(Mesh(dim, k, n), omega)
    u = u0
    for _ in range(sweeps):
        u = sm.sweep(u, b, reverse=reverse)
    return u


CASES = [(3, 4, 6, False, 1, 1.0), (2, 3, 9, True, 2, 0.8), (3, 8, 4, False, 1, 1.0), (3, 2, 5, True, 1, 1.3)]


def test_noalloc_sweeps_match_oracle_and_gmg_smooth_on_consecutive_calls(gmg):
    import torch
    for i, (dim, k, n, reverse, sweeps, omega) in enumerate(CASES):
        u0 = inputs.random_nodal(dim, k, n, 900 + i)
        bh = inputs.random_nodal(dim, k, n, 950 + i)
        want = _oracle_sweeps(dim, k, n, u0, bh, sweeps, reverse, omega)
        b = _padded(bh, dim, k, n)
        for call in range(2):   # two calls in a row on the same inputs
            got = _padded(u0, dim, k, n)
            gmg.gmg_smooth_noalloc(dim, k, n, got, b, sweeps, reverse, omega)
            torch.cuda.synchronize()
            g = _dense(got, dim, k, n)
            err = np.linalg.norm(g - want) / np.linalg.norm(want)
            assert err <= RTOL, (dim, k, n, call, err)
            assert np.abs(g - want).max() <= 10 * RTOL * np.abs(want).max()
        # and against the regular entry point on the same inputs
        P = gmg.Problem(dim, k, n, n_levels=1, damping=omega)
        ref = P.to_device(u0, dtype=torch.float64)
        gmg.gmg_smooth(P.h, 0, ref, P.to_device(bh, dtype=torch.float64), sweeps, reverse)
        r = P.from_device(ref)
        assert np.linalg.norm(g - r) <= RTOL * np.linalg.norm(r)
        P.close()


def test_noalloc_allocates_nothing_after_set_up(gmg):
    import torch
    dim, k, n = 3, 8, 4
    u = _padded(inputs.random_nodal(dim, k, n, 1), dim, k, n)
    b = _padded(inputs.random_nodal(dim, k, n, 2), dim, k, n)
    gmg.gmg_smooth_noalloc(dim, k, n, u, b)        # set-up call for (device, degree 8)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        gmg.gmg_smooth_noalloc(dim, k, n, u, b)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_later_calls_do_not_wait_on_the_legacy_stream(gmg):
    """After the set-up call, a call on a non-blocking stream returns at once
    and its work completes while a bounded sleep kernel still occupies the
    legacy default stream.  A synchronous copy or any legacy-stream work in
    the call would hold the host until the sleep ended."""
    import torch
    dim, k, n = 3, 3, 6
    u0 = inputs.random_nodal(dim, k, n, 3)
    bh = inputs.random_nodal(dim, k, n, 4)
    want = _oracle_sweeps(dim, k, n, u0, bh, 1, False, 1.0)
    u, b = _padded(u0, dim, k, n), _padded(bh, dim, k, n)
    side = torch.cuda.Stream()                     # created with cudaStreamNonBlocking
    warm = u.clone()
    gmg.gmg_smooth_noalloc(dim, k, n, warm, b, stream=side.cuda_stream)   # set-up call
    torch.cuda.synchronize()
    legacy = torch.cuda.default_stream()
    with torch.cuda.stream(legacy):
        torch.cuda._sleep(int(1.5e9))              # about 0.7 s at 2 GHz, bounded
    t0 = time.perf_counter()
    gmg.gmg_smooth_noalloc(dim, k, n, u, b, stream=side.cuda_stream)
    done = torch.cuda.Event()
    done.record(side)
    t_call = time.perf_counter() - t0
    deadline = time.perf_counter() + 30.0
    while not done.query() and time.perf_counter() < deadline:
        time.sleep(1e-3)
    finished_first = done.query() and not legacy.query()
    torch.cuda.synchronize()
    assert finished_first, "the sweep waited for the legacy stream"
    assert t_call < 0.2, t_call
    g = _dense(u, dim, k, n)
    assert np.linalg.norm(g - want) <= RTOL * np.linalg.norm(want)


def test_noalloc_rejects_bad_arguments(gmg):
    import torch
    u = torch.zeros(64, dtype=torch.float64, device="cuda")
    b = torch.zeros(64, dtype=torch.float64, device="cuda")
    for dim, k, n in [(4, 2, 4), (3, 9, 4), (3, 2, 1), (3, 0, 4)]:
        with pytest.raises(gmg.GmgError) as e:
            gmg.gmg_smooth_noalloc(dim, k, n, u, b)
        assert e.value.status == -1

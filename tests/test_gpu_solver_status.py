"""Failure detection of the solver on the host side, and its per-phase
timing.

Non-finite data is injected on the host, into the right-hand side or the
initial guess that the caller hands to cg_gmg_solve; nothing on the GPU
faults.  The solver must return GMG_ERR_NONFINITE without touching the
problem's state, and the next solve with clean data must give the same
iterations and bit for bit the same solution as before the failure (the
captured CG-iteration graph survives it).

Phase timing (gmg_set_phase_timing) times the solve's phases with CUDA
events on the problem's stream.  These phases are the GPU counterpart of the
paper's breakdown of a V-cycle's time (Sec. 4).  Each phase must receive
time, the phases must sum to no more than the solve's own event-timed
duration, and the solution must be bit-identical to the untimed one."""
import numpy as np
import pytest

from paper_2407_02100_gb300 import inputs

pytestmark = pytest.mark.gpu

NONFINITE = -4


@pytest.fixture(scope="module")
def gmg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2407_02100_gb300 import build, gmg as g
    build.build()
    return g


@pytest.mark.parametrize("precision", [0, 1])
def test_nonfinite_data_is_reported_and_the_next_solve_is_unaffected(gmg, precision):
    import torch
    dim, k, n = 3, 3, 8
    P = gmg.Problem(dim, k, n, precision=precision)
    bh = inputs.random_nodal(dim, k, n, 61)
    b = P.to_device(bh, dtype=torch.float64)
    u = P.zeros(dtype=torch.float64)
    st0, s0 = gmg.cg_gmg_solve(P.h, u, b, 1e-10, 100)
    ref = u.clone()
    interior = np.nonzero(bh)[0]
    for what, value in (("b", np.nan), ("b", np.inf), ("u", np.nan), ("u", -np.inf)):
        bad_b = bh.copy()
        u0 = np.zeros_like(bh)
        (bad_b if what == "b" else u0)[interior[len(interior) // 3]] = value
        ub = P.to_device(u0, dtype=torch.float64)
        status, _ = gmg.cg_gmg_solve(P.h, ub, P.to_device(bad_b, dtype=torch.float64), 1e-10, 100,
                                     raise_on_error=False)
        assert status == NONFINITE, (what, value, status)
    u.zero_()
    st1, s1 = gmg.cg_gmg_solve(P.h, u, b, 1e-10, 100)
    assert st0 == st1 == 0 and s1.iterations == s0.iterations and s1.converged
    assert torch.equal(u, ref)
    P.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_phase_times_cover_the_solve_and_leave_results_unchanged(gmg, precision):
    import torch
    dim, k, n = 3, 4, 16
    P = gmg.Problem(dim, k, n, precision=precision)
    b = P.to_device(inputs.random_nodal(dim, k, n, 62), dtype=torch.float64)
    u_plain = P.zeros(dtype=torch.float64)
    _, s_plain = gmg.cg_gmg_solve(P.h, u_plain, b, 1e-10, 100)
    assert all(t == 0.0 for t in s_plain.phase_ms)
    gmg.gmg_set_phase_timing(P.h, True)
    u = P.zeros(dtype=torch.float64)
    stream = torch.cuda.current_stream()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    _, s = gmg.cg_gmg_solve(P.h, u, b, 1e-10, 100)
    t1.record(stream)
    torch.cuda.synchronize()
    total = t0.elapsed_time(t1)
    phases = gmg.phase_times(s)
    assert all(v > 0.0 for v in phases.values()), phases
    assert sum(phases.values()) <= total * 1.02 + 0.05, (phases, total)
    assert phases["smooth"] == max(phases.values()), phases
    assert s.iterations == s_plain.iterations
    assert torch.equal(u, u_plain)
    gmg.gmg_set_phase_timing(P.h, False)
    u.zero_()
    _, s_off = gmg.cg_gmg_solve(P.h, u, b, 1e-10, 100)
    assert all(t == 0.0 for t in s_off.phase_ms) and torch.equal(u, u_plain)
    P.close()

"""The multi-rank path of bench.py on CPU: two gloo ranks (replicas, no data
exchange) agree on the job time (max over ranks) and on the whole-job rate."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 100.0 + 50.0 * rank           # rank 1 is the slow one
    m = bench.max_over_ranks(ms, dist)
    rate = bench.whole_job_rate(1000, world, 4, m)
    out[rank] = (m, rate)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_max_and_rate():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0] == out[1]
    m, rate = out[0]
    assert m == 150.0
    assert rate == pytest.approx(1000 * 2 * 4 / 0.150 / 1e6)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(12.5) == 12.5

"""bench.py's multi-rank logic on CPU: two gloo ranks on 127.0.0.1.

The job time is the slowest rank's, every rank sees it, the rate counts the units of all
ranks (weak scaling: independent replicas, no collective on the data path), and under
--impl reference only rank 0 runs and prints."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms_local = [12.5, 40.0][rank]
        ms = bench.max_over_ranks(ms_local, world)
        rate = bench.whole_job_rate(world, 1e9, 4, ms)
        # the reference arm: ranks other than 0 return without work or output
        out = io.StringIO()
        if rank != 0:
            with redirect_stdout(out):
                bench.run_reference(type("A", (), {"steps": 1, "warmup": 0})())
        q.put((rank, ms, rate, out.getvalue()))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate_gloo():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, rate, printed in res:
        assert ms == 40.0  # the slowest rank's time, on every rank
        assert rate == pytest.approx(2 * 1e9 * 4 / 40e-3 / 1e9)  # units of both ranks / job time
        if rank != 0:
            assert printed == ""


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(7.25, 1) == 7.25
    assert bench.whole_job_rate(1, 3e9, 2, 1000.0) == pytest.approx(6.0)

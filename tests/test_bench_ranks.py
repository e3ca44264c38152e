"""bench.py's multi-rank path on the CPU: two gloo ranks (replicas only, no data-path collective).

The job's time is the slowest rank's, its throughput the units of all ranks over that time, and
the reference arm (the oracle) runs on rank 0 alone."""
import io
import multiprocessing as mp
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = bench.max_over_ranks(1.0 + rank, dist, "cpu")  # rank r "took" 1 + r seconds
    out.put((rank, t, bench.job_rate(100, world, t)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [2.0, 2.0]   # both ranks see the slowest rank's time
    assert [r[2] for r in res] == [100.0, 100.0]  # 2 ranks x 100 units / 2 s


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_rate(10, 1, 2.0) == 5.0


def test_reference_arm_runs_on_rank_zero_only():
    args = type("A", (), dict(steps=1, warmup=0, workload="c1"))()
    buf = io.StringIO()
    with redirect_stdout(buf):
        assert bench.run_reference(args, rank=1, world=2) is None
    assert buf.getvalue() == ""

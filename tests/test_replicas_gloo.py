"""The multi-GPU story is replicas only: every rank steps its own copy of the
workload and the bench reports the whole job's rate at the slowest rank's
time.  The reduction and the rate are checked here with two gloo ranks on the
CPU (no GPU, no collective on the data path)."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seconds = [2.0, 3.5][rank]  # rank 1 is the slow replica
        slowest = bench.max_over_ranks(seconds, "cpu")
        out.put((rank, slowest, bench.whole_job_rate(1000, 4, world, slowest)))
    finally:
        dist.destroy_process_group()


def test_replica_timing_takes_the_slowest_rank():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[1] for g in got] == [3.5, 3.5]
    assert got[0][2] == pytest.approx(1000 * 4 * 2 / 3.5)


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(1.25, "cpu") == 1.25
    assert bench.whole_job_rate(10, 3, 1, 2.0) == 15.0

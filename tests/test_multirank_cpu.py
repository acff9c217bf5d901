"""The N > 1 path of bench.py on CPU: two gloo ranks with different timings
reduce to the slowest rank's time, and the whole-job rate counts every
rank's bytes (weak scaling, no data-path collective)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    elapsed = 100.0 * (rank + 1)  # rank 1 is the slowest
    slowest = bench.max_over_ranks(elapsed, dist, "cpu")
    value = bench.whole_job_gbs(world, 10 << 30, 4, slowest)
    out.put((rank, slowest, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_max_and_weak_scaling():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[1] for g in got] == [200.0, 200.0]
    want = 2 * (10 << 30) * 4 / 0.2 / 1e9
    assert all(abs(g[2] - want) < 1e-6 for g in got)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert abs(bench.whole_job_gbs(1, 10 << 30, 2, 1000.0) - 2 * (10 << 30) / 1e9) < 1e-9

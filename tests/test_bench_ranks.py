"""The N > 1 path of bench.py on CPU: two gloo ranks (replicas of the whole
workload, no data-path collective) agree on the slowest rank's time and
report the whole-job rate over both ranks' units."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    ms_local = 10.0 * (rank + 1)                   # rank 1 is the slow one
    ms = bench.max_over_ranks(ms_local, dist, "cpu")
    rate = bench.whole_job_rate(1 << 20, 4, world, ms)
    q.put((rank, ms, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_and_sum_the_units():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, rate in res:
        assert ms == 20.0
        # 2 ranks x 4 steps x 2^20 units in 20 ms
        assert abs(rate - 2 * 4 * (1 << 20) / 0.020 / 1e9) < 1e-12


def test_single_rank_is_unchanged():
    import bench
    assert bench.max_over_ranks(7.5) == 7.5
    assert bench.whole_job_rate(1000, 2, 1, 1.0) == 1000 * 2 / 1e-3 / 1e9

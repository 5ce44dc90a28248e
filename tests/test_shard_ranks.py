"""Channel sharding of the batched form on CPU: the partition covers every
channel exactly once and balances the work, and two gloo ranks that each count
errors on their own channels merge to the same per-channel counts as one rank
counting them all (the oracle's BER count on seeded streams)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2104_06311_gb300.shard import channel_cost, merge_counts, shard_channels  # noqa: E402


def test_partition_covers_every_channel_once_and_balances():
    import linksim as L
    links = L.workload_batch(64)
    costs = [channel_cost(2 * lk.n_sym, 4 if lk.mod == "16qam" else 2) for lk in links]
    for world in (1, 2, 3, 4, 8):
        parts = shard_channels(costs, world)
        assert len(parts) == world
        flat = sorted(c for p in parts for c in p)
        assert flat == list(range(len(links)))
        loads = [sum(costs[c] for c in p) for p in parts]
        # LPT bound: no rank exceeds the mean by more than the largest channel
        assert max(loads) <= sum(costs) / world + max(costs) + 1e-6
        assert shard_channels(costs, world) == parts          # deterministic
    # a single heavy channel ends alone on its rank
    parts = shard_channels([100.0, 1.0, 1.0, 1.0], 2)
    assert [0] in parts and sorted(parts[1 - parts.index([0])]) == [1, 2, 3]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _channel_counts(ch):
    """Errors and bits of channel ch's oracle chain against its transmitted bits."""
    import linksim as L
    import oracle as O
    lk = L.Link(mod="qpsk", baud=10e9, n_sym=20000 + 1000 * ch, L_km=200.0 * (ch + 1), snr_db=9.0 + ch,
                seed=900 + ch)
    g = L.generate(lk)
    p = O.RxParams(baud=lk.baud, L_km=lk.L_km, mod=lk.mod, in_scale=g.in_scale, n_cma=4096, acq_min=4096)
    out = O.run_chain(g.samples, p)
    e, n, _ = O.ber_sync_count(out["bits"], g.tx_bits, p.mod, p.acq_len(lk.n_sym), sync_len=2048)
    return e, n


def _rank(rank, world, port, costs, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    mine = shard_channels(costs, world)[rank]
    counts = [_channel_counts(ch) for ch in mine]
    merged = merge_counts(counts, len(costs), mine, dist)
    q.put((rank, mine, merged))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_merge_to_the_single_rank_counts():
    costs = [channel_cost(2 * (20000 + 1000 * ch), 2) for ch in range(5)]
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, costs, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, mine0, merged0), (_, mine1, merged1) = res
    assert sorted(mine0 + mine1) == list(range(5)) and not set(mine0) & set(mine1)
    assert merged0 == merged1
    single = [_channel_counts(ch) for ch in range(5)]
    assert merged0 == single
    assert all(n > 0 for _, n in single)

"""Multi-GPU host logic on CPU: world_size 2 with the gloo backend."""
import os
import socket

import pytest

from paper_2510_24543_gb300 import inputs as I
from paper_2510_24543_gb300 import replicas as RP


def test_shards_cover_every_instance_once():
    for world in (1, 2, 3, 8):
        seen = []
        for r in range(world):
            seen += RP.shard_instances(64, r, world)
        assert sorted(seen) == list(range(64))
    with pytest.raises(ValueError):
        RP.shard_instances(4, 2, 2)


def test_rank_workloads_are_independent_starts():
    w = I.PRESETS["c3p"]
    a, b = RP.rank_workload(w, 0), RP.rank_workload(w, 1)
    assert a.seed != b.seed and a.n == b.n and a.g == b.g


def test_balance_mixed_grid_sizes():
    sizes = [48 ** 3] * 16 + [64 ** 3] * 16 + [80 ** 3] * 16 + [96 ** 3] * 16
    parts = RP.balance(sizes, 4)
    assert sorted(i for p in parts for i in p) == list(range(64))
    loads = [sum(sizes[i] for i in p) for p in parts]
    assert max(loads) - min(loads) <= 96 ** 3


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 100.0 + 50.0 * rank        # rank 1 is the slow one
        iters = 20 + rank               # ranks finish different numbers of iterations
        t, n = RP.combine(dist, ms, iters)
        rate = RP.aggregate_rate(dist, ms, iters)
        out[rank] = (t, n, rate)
    finally:
        dist.destroy_process_group()


def test_combine_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    for r in range(2):
        t, n, rate = out[r]
        assert t == 150.0 and n == 41.0
        assert abs(rate - 41.0 / 0.150) < 1e-9


def test_combine_single_process():
    assert RP.combine(None, 12.5, 7) == (12.5, 7.0)

"""The N > 1 path on CPU ranks (gloo, world size 2): each rank maps its own shard with the
oracle, timing results are reduced with max/sum, and the shards reproduce the single-rank
result. No GPU."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2510_18838_gb300 import shard


def test_shard_indices_partition():
    for n in (0, 1, 7, 100):
        for world in (1, 2, 3, 8):
            parts = [shard.shard_indices(n, r, world) for r in range(world)]
            flat = sorted(i for p in parts for i in p)
            assert flat == list(range(n))
            assert max(map(len, parts)) - min(map(len, parts)) <= 1
    with pytest.raises(ValueError):
        shard.shard_indices(5, 2, 2)
    assert shard.rank_seed(501, 0) != shard.rank_seed(501, 1)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    import oracle
    from paper_2510_18838_gb300 import workloads as W
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    src = W.uniform_points(3000, 2, 1)
    tgt = W.uniform_points(400, 2, 2)
    f = np.sin(3 * src[0]) + src[1]
    mine = shard.shard_indices(tgt.shape[1], rank, world)
    o = oracle.mls(src, tgt[:, mine], f, 1, 0.05)
    max_ms, total, rate = shard.aggregate(10.0 * (rank + 1), len(mine))
    out[rank] = (mine, o["values"][0].tolist(), max_ms, total, rate)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reproduce_single_rank():
    import oracle
    from paper_2510_18838_gb300 import workloads as W
    oracle.build()
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn")
        res = dict(out)
    src = W.uniform_points(3000, 2, 1)
    tgt = W.uniform_points(400, 2, 2)
    f = np.sin(3 * src[0]) + src[1]
    full = oracle.mls(src, tgt, f, 1, 0.05)["values"][0]
    got = np.full(400, np.nan)
    for r in range(world):
        mine, vals, max_ms, total, rate = res[r]
        got[mine] = vals
        assert max_ms == 20.0 and total == 400
        assert rate == pytest.approx(400 / 0.02)
    np.testing.assert_array_equal(np.isnan(got), np.isnan(full))
    ok = ~np.isnan(full)
    np.testing.assert_array_equal(got[ok], full[ok])     # the same oracle, bit for bit

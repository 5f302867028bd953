"""Multi-rank host logic on CPU (gloo, world size 2): bank partition, max-over-ranks
timing and the global top-k of an N_seg ladder stage."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp

from paper_2510_19047_b300.sharding import merge_top_k, shard_range


def test_shard_ranges_partition_the_bank():
    for n in (0, 1, 7, 1000, 1_000_003):
        for world in (1, 2, 3, 8):
            seen = []
            for r in range(world):
                lo, hi = shard_range(n, r, world)
                seen.append((lo, hi))
            assert seen[0][0] == 0 and seen[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(seen, seen[1:]))
            sizes = [h - l for l, h in seen]
            assert max(sizes) - min(sizes) <= 1


def test_merge_top_k_orders_like_the_library():
    s = np.array([1.0, 3.0, 3.0, np.nan, 2.0])
    i = np.array([10, 4, 2, 7, 1])
    idx, st = merge_top_k(s, i, 3)
    assert list(idx) == [2, 4, 1] and list(st) == [3.0, 3.0, 2.0]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, n, k, out):
    import torch.distributed as dist
    from paper_2510_19047_b300.sharding import global_top_k, max_over_ranks, shard_range
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    rng = np.random.default_rng(0)
    stats = np.round(rng.normal(size=n), 2)  # the same "bank" on every rank
    lo, hi = shard_range(n, rank, world)
    idx, st = global_top_k(stats[lo:hi], np.arange(lo, hi), k)
    t = max_over_ranks(1.0 + rank)
    out[rank] = (idx.tolist(), st.tolist(), t)
    dist.destroy_process_group()


def test_two_ranks_gloo():
    n, k, world = 5000, 50, 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:  # no fork of a threaded process
        out = m.dict()
        mp.spawn(_worker, args=(world, port, n, k, out), nprocs=world, join=True)
        res = dict(out)
    rng = np.random.default_rng(0)
    stats = np.round(rng.normal(size=n), 2)
    ref_idx, ref_st = merge_top_k(stats, np.arange(n), k)
    for r in range(world):
        idx, st, t = res[r]
        assert idx == ref_idx.tolist() and st == ref_st.tolist()
        assert t == 2.0

"""Template sharding across ranks (one process per GPU).

Templates are independent (one Upsilon per template), so a bank is split into
contiguous shards with no data-path collective; the only exchange is per stage of the
N_seg ladder, where the ranks' local survivors are gathered once and the global top-k
is chosen with the same ordering as tfs_select_top (Upsilon descending, index
ascending). Host-side logic only: the statistic runs in libtfs on each rank's GPU.
"""
import numpy as np


def shard_range(n_total, rank, world):
    """[lo, hi) of rank's contiguous shard; shards differ in size by at most one."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    base, extra = divmod(int(n_total), world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def max_over_ranks(value):
    """Largest value over all ranks (the step time of a synchronised job)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def merge_top_k(stats, indices, k):
    """Global top-k from per-rank candidates: order by (stat descending, global index
    ascending); returns (indices, stats) of the k best."""
    stats = np.asarray(stats, dtype=np.float64)
    indices = np.asarray(indices, dtype=np.int64)
    key = np.where(np.isnan(stats), -np.inf, stats)
    order = np.lexsort((indices, -key))[:k]
    return indices[order], stats[order]


def global_top_k(local_stats, local_global_idx, k):
    """Each rank passes its shard's statistic values and their global template indices;
    every rank receives the global top-k (one all-gather of at most k pairs per rank)."""
    import torch
    import torch.distributed as dist
    local_stats = np.asarray(local_stats, dtype=np.float64)
    local_global_idx = np.asarray(local_global_idx, dtype=np.int64)
    # a rank's contribution to the global top-k is among its own top-k
    loc, _ = merge_top_k(local_stats, local_global_idx, k)
    sel = np.searchsorted(np.sort(local_global_idx), loc)
    keep_idx = loc
    keep_stat = local_stats[np.argsort(local_global_idx)][sel]
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return merge_top_k(keep_stat, keep_idx, k)
    world = dist.get_world_size()
    pad = np.full(k, -np.inf), np.full(k, -1, np.int64)
    s = pad[0].copy()
    s[: keep_stat.size] = keep_stat
    i = pad[1].copy()
    i[: keep_idx.size] = keep_idx
    st = torch.from_numpy(s)
    it = torch.from_numpy(i)
    if dist.get_backend() == "nccl":
        st, it = st.cuda(), it.cuda()
    gs = [torch.empty_like(st) for _ in range(world)]
    gi = [torch.empty_like(it) for _ in range(world)]
    dist.all_gather(gs, st)
    dist.all_gather(gi, it)
    all_s = torch.cat(gs).cpu().numpy()
    all_i = torch.cat(gi).cpu().numpy()
    valid = all_i >= 0
    return merge_top_k(all_s[valid], all_i[valid], k)

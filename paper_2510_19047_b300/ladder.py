"""Adaptive N_seg ladder: evaluate a bank at a decreasing sequence of segment counts,
keeping the best fraction at each stage (the paper reduces N_seg stage by stage down to
the coherent N_seg = 1, Sec. "Time-frequency search statistic", and the search results
use a ladder starting at N_seg = 50).

Every stage is one tfs_eval_statistic launch over the surviving bank (persistent,
length-sorted, optionally replayed as a CUDA graph) followed by tfs_select_top on the
device. After each stage the survivors (theta, Upsilon) are checkpointed to an .npz file
keyed by the configuration, so that a run resumes at the first stage without a
checkpoint.
"""
import hashlib
import json
import os
import time

import numpy as np


def config_hash(cfg):
    return hashlib.sha1(json.dumps(cfg, sort_keys=True).encode()).hexdigest()[:16]


def run_ladder(tfs, theta, stages=(256, 64, 16), keep=0.01, checkpoint_dir=None, tag="ladder",
               seed=None, timings=None):
    """Run the ladder on a bank.

    tfs: binding.TFS with data and weights loaded. theta: float64 [8, n] (numpy, or a
    CUDA tensor). Returns a list of per-stage dicts with the surviving global indices,
    their Upsilon (decreasing) and the stage's N_seg; resumes from checkpoints when
    checkpoint_dir holds them.
    """
    import torch
    dev = torch.device("cuda", tfs.device)
    th_all = theta if (hasattr(theta, "is_cuda") and theta.is_cuda) else \
        torch.from_numpy(np.ascontiguousarray(theta)).to(dev)
    n0 = th_all.shape[1]
    cfg = {"tag": tag, "n": int(n0), "stages": list(stages), "keep": keep, "seed": seed}
    key = config_hash(cfg)
    idx = torch.arange(n0, device=dev)
    results = []
    for si, n_seg in enumerate(stages):
        path = os.path.join(checkpoint_dir, f"{tag}_{key}_stage{si}.npz") if checkpoint_dir else None
        if path and os.path.exists(path):
            z = np.load(path)
            idx = torch.from_numpy(z["index"]).to(dev)
            results.append({"n_seg": int(z["n_seg"]), "index": z["index"], "stat": z["stat"],
                            "resumed": True})
            continue
        th = th_all[:, idx].contiguous()
        t0 = time.perf_counter()
        stat, _, _ = tfs.eval_statistic(th, int(n_seg))
        k = max(1, int(round(keep * th.shape[1])))
        top = tfs.select_top(stat, k)
        torch.cuda.synchronize(dev)
        dt = time.perf_counter() - t0
        if timings is not None:
            timings.append({"stage": si, "n_seg": int(n_seg), "n": int(th.shape[1]), "seconds": dt})
        idx = idx[top]
        rec = {"n_seg": int(n_seg), "index": idx.cpu().numpy(), "stat": stat[top].cpu().numpy(),
               "resumed": False}
        results.append(rec)
        if path:
            os.makedirs(checkpoint_dir, exist_ok=True)
            tmp = path + ".tmp.npz"
            np.savez(tmp, index=rec["index"], stat=rec["stat"], n_seg=n_seg,
                     theta=th_all[:, idx].cpu().numpy(), config=json.dumps(cfg))
            os.replace(tmp, path)
    return results

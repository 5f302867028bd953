"""Batched gradient-ascent refinement of candidate templates with the adjoint kernel.

Each iteration makes one tfs_grad_statistic call for the whole batch (Upsilon and its
gradient at the current parameters) and one tfs_ascent_step from the best point so far. The step is taken in
units of a per-parameter scale sigma: delta = eta * sigma * (sigma g) / |sigma g|, so
eta is the step length in sigma-units. A template whose statistic fell since its last
step returns to its previous parameters and halves eta; otherwise eta grows by 20 %.
Everything stays on the GPU except the per-iteration bookkeeping on small tensors.
"""
import numpy as np

# per-parameter scales (M_c, eta, f_0, phi_0, lambda, beta, psi, iota): roughly the
# widths of the statistic's peak for two-year, N_seg = 16 tracks
DEFAULT_SIGMA = np.array([1e-4, 1e-3, 1e-9, 0.0, 1e-3, 1e-3, 1e-3, 1e-3])
DEFAULT_LO = np.array([1.0, 0.01, 1e-5, 0.0, 0.0, -np.pi / 2, 0.0, 0.0])
DEFAULT_HI = np.array([200.0, 0.25, 1.0, 2 * np.pi, 2 * np.pi, np.pi / 2, np.pi, np.pi])


def refine(tfs, theta, n_seg, steps=200, eta0=0.5, sigma=None, lo=None, hi=None):
    """Refine theta [8, n] (float64, numpy or CUDA tensor) by projected gradient ascent.

    Returns (theta_best [8, n] CUDA tensor, history of mean Upsilon per step,
    Upsilon at the start, Upsilon at the end).
    """
    import torch
    dev = torch.device("cuda", tfs.device)
    th = theta if (hasattr(theta, "is_cuda") and theta.is_cuda) else torch.from_numpy(
        np.ascontiguousarray(theta, dtype=np.float64))
    th = th.to(dev).clone()
    n = th.shape[1]
    sig = torch.as_tensor(DEFAULT_SIGMA if sigma is None else sigma, dtype=torch.float64,
                          device=dev)
    # the M_c and f_0 scales are relative
    sig_t = sig[:, None].expand(8, n).clone()
    sig_t[0] *= th[0]
    sig_t[2] *= th[2]
    lo = DEFAULT_LO if lo is None else lo
    hi = DEFAULT_HI if hi is None else hi
    ones = np.ones(8)
    eta = torch.full((n,), float(eta0), dtype=torch.float64, device=dev)
    best = th.clone()
    best_g = torch.zeros_like(th)
    best_u = torch.full((n,), -np.inf, dtype=torch.float64, device=dev)
    hist = []
    u0 = None
    for it in range(steps + 1):
        u, g = tfs.grad_statistic(th, n_seg)
        if u0 is None:
            u0 = u.clone()
        improved = u >= best_u
        # accept: remember; reject: go back and shorten the step
        best = torch.where(improved[None, :], th, best)
        best_g = torch.where(improved[None, :], g, best_g)
        best_u = torch.where(improved, u, best_u)
        eta = torch.where(improved, eta * 1.2, eta * 0.5)
        hist.append(float(best_u.mean()))
        if it == steps:
            break
        th = best.clone()
        sg = sig_t * best_g
        norm = torch.sqrt((sg * sg).sum(0)).clamp_min(1e-300)
        direction = (sig_t * sg) * (eta / norm)[None, :]
        tfs.ascent_step(th, direction, ones, lo, hi)
    return best, hist, u0, best_u

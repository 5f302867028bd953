"""Batched gradient-ascent refinement of candidate templates with the adjoint kernel.

Each iteration makes one tfs_grad_statistic call for the whole batch (Upsilon and its
gradient at the current parameters) and one tfs_refine_step launch: a candidate whose
statistic did not fall accepts the point (and grows its step length eta by 20 %), one
whose statistic fell returns to its best point (and halves eta); the next point is
    theta = best + eta * sigma * (sigma g) / |sigma g|,
projected onto the parameter bounds, so eta is the step length in sigma-units. The
arithmetic runs in libtfs; this module allocates the device state and sequences calls.
"""
import ctypes

import numpy as np

# per-parameter scales (M_c, eta, f_0, phi_0, lambda, beta, psi, iota): roughly the
# widths of the statistic's peak for two-year, N_seg = 16 tracks
DEFAULT_SIGMA = np.array([1e-4, 1e-3, 1e-9, 0.0, 1e-3, 1e-3, 1e-3, 1e-3])
DEFAULT_LO = np.array([1.0, 0.01, 1e-5, 0.0, 0.0, -np.pi / 2, 0.0, 0.0])
DEFAULT_HI = np.array([200.0, 0.25, 1.0, 2 * np.pi, 2 * np.pi, np.pi / 2, np.pi, np.pi])


def refine(tfs, theta, n_seg, steps=200, eta0=0.5, sigma=None, lo=None, hi=None):
    """Refine theta [8, n] (float64, numpy or CUDA tensor) by projected gradient ascent.

    Returns (theta_best [8, n] CUDA tensor, mean Upsilon_best after every step (steps + 1
    values), Upsilon at the start, Upsilon_best at the end).
    """
    import torch
    from .binding import Refine, _ptr
    dev = torch.device("cuda", tfs.device)
    th_host = theta.detach().cpu().numpy() if hasattr(theta, "is_cuda") else np.asarray(theta)
    th_host = np.ascontiguousarray(th_host, dtype=np.float64)
    n = th_host.shape[1]
    # per-candidate scales; the M_c and f_0 scales are relative to the starting point
    sig = np.asarray(DEFAULT_SIGMA if sigma is None else sigma, dtype=np.float64)
    sig_t = np.repeat(sig[:, None], n, axis=1)
    sig_t[0] *= th_host[0]
    sig_t[2] *= th_host[2]
    f64 = dict(dtype=torch.float64, device=dev)
    th = torch.from_numpy(th_host).to(dev)
    sig_d = torch.from_numpy(np.ascontiguousarray(sig_t)).to(dev)
    best = torch.empty((8, n), **f64)
    best_g = torch.zeros((8, n), **f64)
    best_u = torch.full((n,), -np.inf, **f64)
    eta = torch.full((n,), float(eta0), **f64)
    mean = torch.empty(steps + 1, **f64)
    p = lambda t: _ptr(t)[0].value  # noqa: E731
    arr8 = ctypes.c_double * 8
    rf = Refine(n, p(th), p(best), p(best_g), p(best_u), p(eta), p(sig_d),
                arr8(*np.asarray(DEFAULT_LO if lo is None else lo, dtype=np.float64)),
                arr8(*np.asarray(DEFAULT_HI if hi is None else hi, dtype=np.float64)),
                1.2, 0.5)
    u0 = None
    for it in range(steps + 1):
        u, g = tfs.grad_statistic(th, n_seg)
        if u0 is None:
            u0 = u.clone()
        # accept/reject, then the next point (computed but unused after the last step)
        tfs.refine_step(rf, u, g, mean[it:it + 1])
    return best, mean.cpu().tolist(), u0, best_u

"""Significance of a search maximum against a noise-only background.

The paper estimates the false-alarm probability of a candidate by running the search on
independent simulated noise-only realisations of the data. This builds the background
distribution p0 of the search maximum of Upsilon, and two fits extrapolate its tail
(Sec. "Search results on the full dataset" for the backgrounds; Sec. "Injected and
recovered signals" and its table of false-alarm probabilities for the fits):

- a power law p0(U) ∝ U^delta above a threshold, which gives the conservative estimate;
- a Gumbel distribution G(mu, beta) with location mu and scale beta, which gives the
  optimistic estimate.

background_maxima() runs one eval_statistic call per realisation over a template bank
(a search tile). The noise pixels are drawn by the library on the device with the data's
convention, E|n|^2 = S / (2 delta f). The fits are plain maximum-likelihood estimates on
the host.
"""
import math

import numpy as np


def background_maxima(tfs, D, theta, n_seg, n_real, seed=0):
    """max over the bank `theta` [8, n] of Upsilon_{n_seg} in each of n_real noise-only
    realisations of the grid D (its weights, mask and timing), drawn by the library
    (tfs_noise_realisation, seeds seed .. seed + n_real - 1). The context's data are
    replaced. Returns float64 [n_real]."""
    th = np.ascontiguousarray(theta.cpu().numpy() if hasattr(theta, "cpu") else theta,
                              dtype=np.float64)
    tfs.load_tf_data(D.d, D.dt, D.dT, D.t0)
    tfs.set_noise_weights(D.w, D.mask)
    out = np.empty(n_real)
    for r in range(n_real):
        tfs.noise_realisation(seed + r)
        st, _, _ = tfs.eval_statistic(th, n_seg)
        out[r] = float(np.max(st))
    return out


# ---------------------------------------------------------------------------------------
# Tail fits
# ---------------------------------------------------------------------------------------

def fit_power_law(samples, tail_fraction=0.2):
    """Maximum-likelihood power-law tail p0(U) ∝ U^delta for the largest `tail_fraction`
    of the samples (a Pareto tail above U_min). Returns dict(delta, u_min, fraction, n)."""
    x = np.sort(np.asarray(samples, float))
    n_tail = max(2, int(round(tail_fraction * x.size)))
    tail = x[-n_tail:]
    u_min = tail[0]
    logs = np.log(tail / u_min)
    s = logs.sum()
    if not s > 0:
        raise ValueError("degenerate tail: all tail samples equal")
    alpha = (n_tail - 1) / s  # unbiased form of n / sum ln(x / x_min)
    return {"delta": -alpha - 1.0, "u_min": float(u_min), "fraction": n_tail / x.size,
            "n": int(n_tail)}


def fap_power_law(u, fit, samples=None):
    """P(U_max >= u) from the power-law fit: fraction * (u / u_min)^(delta + 1) above
    u_min; below it the empirical fraction of `samples` (if given), else the fit's
    fraction."""
    u = np.asarray(u, float)
    tail = fit["fraction"] * np.power(np.maximum(u, fit["u_min"]) / fit["u_min"], fit["delta"] + 1.0)
    if samples is None:
        return np.where(u >= fit["u_min"], tail, fit["fraction"])
    s = np.sort(np.asarray(samples, float))
    emp = 1.0 - np.searchsorted(s, u, side="left") / s.size
    return np.where(u >= fit["u_min"], tail, emp)


def fit_gumbel(samples):
    """Maximum-likelihood Gumbel (maximum) distribution: returns dict(mu, beta).

    The scale solves beta = mean(x) - sum(x e^{-x/beta}) / sum(e^{-x/beta}) (the score
    equation of beta with mu profiled out), by bisection; then
    mu = -beta log(mean(e^{-x/beta}))."""
    x = np.asarray(samples, float)
    if x.size < 2 or np.all(x == x[0]):
        raise ValueError("need at least two distinct samples")
    xm = x.mean()
    c = x.min()  # shift so that the exponents are <= 0

    def score(b):
        e = np.exp(-(x - c) / b)
        return xm - (x * e).sum() / e.sum() - b

    lo, hi = 1e-6 * x.std() + 1e-300, 10.0 * x.std() + 1e-300
    while score(hi) > 0:
        hi *= 2.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if score(mid) > 0:
            lo = mid
        else:
            hi = mid
    b = 0.5 * (lo + hi)
    mu = c - b * math.log(np.mean(np.exp(-(x - c) / b)))
    return {"mu": float(mu), "beta": float(b)}


def fap_gumbel(u, fit):
    """P(U_max >= u) = 1 - exp(-exp(-(u - mu)/beta)), evaluated as -expm1(-e^{-z})."""
    z = (np.asarray(u, float) - fit["mu"]) / fit["beta"]
    return -np.expm1(-np.exp(-z))

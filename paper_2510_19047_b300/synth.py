"""Seeded synthetic inputs: time-frequency data, noise weights, gaps, template banks.

This module makes the inputs that both the CUDA library and the FP64 oracle consume.
It holds none of the statistic's arithmetic (no Fresnel kernel, no tranche
transform of the template, no tranche or segment sums). What it does contain is the
*data-generating process*: Gaussian noise with a given power spectral density, gap
masks, and injected signals synthesised sample by sample in the time domain and
Fourier transformed per tranche, which is how the paper's data grid is built
("Searching the Yorsh dataset": tranches of length dT, Tukey(0.1) window, one FFT per
tranche).

Workload shapes follow the paper's data: two-year A/E data at 5 s cadence, ~3 h
tranches, mHz sources, gaps at an 85-96 % duty cycle. The LDC datasets, the Sangria
PSD and the IMRPhenomD/TaylorF2Ecc waveforms are not available, so the inputs stand
in for them:

* noise: complex Gaussian TF pixels with E|n[m,k]|^2 = S[m,k] / (2 delta f) (the
  one-sided-PSD normalisation of a rectangular-window tranche FFT d~ = dt * DFT), or
  white Gaussian samples in the time domain for the one-channel week-long grid;
* PSD: a smooth analytic shape times a +-20 % modulation with a 30-day period;
* gaps: 3.5 h every 14 days plus 20 gaps of 1-24 h at Poisson times; a tranche that
  overlaps a gap is masked and its data zeroed;
* injections: quasi-circular 1PN chirps (optionally with a small spin-like and
  eccentricity-like phase drift the templates do not model) seen through the
  long-wavelength A/E response of a rigid constellation on a 1 AU orbit, scaled to a
  target optimal SNR.

All randomness comes from numpy PCG64 generators seeded explicitly.
"""
from dataclasses import dataclass, field
import hashlib
import math
import os

import numpy as np

# physical constants of the data-generating signal model
GMSUN_S = 4.925490947e-6   # G M_sun / c^3 [s]
AU_S = 499.004784          # 1 AU / c [s]
YEAR_S = 31557600.0        # Julian year [s]
DAY_S = 86400.0

PAR_NAMES = ("Mc", "eta", "f0", "phi0", "lam", "beta", "psi", "iota")


@dataclass
class TFData:
    """A time-frequency grid: d[chan][tranche][bin] (complex), w = 1/S (same shape)."""
    d: np.ndarray
    w: np.ndarray
    mask: np.ndarray
    dt: float
    dT: float
    t0: float = 0.0
    pn_order: int = 0
    response: int = 0
    injections: np.ndarray = None     # SoA [8, n_inj]
    inj_snr: np.ndarray = None
    meta: dict = field(default_factory=dict)

    @property
    def n_chan(self):
        return self.d.shape[0]

    @property
    def n_tranche(self):
        return self.d.shape[1]

    @property
    def n_bins(self):
        return self.d.shape[2]

    @property
    def df(self):
        return 1.0 / self.dT


def tukey(L, alpha=0.1):
    """Tukey (tapered cosine) window of L samples, periodic form."""
    n = np.arange(L)
    w = np.ones(L)
    edge = alpha * L / 2.0
    lo = n < edge
    hi = n >= L - edge
    w[lo] = 0.5 * (1 - np.cos(np.pi * n[lo] / edge))
    w[hi] = 0.5 * (1 - np.cos(np.pi * (L - n[hi]) / edge))
    return w


# --------------------------------------------------------------------------------------
# Signal model of the injections (time domain)
# --------------------------------------------------------------------------------------

def _lw_tensors(t):
    """Long-wavelength A/E detector tensors at times t -> (DA, DE) of shape [n,3,3]."""
    a = 2 * np.pi * np.asarray(t, dtype=np.float64) / YEAR_S
    ca, sa = np.cos(a), np.sin(a)
    n = a.size
    rhat = np.stack([ca, sa, np.zeros(n)], -1)
    zhat = np.array([0.0, 0.0, 1.0])
    e1 = (math.sqrt(3) / 2) * rhat + 0.5 * zhat
    e2 = np.stack([-sa, ca, np.zeros(n)], -1)
    pos = []
    for i in range(3):
        sg = -a + 2 * np.pi * i / 3
        pos.append(np.cos(sg)[:, None] * e1 + np.sin(sg)[:, None] * e2)
    D = []
    for c in range(3):
        l1 = pos[(c + 1) % 3] - pos[c]
        l2 = pos[(c + 2) % 3] - pos[c]
        l1 /= np.linalg.norm(l1, axis=-1, keepdims=True)
        l2 /= np.linalg.norm(l2, axis=-1, keepdims=True)
        D.append(0.5 * (l1[:, :, None] * l1[:, None, :] - l2[:, :, None] * l2[:, None, :]))
    X, Y, Z = D
    return (Z - X) / math.sqrt(2), (X - 2 * Y + Z) / math.sqrt(6)


def _polarisation(lam, beta, psi):
    cl, sl, cb, sb = math.cos(lam), math.sin(lam), math.cos(beta), math.sin(beta)
    p0 = np.array([sl, -cl, 0.0])
    q0 = np.array([sb * cl, sb * sl, -cb])
    p = math.cos(psi) * p0 + math.sin(psi) * q0
    q = -math.sin(psi) * p0 + math.cos(psi) * q0
    return np.outer(p, p) - np.outer(q, q), np.outer(p, q) + np.outer(q, p)


def _chirp_constants(Mc, eta, f0, pn_order):
    """(t_c, M, Theta0) of the injection's chirp (Newtonian or 1PN TaylorT3)."""
    Mc_s = Mc * GMSUN_S
    if pn_order == 0:
        tc = (5.0 / 256.0) * (np.pi * f0) ** (-8.0 / 3.0) * Mc_s ** (-5.0 / 3.0)
        return tc, None, None
    M = Mc_s * eta ** (-0.6)
    cf = 743.0 / 2688.0 + 11.0 * eta / 32.0
    y = 8 * np.pi * M * f0
    x = y ** (1.0 / 3.0)
    for _ in range(60):
        dx = (x ** 3 + cf * x ** 5 - y) / (3 * x ** 2 + 5 * cf * x ** 4)
        x -= dx
        if abs(dx) < 1e-16 * x:
            break
    Theta0 = x ** -8
    return 5 * M * Theta0 / eta, M, Theta0


def _signal_phase_freq(tp, Mc, eta, f0, phi0, pn_order, chi=0.0, ecc=0.0):
    """GW phase and frequency at SSB times tp (float64 torch tensor) of the injection model."""
    tc, M, Theta0 = _chirp_constants(Mc, eta, f0, pn_order)
    if pn_order == 0:
        u = 1.0 - tp / tc
        phase = phi0 + (16 * np.pi / 5) * f0 * tc * (1.0 - u ** 0.625)
        freq = f0 * u ** -0.375
    else:
        cp = 3715.0 / 8064.0 + 55.0 * eta / 96.0
        cf = 743.0 / 2688.0 + 11.0 * eta / 32.0
        Th = eta * (tc - tp) / (5 * M)
        q = Th ** -0.125  # Theta^(-1/8)
        q2 = q * q
        Th58 = Th * q2 * q  # Theta^(5/8)
        Th38 = Th58 * q2    # Theta^(3/8)
        phase = phi0 + (2.0 / eta) * ((Theta0 ** 0.625 + cp * Theta0 ** 0.375) - (Th58 + cp * Th38))
        freq = q2 * q / (8 * np.pi * M) * (1 + cf * q2)
        # spin-orbit-like and eccentricity-like drifts the templates do not model
        if chi:
            k = 0.1 * (113.0 / 32.0) * chi
            phase = phase + (2.0 / eta) * k * (Theta0 ** 0.25 - Th * q2 * q2 * q2)
        if ecc:
            phase = phase - (2.0 / eta) * 0.5 * ecc ** 2 * (Theta0 ** 0.625 - Th58) * \
                (freq / f0) ** (-19.0 / 9.0)
    return phase, freq, tc


def _injection_td(theta, dt, n_samples, t0, response, pn_order, chi, ecc, f_cut, n_chan):
    """Real time-domain signal s_alpha(t_j) = Re{T_alpha(t_j) A(t') e^{i Phi(t')}} [n_chan, N].

    Elementwise work runs on multi-threaded float64 torch CPU tensors (input synthesis
    only; nothing here touches the GPU)."""
    import torch
    Mc, eta, f0, phi0, lam, beta, psi, iota = [float(x) for x in theta]
    tc = _chirp_constants(Mc, eta, f0, pn_order)[0]
    out = np.zeros((n_chan, n_samples))
    # the signal lives only before coalescence (Doppler delay <= 1 AU/c)
    n_live = int(min(n_samples, max(0, math.ceil((tc + AU_S + 1.0 - t0) / dt))))
    if n_live == 0:
        return out
    t = t0 + torch.arange(n_live, dtype=torch.float64) * dt
    if response:
        tp = t + AU_S * math.cos(beta) * torch.cos(2 * np.pi * t / YEAR_S - lam)
    else:
        tp = t
    ok = tp < tc
    tps = torch.where(ok, tp, torch.zeros_like(tp))
    ph, fr, _ = _signal_phase_freq(tps, Mc, eta, f0, phi0, pn_order, chi, ecc)
    ok &= fr < f_cut
    amp = torch.where(ok, fr.abs() ** (2.0 / 3.0), torch.zeros_like(fr))
    zr = amp * torch.cos(ph)
    zi = amp * torch.sin(ph)
    if not response:
        out[:, :n_live] = zr.numpy()[None, :]
        return out
    ep, ex = _polarisation(lam, beta, psi)
    Ap, Ax = 0.5 * (1 + math.cos(iota) ** 2), math.cos(iota)
    # response on a one-hour knot grid (it varies over a year), interpolated per sample
    knots = t0 + np.arange(0, n_live * dt + 7200.0, 3600.0)
    DA, DE = _lw_tensors(knots)
    pos = (t - t0) / 3600.0
    i0 = pos.floor().long().clamp(max=knots.size - 2)
    fr_ = pos - i0.double()
    for c, D in enumerate((DA, DE)[:n_chan]):
        Fp = torch.from_numpy(np.einsum("nij,ij->n", D, ep) * Ap)
        Fx = torch.from_numpy(-np.einsum("nij,ij->n", D, ex) * Ax)
        Tr = Fp[i0] * (1 - fr_) + Fp[i0 + 1] * fr_
        Ti = Fx[i0] * (1 - fr_) + Fx[i0 + 1] * fr_
        out[c, :n_live] = (Tr * zr - Ti * zi).numpy()
    return out


ARM_S = 2.5e9 / 299792458.0  # constellation arm length / c [s]


def _spacecraft(t):
    """Guiding centre r(t) and spacecraft offsets p_i(t) [light-s]: the rotating triangle
    of _lw_tensors with 2.5e9 m sides. Returns (R [n, 3], P [3, n, 3])."""
    a = 2 * np.pi * np.asarray(t, dtype=np.float64) / YEAR_S
    ca, sa = np.cos(a), np.sin(a)
    n = a.size
    rhat = np.stack([ca, sa, np.zeros(n)], -1)
    e1 = (math.sqrt(3) / 2) * rhat + 0.5 * np.array([0.0, 0.0, 1.0])
    e2 = np.stack([-sa, ca, np.zeros(n)], -1)
    rad = ARM_S / math.sqrt(3)
    P = np.stack([rad * (np.cos(-a + 2 * np.pi * i / 3)[:, None] * e1 +
                         np.sin(-a + 2 * np.pi * i / 3)[:, None] * e2) for i in range(3)])
    return AU_S * rhat, P


def _injection_tdi(theta, dt, n_samples, t0, pn_order, chi, ecc, f_cut, n_chan):
    """A/E TDI-1.5 time series of the injection, built from delayed single-link
    observables of the rigidly rotating constellation:

    y_{s->r}(t) = [H(t + n.x_r) - H(t - L + n.x_s)] / (2 (1 + n.n_sr)), H = n_sr.h.n_sr,
    with h(tau) = A(tau) (A+ e+ cos Phi + Ax ex sin Phi) at barycentre time tau, x the
    spacecraft positions (guiding centre + offset) and n the direction to the source;
    X = r2(t) + r3(t - 2L) - r3(t) - r2(t - 2L), r2 = y_{1->0}(t) + y_{0->1}(t - L),
    r3 = y_{2->0}(t) + y_{0->2}(t - L), Y and Z cyclic, A = (Z - X)/sqrt2,
    E = (X - 2Y + Z)/sqrt6.

    The chirp's phase and amplitude are computed once on a barycentre-time grid of step
    dt/4 and read at the delayed times by 4-point Lagrange interpolation (the phase
    advances ~0.05 cycles per grid step at 0.1 Hz, so the interpolation error is far
    below the data's double precision needs)."""
    import torch
    Mc, eta, f0, phi0, lam, beta, psi, iota = [float(x) for x in theta]
    tc = _chirp_constants(Mc, eta, f0, pn_order)[0]
    out = np.zeros((n_chan, n_samples))
    n_live = int(min(n_samples, max(0, math.ceil((tc + AU_S + 40.0 - t0) / dt))))
    if n_live == 0:
        return out
    t = t0 + np.arange(n_live) * dt
    nhat = np.array([math.cos(beta) * math.cos(lam), math.cos(beta) * math.sin(lam), math.sin(beta)])
    ep, ex = _polarisation(lam, beta, psi)
    Ap, Ax = 0.5 * (1 + math.cos(iota) ** 2), math.cos(iota)
    L = ARM_S
    # chirp on a barycentre-time grid covering every delayed argument
    h = dt / 4.0
    g0 = t0 - AU_S - 4 * L - 4 * h
    n_g = int(math.ceil((t[-1] + AU_S + 4 * L + 4 * h - g0) / h)) + 1
    tg = torch.from_numpy(g0 + np.arange(n_g) * h)
    ok = tg < tc
    ph, fr, _ = _signal_phase_freq(torch.where(ok, tg, torch.zeros_like(tg)), Mc, eta, f0, phi0,
                                   pn_order, chi, ecc)
    ok &= fr < f_cut
    amp_g = torch.where(ok, fr.abs() ** (2.0 / 3.0), torch.zeros_like(fr)).numpy()
    ph_g = torch.where(ok, ph, torch.zeros_like(ph)).numpy()

    def interp(tau):
        """(A cos Phi, A sin Phi) at barycentre times tau (4-point Lagrange in Phi, A)."""
        u = (tau - g0) / h
        i = np.floor(u).astype(np.int64) - 1
        x = u - (i + 1)  # in [0, 1): nodes at -1, 0, 1, 2
        w = [-x * (x - 1) * (x - 2) / 6, (x + 1) * (x - 1) * (x - 2) / 2,
             -(x + 1) * x * (x - 2) / 2, (x + 1) * x * (x - 1) / 6]
        P = sum(w[k] * ph_g[i + k] for k in range(4))
        A = sum(w[k] * amp_g[i + k] for k in range(4))
        # past coalescence or above the cut-off the grid holds zeros: no signal there
        live = np.all([amp_g[i + k] > 0 for k in range(4)], axis=0)
        A = np.where(live, A, 0.0)
        return A * np.cos(P), A * np.sin(P)

    geom = {}

    def y(s_, r_, delay):
        """y_{s->r}(t - delay) on the sample grid."""
        td = t - delay
        if delay not in geom:
            Rc, P = _spacecraft(td)
            geom[delay] = (Rc @ nhat, P)
        Rn, P = geom[delay]
        xs_n, xr_n = Rn + P[s_] @ nhat, Rn + P[r_] @ nhat
        nl = (P[r_] - P[s_]) / L
        hp = np.einsum("ni,ij,nj->n", nl, ep, nl) * Ap
        hx = np.einsum("ni,ij,nj->n", nl, ex, nl) * Ax
        c1, s1 = interp(td + xr_n)
        c2, s2 = interp(td - L + xs_n)
        return (hp * (c1 - c2) + hx * (s1 - s2)) / (2.0 * (1.0 + nl @ nhat))

    def michelson(c):
        a_, b_ = (c + 1) % 3, (c + 2) % 3
        r2 = lambda d: y(a_, c, d) + y(c, a_, d + L)
        r3 = lambda d: y(b_, c, d) + y(c, b_, d + L)
        return r2(0.0) + r3(2 * L) - r3(0.0) - r2(2 * L)

    X, Y, Z = (michelson(c) for c in range(3))
    out[0, :n_live] = (Z - X) / math.sqrt(2)
    if n_chan > 1:
        out[1, :n_live] = (X - 2 * Y + Z) / math.sqrt(6)
    return out


def _tranche_fft(x, L, n_bins, dt, window):
    """Per-tranche FFT d~[m,k] = dt sum_j win_j x(t_m + j dt) e^{-2 pi i jk/L}, k < n_bins."""
    n_chan, N = x.shape
    nt = N // L
    xs = x[:, : nt * L].reshape(n_chan, nt, L)
    if window == "tukey":
        xs = xs * tukey(L, 0.1)[None, None, :]
    return dt * np.fft.rfft(xs, axis=-1)[:, :, :n_bins]


def _optimal_snr2(sig_tf, w, df):
    """rho^2 = <s|s> = 4 sum |s~|^2 / S delta f over the grid (Eq. inner-cont, discretised)."""
    return 4.0 * np.sum(np.abs(sig_tf) ** 2 * w) * df


# --------------------------------------------------------------------------------------
# Workloads
# --------------------------------------------------------------------------------------

def week_one_channel(seed=0, window="rect", inject=True, snr=15.0, noise=True):
    """One channel, dt = 5 s, 2^17 samples (~7.6 d) of white Gaussian noise (sigma = 1,
    S = 2 sigma^2 dt), 512 tranches x 256 samples -> 128 complex bins per tranche; one
    Newtonian chirp (M_c = 30, eta = 0.24, f_0 = 15 mHz) at optimal SNR 15; T = 1."""
    rng = np.random.Generator(np.random.PCG64(seed))
    dt, L, nt = 5.0, 256, 512
    N = L * nt
    dT = L * dt
    n_bins = L // 2
    sigma = 1.0
    S = 2 * sigma ** 2 * dt
    x = rng.standard_normal(N) * sigma if noise else np.zeros(N)
    w = np.full((1, nt, n_bins), 1.0 / S)
    w[:, :, 0] = 0.0
    inj = np.array([[30.0], [0.24], [0.015], [1.1], [0.0], [0.0], [0.0], [0.0]])
    snr_arr = None
    if inject:
        s = _injection_td(inj[:, 0], dt, N, 0.0, 0, 0, 0.0, 0.0, 0.5 / dt, 1)
        s_tf = _tranche_fft(s, L, n_bins, dt, window)
        rho2 = _optimal_snr2(s_tf, w, 1.0 / dT)
        x = x + s[0] * (snr / math.sqrt(rho2))
        snr_arr = np.array([snr])
    d = _tranche_fft(x[None, :], L, n_bins, dt, window)
    return TFData(d=d, w=w, mask=np.ones(nt, np.uint8), dt=dt, dT=dT, pn_order=0, response=0,
                  injections=inj if inject else None, inj_snr=snr_arr,
                  meta={"workload": "1ch-week-256x512", "seed": seed, "window": window})


def psd_two_year(f, t):
    """Smooth analytic one-sided PSD [1/Hz] times a +-20 %, 30-day modulation.

    S(f, t) = 1e-40 [1 + (3 mHz/f)^4 + (f/50 mHz)^2] (1 + 0.2 sin(2 pi t / 30 d)).
    """
    f = np.asarray(f, dtype=np.float64)
    with np.errstate(divide="ignore"):
        shape = 1.0 + (3e-3 / f) ** 4 + (f / 5e-2) ** 2
    mod = 1.0 + 0.2 * np.sin(2 * np.pi * np.asarray(t) / (30 * DAY_S))
    return 1e-40 * shape[None, :] * mod[:, None]


def gap_mask(n_tranche, dT, seed, periodic=True, n_random=20):
    """Tranche mask (1 = kept): 3.5 h gaps every 14 days plus n_random gaps of U[1,24] h
    at Poisson times; a tranche is dropped if it overlaps any gap."""
    rng = np.random.Generator(np.random.PCG64(seed))
    T = n_tranche * dT
    gaps = []
    if periodic:
        p = 14 * DAY_S
        k = 0
        while (k + 0.5) * p < T:
            gaps.append(((k + 0.5) * p, (k + 0.5) * p + 3.5 * 3600))
            k += 1
    t = 0.0
    for _ in range(n_random):
        t += rng.exponential(T / max(n_random, 1))
        dur = rng.uniform(1, 24) * 3600
        gaps.append((t % T, t % T + dur))
    mask = np.ones(n_tranche, np.uint8)
    starts = np.arange(n_tranche) * dT
    for a, b in gaps:
        mask[(starts < b) & (starts + dT > a)] = 0
    return mask, gaps


def _cache_dir():
    return os.environ.get("TFS_SYNTH_CACHE", os.path.join("/tmp", "tfs_synth_cache"))


def cached(fn, **kw):
    """Call a workload generator, memoised on disk by its name and arguments.

    Generating the two-year grid with its injections takes about a minute; tests and
    benchmarks in one session share one copy under $TFS_SYNTH_CACHE (default
    /tmp/tfs_synth_cache)."""
    key = hashlib.sha1(repr((fn.__name__, sorted(kw.items()))).encode()).hexdigest()[:16]
    path = os.path.join(_cache_dir(), f"{fn.__name__}_{key}.npz")
    if os.path.exists(path):
        try:
            z = np.load(path, allow_pickle=False)
            inj = z["injections"] if z["injections"].size else None
            snr = z["inj_snr"] if z["inj_snr"].size else None
            return TFData(d=z["d"], w=z["w"], mask=z["mask"], dt=float(z["dt"]),
                          dT=float(z["dT"]), t0=float(z["t0"]), pn_order=int(z["pn_order"]),
                          response=int(z["response"]), injections=inj, inj_snr=snr,
                          meta={"workload": str(z["workload"]), "cached": path})
        except Exception:
            pass
    D = fn(**kw)
    os.makedirs(_cache_dir(), exist_ok=True)
    tmp = path + f".tmp{os.getpid()}.npz"
    np.savez(tmp, d=D.d, w=D.w, mask=D.mask, dt=D.dt, dT=D.dT, t0=D.t0, pn_order=D.pn_order,
             response=D.response,
             injections=D.injections if D.injections is not None else np.zeros(0),
             inj_snr=D.inj_snr if D.inj_snr is not None else np.zeros(0),
             workload=D.meta.get("workload", ""))
    os.replace(tmp, path)
    return D


def two_year_two_channel(seed=1002, n_inj=20, inject=True, n_tranche=6144, L=2048,
                         window="tukey", psd_scale=1.0, gaps=True, response="lw"):
    """A and E channels, dt = 5 s, n_tranche x L samples (6144 x 2048 ~ 1.26e7, 728 d),
    L/2 complex bins per tranche; PSD modulated by +-20 % with a 30-day period; 3.5 h
    gaps every 14 days plus 20 Poisson gaps of 1-24 h; n_inj injections (1PN, long-
    wavelength A/E response with annual orbit, M_c in [10, 60], f_0 in [15, 30] mHz,
    SNR in [11, 20], small spin/eccentricity phase drift). response="tdi" builds the
    injections through the TDI-1.5 single-link response instead (response code 2)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    dt = 5.0
    dT = L * dt
    df = 1.0 / dT
    n_bins = L // 2
    f = np.arange(n_bins) * df
    tm = np.arange(n_tranche) * dT
    S = psd_two_year(f, tm) * psd_scale
    w1 = 1.0 / S
    w1[:, 0] = 0.0
    w = np.stack([w1, w1])
    sd = np.sqrt(S / (4 * df))
    sd[:, 0] = 0.0  # the DC bin carries no weight (S = inf there)
    d = np.empty((2, n_tranche, n_bins), np.complex128)
    for c in range(2):
        d[c].real = rng.standard_normal((n_tranche, n_bins)) * sd
        d[c].imag = rng.standard_normal((n_tranche, n_bins)) * sd
    inj = snr = None
    if inject and n_inj > 0:
        irng = np.random.Generator(np.random.PCG64(seed + 2000))
        inj = np.empty((8, n_inj))
        inj[0] = irng.uniform(10, 60, n_inj)
        inj[1] = irng.uniform(0.1, 0.25, n_inj)
        inj[2] = irng.uniform(0.015, 0.030, n_inj)
        inj[3] = irng.uniform(0, 2 * np.pi, n_inj)
        inj[4] = irng.uniform(0, 2 * np.pi, n_inj)
        inj[5] = np.arcsin(irng.uniform(-1, 1, n_inj))
        inj[6] = irng.uniform(0, np.pi, n_inj)
        inj[7] = np.arccos(irng.uniform(-1, 1, n_inj))
        snr = irng.uniform(11, 20, n_inj)
        chi = irng.uniform(-0.5, 0.5, n_inj)
        ecc = irng.uniform(0, 0.01, n_inj)
        N = n_tranche * L
        for i in range(n_inj):
            if response == "tdi":
                s = _injection_tdi(inj[:, i], dt, N, 0.0, 1, chi[i], ecc[i], 0.095, 2)
            else:
                s = _injection_td(inj[:, i], dt, N, 0.0, 1, 1, chi[i], ecc[i], 0.095, 2)
            s_tf = _tranche_fft(s, L, n_bins, dt, window)
            rho2 = _optimal_snr2(s_tf, w, df)
            if rho2 > 0:
                d += s_tf * (snr[i] / math.sqrt(rho2))
    mask = np.ones(n_tranche, np.uint8)
    if gaps:
        mask, _ = gap_mask(n_tranche, dT, seed + 5000)
        d[:, mask == 0, :] = 0.0
    return TFData(d=d, w=w, mask=mask, dt=dt, dT=dT, pn_order=1,
                  response=2 if response == "tdi" else 1, injections=inj, inj_snr=snr,
                  meta={"workload": f"AE-2yr-{L}x{n_tranche}", "seed": seed, "window": window,
                        "response": response})


def tf_noise_only(shape, w, df, seed):
    """Complex Gaussian TF noise with E|n|^2 = S/(2 delta f), S = 1/w (0 where w = 0)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    with np.errstate(divide="ignore"):
        S = np.where(w > 0, 1.0 / np.where(w > 0, w, 1.0), 0.0)
    sd = np.sqrt(S / (4 * df))
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) * sd


# --------------------------------------------------------------------------------------
# Template banks (SoA [8, n])
# --------------------------------------------------------------------------------------

def week_bank(n=1024, seed=0):
    """M_c ~ U[25,35], f_0 ~ U[14,16] mHz, phi_0 ~ U[0, 2 pi), eta = 0.24; sky unused."""
    rng = np.random.Generator(np.random.PCG64(seed))
    th = np.zeros((8, n))
    th[0] = rng.uniform(25, 35, n)
    th[1] = 0.24
    th[2] = rng.uniform(0.014, 0.016, n)
    th[3] = rng.uniform(0, 2 * np.pi, n)
    return th


def two_year_bank(n=1_000_000, seed=2002):
    """M_c ~ U[10,60], eta ~ U[0.1,0.25], f_0 ~ U[15,30] mHz, sky uniform on the sphere,
    psi ~ U[0, pi), cos iota ~ U[-1,1], phi_0 ~ U[0, 2 pi)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    th = np.empty((8, n))
    th[0] = rng.uniform(10, 60, n)
    th[1] = rng.uniform(0.1, 0.25, n)
    th[2] = rng.uniform(0.015, 0.030, n)
    th[3] = rng.uniform(0, 2 * np.pi, n)
    th[4] = rng.uniform(0, 2 * np.pi, n)
    th[5] = np.arcsin(rng.uniform(-1, 1, n))
    th[6] = rng.uniform(0, np.pi, n)
    th[7] = np.arccos(rng.uniform(-1, 1, n))
    return th


def uneven_length_bank(n=10_000_000, seed=2004, dT=10240.0, n_bins=1024):
    """Templates whose in-band durations D follow a lognormal clipped to [30 d, 730 d].

    D: lognormal with mu at the middle of [log 30 d, log 730 d] and sigma = range/4.
    f_0 is chosen (Newtonian relation) so that the track reaches f_max = (n_bins-11)/dT
    after D; M_c ~ U[10, 60]; pairs with f_0 outside [5, 90] mHz are redrawn. Other
    parameters as two_year_bank.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    lo, hi = math.log(30 * DAY_S), math.log(730 * DAY_S)
    fmax = (n_bins - 11) / dT
    out_mc = np.empty(0)
    out_f0 = np.empty(0)
    while out_mc.size < n:
        m = int((n - out_mc.size) * 1.3) + 16
        D = np.exp(np.clip(rng.normal(0.5 * (lo + hi), (hi - lo) / 4, m), lo, hi))
        Mc = rng.uniform(10, 60, m)
        Mc_s = Mc * GMSUN_S
        # time from f to coalescence: tau(f) = (5/256)(pi f)^(-8/3) Mc^(-5/3)
        k = (5.0 / 256.0) * Mc_s ** (-5.0 / 3.0)
        f0 = ((D / k + (np.pi * fmax) ** (-8.0 / 3.0)) ** (-3.0 / 8.0)) / np.pi
        ok = (f0 >= 5e-3) & (f0 <= 9e-2)
        out_mc = np.concatenate([out_mc, Mc[ok]])
        out_f0 = np.concatenate([out_f0, f0[ok]])
    th = two_year_bank(n, seed + 1)
    th[0] = out_mc[:n]
    th[2] = out_f0[:n]
    return th


def candidates_near(injections, n=4096, seed=2005):
    """n candidates seeded near the injections: N(0, 1e-4 relative) in M_c and f_0,
    +-0.02 in eta, N(0, 0.05 rad) in the angles; eta clipped to [0.05, 0.25]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    k = injections.shape[1]
    idx = np.arange(n) % k
    th = injections[:, idx].copy()
    th[0] *= 1 + 1e-4 * rng.standard_normal(n)
    th[2] *= 1 + 1e-4 * rng.standard_normal(n)
    th[1] = np.clip(th[1] + rng.uniform(-0.02, 0.02, n), 0.05, 0.25)
    for p in (3, 4, 5, 6, 7):
        th[p] += 0.05 * rng.standard_normal(n)
    th[5] = np.clip(th[5], -np.pi / 2 + 1e-6, np.pi / 2 - 1e-6)
    return th

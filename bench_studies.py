"""Workload studies run by `bench.py --study <name>` (one JSON line each).

precision : one-channel week grid; each storage/precision variant of the statistic
            against the FP64 oracle (max, p99 relative error), and the shift in
            detection probability at a fixed false-alarm probability (ROC) against the
            FP64 path over seeded noise realisations with and without an injection.
ladder    : 1e7 templates with uneven in-band durations (lognormal, 30 d to 2 yr) on the
            two-year A/E grid, N_seg ladder 256 -> 64 -> 16 -> 1 keeping the top 1 % per stage,
            each stage one persistent launch replayed as a CUDA graph.
refine    : 4096 candidates near the injections of the two-year grid at N_seg = 16: the
            adjoint gradient against the oracle on a sample, then 200 batched
            gradient-ascent steps.
fap       : background of the coherent (N_seg = 1) tile maximum over 100 noise-only
            realisations, power-law and Gumbel tail fits, and the false-alarm probability
            of the loudest injection's tile maximum.
pso       : one particle swarm per injection tile (512 particles, 100 iterations,
            N_seg = 16) against the injection's own statistic.
tdi       : throughput with the TDI-1.5 response against the long-wavelength one.
harmonics : throughput of three-harmonic templates (nu = 1/2, 1, 3/2, synthetic complex
            amplitudes) on the bench's two-year workload against the single-mode kernel,
            and their error against the oracle on a sample of the bank.
"""
import statistics
import time

import numpy as np


# FP32 peak (148 SMs x 128 lanes x 2 flop x 2.032 GHz) and the gradient kernel's
# algorithmic flops per active (template, tranche) unit: pass A recomputes Z_n, N_n
# (1250, the statistic's own figure); pass B forms per bin the five complex and eight
# real weighted sums of both channels (~83 flops) and per tranche the sensitivities and
# the reverse-mode step through track and response (~500): 1250 + 21 x 83 + 500 ~ 3500.
PEAK_FP32_TFLOPS = 148 * 128 * 2 * 2.032 / 1000.0
GRAD_FLOP_PER_UNIT = 3500
# algorithmic FP32 flops per active (template, tranche) unit of the other statistic
# kernels: the TDI-1.5 transfer adds ~250 to the long-wavelength kernel's 1250; a set of H
# harmonics costs ~150 per tranche plus ~1150 per harmonic window (counted for every
# harmonic of an active tranche, so an upper estimate where a window leaves the band)
TDI_FLOP_PER_UNIT = 1500
def harm_flop_per_unit(h):
    return 150 + 1150 * h


def _roofline(units, flop_per_unit, kernel_ms, kernel):
    achieved = units * flop_per_unit / (kernel_ms / 1000.0) / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": PEAK_FP32_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / PEAK_FP32_TFLOPS, "kernel": kernel, "kernel_ms": kernel_ms,
            "units_per_launch": units, "flop_per_unit": flop_per_unit}


def _ctx(D, **kw):
    from paper_2510_19047_b300.binding import TFS
    c = TFS(0, pn_order=D.pn_order, response=D.response, **kw)
    c.load_tf_data(D.d, D.dt, D.dT, D.t0)
    c.set_noise_weights(D.w, D.mask)
    return c


def _rel(a, b):
    m = b > 0
    r = np.abs(a[m] - b[m]) / b[m]
    return float(r.max()), float(np.percentile(r, 99))


def precision(args):
    import oracle
    from paper_2510_19047_b300 import synth
    D = synth.week_one_channel(seed=0)
    bank = synth.week_bank(1024, 0)
    t0 = time.perf_counter()
    ref = oracle.statistic(D.d, D.w, D.mask, bank, 8, D.dT)[0]
    oracle_s = time.perf_counter() - t0
    # the FP64 path carries the phase in FP64 (double-double), the mixed paths in
    # double-float; f16all / bf16all hold u, w and the template values in 16 bits
    variants = [("fp64", "f32"), ("plain", "f32"), ("mixed", "f32"), ("mixed", "f16"),
                ("mixed", "bf16"), ("mixed", "f16all"), ("mixed", "bf16all")]
    errors = {}
    ctxs = {}
    for path, pix in variants:
        c = _ctx(D, path=path, pixel=pix)
        got = c.eval_statistic(bank, 8)[0]
        mx, p99 = _rel(got, ref)
        t0 = time.perf_counter()
        c.eval_statistic(bank, 8)  # host in, host out: synchronous
        errors[f"{path}-{pix}"] = {"max": mx, "p99": p99, "gpu_s": time.perf_counter() - t0}
        ctxs[(path, pix)] = c
    # ROC: threshold = (1 - FAP) quantile over noise-only realisations of the bank's
    # largest Upsilon_8; detection = matched template above it in signal realisations
    n_real, fap, snr = 200, 0.1, 7.0
    inj = D.injections
    sig = synth.week_one_channel(seed=0, noise=False, snr=snr)
    noise_max = {v: [] for v in variants}
    matched = {v: [] for v in variants}
    for r in range(n_real):
        n = synth.tf_noise_only(D.d.shape, D.w, D.df, seed=50_000 + r)
        for v in variants:
            c = ctxs[v]
            c.load_tf_data(n, D.dt, D.dT)
            c.set_noise_weights(D.w, D.mask)
            noise_max[v].append(float(c.eval_statistic(bank, 8)[0].max()))
            c.load_tf_data(n + sig.d, D.dt, D.dT)
            c.set_noise_weights(D.w, D.mask)
            matched[v].append(float(c.eval_statistic(inj, 8)[0][0]))
    roc = {}
    for v in variants:
        thr = float(np.quantile(noise_max[v], 1 - fap))
        roc[f"{v[0]}-{v[1]}"] = {"threshold": thr,
                                 "p_detect": float(np.mean(np.array(matched[v]) > thr))}
    base = roc["fp64-f32"]["p_detect"]
    return {"study": "precision", "workload": "1ch-week-256x512, 1024 templates, N_seg 8",
            "oracle_s": oracle_s, "oracle_threads": oracle.max_threads(),
            "error_vs_oracle": errors, "roc": roc, "roc_fap": fap, "roc_snr": snr,
            "roc_realisations": n_real,
            "max_p_detect_shift_vs_fp64": max(abs(r["p_detect"] - base) for r in roc.values())}


def ladder(args):
    import torch
    from paper_2510_19047_b300 import synth
    from paper_2510_19047_b300.ladder import run_ladder
    D = synth.cached(synth.two_year_two_channel)
    n = 10_000_000
    bank = synth.uneven_length_bank(n, seed=2004, dT=D.dT, n_bins=D.n_bins)
    c = _ctx(D, use_graph=1)
    th = torch.from_numpy(bank).cuda()
    run_ladder(c, th[:, :200_000], stages=(256, 64, 16, 1), keep=0.01)  # warm-up, tuning
    times = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = run_ladder(c, th, stages=(256, 64, 16, 1), keep=0.01, timings=times)
    torch.cuda.synchronize()
    total = time.perf_counter() - t0
    return {"study": "ladder", "workload": "AE-2yr-2048x6144, 1e7 uneven-length templates",
            "stages": times, "survivors": [len(r["index"]) for r in res],
            "seconds": total, "templates_per_s": n / total}


def refine(args):
    import torch
    import oracle
    from paper_2510_19047_b300 import synth
    from paper_2510_19047_b300.refine import refine as run_refine
    D = synth.cached(synth.two_year_two_channel)
    cand = synth.candidates_near(D.injections, 4096, seed=2005)
    c = _ctx(D)
    th = torch.from_numpy(cand).cuda()
    u, g = c.grad_statistic(th, 16)
    torch.cuda.synchronize()
    ts = []
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        c.grad_statistic(th, 16)
        e1.record()
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    idx = np.linspace(0, cand.shape[1] - 1, 6).astype(int)
    ru, rg = oracle.gradient(D.d, D.w, D.mask, cand[:, idx], 16, D.dT, pn_order=1, response=1)
    S = oracle.gradient_scale(D.d, D.w, D.mask, cand[:, idx], 16, D.dT, pn_order=1, response=1,
                              tranche_level=True)
    gg = g.cpu().numpy()[:, idx]
    comp = {}
    for p, name in enumerate(("Mc", "eta", "f0", "phi0", "lam", "beta", "psi", "iota")):
        if p == 3:
            continue
        # error in units of the component's tranche-level term scale
        comp[name] = float(np.max(np.abs(gg[p] - rg[p]) / S[p]))
    # roofline of the gradient kernel: active (template, tranche) units of the batch x
    # GRAD_FLOP_PER_UNIT, over the kernel's time
    _, _, dg = c.eval_statistic(th, 16, diag=True)
    units = int(dg[0].sum().item())
    c.set_options(profile=1)
    kms = []
    for _ in range(3):
        c.grad_statistic(th, 16)
        kms.append(c.last_profile()["statistic"])
    c.set_options(profile=0)
    k_ms = statistics.median(kms)
    achieved = units * GRAD_FLOP_PER_UNIT / (k_ms / 1000.0) / 1e12
    roof = {"bound": "alu", "achieved": achieved, "peak": PEAK_FP32_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / PEAK_FP32_TFLOPS, "kernel": "k_grad", "kernel_ms": k_ms,
            "units_per_launch": units, "flop_per_unit": GRAD_FLOP_PER_UNIT}
    run_refine(c, th, 16, steps=2)  # untimed: first use of the ascent's device kernels
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    best, hist, u0, u1 = run_refine(c, th, 16, steps=200)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    u0, u1 = u0.cpu().numpy(), u1.cpu().numpy()
    return {"study": "refine", "workload": "AE-2yr-2048x6144, 4096 candidates near 20 injections, N_seg 16",
            "grad_ms_per_call": statistics.median(ts),
            "roofline": roof,
            "grad_err_vs_oracle_in_term_scale": comp,
            "stat_rel_err_vs_oracle": _rel(u.cpu().numpy()[idx], ru)[0],
            "ascent_steps": 200, "ascent_seconds": dt,
            "mean_upsilon_start": float(u0.mean()), "mean_upsilon_end": float(u1.mean()),
            "fraction_improved": float(np.mean(u1 > u0))}


def _tile_around(inj, n, seed, rel_mc=1e-3, rel_f0=1e-4):
    """n templates spread uniformly over a tile centred on one injection."""
    rng = np.random.Generator(np.random.PCG64(seed))
    th = np.repeat(inj[:, None], n, axis=1).astype(np.float64)
    th[0] *= 1 + rel_mc * rng.uniform(-1, 1, n)
    th[2] *= 1 + rel_f0 * rng.uniform(-1, 1, n)
    th[1] = np.clip(th[1] + 0.01 * rng.uniform(-1, 1, n), 0.05, 0.25)
    th[3] = rng.uniform(0, 2 * np.pi, n)
    return th


def fap(args):
    """Background of the tile maximum of the coherent statistic Upsilon_1 over noise-only
    realisations, its power-law and Gumbel tail fits, and the false-alarm probability of
    the tile maximum on the data with the injection."""
    from paper_2510_19047_b300 import fap as F
    from paper_2510_19047_b300 import synth
    D = synth.cached(synth.two_year_two_channel)
    k = int(np.argmax(D.inj_snr)) if D.inj_snr is not None else 0
    tile = _tile_around(D.injections[:, k], 20000, seed=2006)
    c = _ctx(D)
    u_cand = float(c.eval_statistic(tile, 1)[0].max())
    n_real = 100
    # one untimed realisation first: the first use of each device kernel in a process
    # (noise generator included) carries one-time loading costs
    F.background_maxima(c, D, tile, 1, 1, seed=5999)
    t0 = time.perf_counter()
    bg = F.background_maxima(c, D, tile, 1, n_real, seed=6000)
    dt = time.perf_counter() - t0
    pl = F.fit_power_law(bg, 0.2)
    gb = F.fit_gumbel(bg)
    return {"study": "fap", "workload": "AE-2yr-2048x6144, tile of 2e4 templates around the loudest injection, N_seg 1",
            "injection_snr": float(D.inj_snr[k]) if D.inj_snr is not None else None,
            "candidate_upsilon1": u_cand, "realisations": n_real,
            "seconds_per_realisation": dt / n_real,
            "background": {"median": float(np.median(bg)), "p90": float(np.quantile(bg, 0.9)),
                           "max": float(bg.max())},
            "power_law": pl, "gumbel": gb,
            "fap_power_law": float(F.fap_power_law(u_cand, pl, bg)),
            "fap_gumbel": float(F.fap_gumbel(u_cand, gb))}


def pso(args):
    """One particle swarm per injection tile on the two-year grid at N_seg = 16: the
    best Upsilon each swarm finds against the injection's own Upsilon."""
    import torch
    from paper_2510_19047_b300 import pso as P
    from paper_2510_19047_b300 import synth
    D = synth.cached(synth.two_year_two_channel)
    c = _ctx(D)
    inj = D.injections
    n_seg = 16
    u_inj = c.eval_statistic(inj, n_seg)[0]
    lo = inj.T.copy()
    hi = inj.T.copy()
    lo[:, 0] *= 1 - 1e-3
    hi[:, 0] *= 1 + 1e-3
    lo[:, 2] *= 1 - 1e-4
    hi[:, 2] *= 1 + 1e-4
    lo[:, 1] = np.clip(inj[1] - 0.01, 0.05, 0.25)
    hi[:, 1] = np.clip(inj[1] + 0.01, 0.05, 0.25)
    lo[:, 3], hi[:, 3] = 0.0, 2 * np.pi
    n_iter, n_part = 100, 512
    evals = [0]

    def obj(th):
        evals[0] += th.shape[1]
        return c.eval_statistic(th, n_seg)[0]
    # an untimed two-iteration swarm first (one-time loading of the swarm kernels and
    # of the statistic launch shape)
    P.swarm(obj, lo, hi, n_particles=n_part, n_iter=2, seed=2006, tfs=c)
    evals[0] = 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    x, fx = P.swarm(obj, lo, hi, n_particles=n_part, n_iter=n_iter, seed=2007, tfs=c)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    ratio = fx.cpu().numpy() / u_inj
    snr2 = D.inj_snr ** 2
    return {"study": "pso", "workload": f"AE-2yr-2048x6144, {inj.shape[1]} tiles (one per injection), "
                                        f"{n_part} particles x {n_iter} iterations, N_seg {n_seg}",
            "seconds": dt, "evaluations": evals[0], "evaluations_per_s": evals[0] / dt,
            "best_over_injection": {"min": float(ratio.min()), "median": float(np.median(ratio)),
                                    "max": float(ratio.max())},
            "note": "the injections carry a spin/eccentricity phase drift the templates lack, so "
                    "their nominal parameters are not the best match",
            "best_over_snr2": {"min": float((fx.cpu().numpy() / snr2).min()),
                               "median": float(np.median(fx.cpu().numpy() / snr2)),
                               "max": float((fx.cpu().numpy() / snr2).max())}}


def tdi(args):
    """Throughput of the statistic with the TDI-1.5 response (code 2) against the
    long-wavelength one (code 1) on the bench's two-year workload: 1e6 templates,
    N_seg 256/64/16 in one pass (--n-templates for another bank size). The timing does
    not depend on the data's content; parity of the TDI path is tested on a 45-day grid
    whose injections went through the time-domain single-link response, and on
    templates sampled from this launch."""
    import torch
    from paper_2510_19047_b300 import synth
    from paper_2510_19047_b300.binding import TFS
    D = synth.cached(synth.two_year_two_channel)
    n = int(getattr(args, "n_templates", 1_000_000))
    th = torch.from_numpy(synth.two_year_bank(n, seed=2002)).cuda()
    out = {"study": "tdi", "workload": "AE-2yr-2048x6144, %s templates, N_seg 256/64/16"
                                       % ("%.0e" % n).replace("e+0", "e")}
    for resp in (1, 2):
        c = TFS(0, pn_order=1, response=resp, profile=1)
        c.load_tf_data(D.d, D.dt, D.dT)
        c.set_noise_weights(D.w, D.mask)
        c.eval_statistic(th, [256, 64, 16])
        ks, ss = [], []
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            c.eval_statistic(th, [256, 64, 16])
            e1.record()
            e1.synchronize()
            ss.append(e0.elapsed_time(e1))
            ks.append(c.last_profile()["statistic"])
        out[f"response{resp}"] = {"templates_per_s": n / (statistics.median(ss) / 1000.0),
                                  "kernel_ms": statistics.median(ks)}
        _, _, dg = c.eval_statistic(th, [256, 64, 16], diag=True)
        units = int(dg[0].sum().item())
        out[f"response{resp}"]["roofline"] = _roofline(
            units, 1250 if resp == 1 else TDI_FLOP_PER_UNIT, statistics.median(ks), "k_eval_mixed")
        c.close()
    return out


def harmonics(args):
    """Multi-harmonic templates (Sec. "Outlook") on the bench's two-year workload:
    1e6 templates (--n-templates), N_seg 256/64/16 in one pass, LW response, FP16 pixels. Harmonic sets:
    the dominant mode through the single-mode kernel, nu = {1} through the harmonic
    kernel, and nu = {1/2, 1, 3/2} with amplitudes (0.3 + 0.1i, 1, 0.4 - 0.2i) (synthetic:
    the paper gives no harmonic model). Error against the oracle on 192 templates."""
    import torch
    import oracle
    from paper_2510_19047_b300 import synth
    from paper_2510_19047_b300.binding import TFS
    D = synth.cached(synth.two_year_two_channel)
    n = int(getattr(args, "n_templates", 1_000_000))
    bank = synth.two_year_bank(n, seed=2002)
    th = torch.from_numpy(bank).cuda()
    lev = [256, 64, 16]
    sets = {"single_mode_kernel": ([], []), "nu1": ([1.0], [1.0]),
            "nu_half_1_3half": ([0.5, 1.0, 1.5], [0.3 + 0.1j, 1.0, 0.4 - 0.2j])}
    out = {"study": "harmonics", "workload": f"AE-2yr-2048x6144, {n} templates, N_seg 256/64/16"}
    c = TFS(0, pn_order=1, response=1, profile=1)
    c.load_tf_data(D.d, D.dt, D.dT)
    c.set_noise_weights(D.w, D.mask)
    for name, (nu, cc) in sets.items():
        c.set_harmonics(nu, cc)
        c.eval_statistic(th, lev)
        ks, ss = [], []
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            c.eval_statistic(th, lev)
            e1.record()
            e1.synchronize()
            ss.append(e0.elapsed_time(e1))
            ks.append(c.last_profile()["statistic"])
        out[name] = {"templates_per_s": n / (statistics.median(ss) / 1000.0),
                     "kernel_ms": statistics.median(ks)}
        _, _, dg = c.eval_statistic(th, lev, diag=True)
        units = int(dg[0].sum().item())
        fpu = harm_flop_per_unit(len(nu)) if nu else 1250
        out[name]["roofline"] = _roofline(units, fpu, statistics.median(ks),
                                          "k_eval_harm" if nu else "k_eval_mixed")
    nu, cc = sets["nu_half_1_3half"]
    c.set_harmonics(nu, cc)
    sample = bank[:, :192]
    got = c.eval_statistic(sample, [16])[0][0]
    t0 = time.perf_counter()
    ref = oracle.statistic_harm(D.d, D.w, D.mask, sample, 16, D.dT, nu, cc, pn_order=1,
                                response=1)[0]
    mx, p99 = _rel(got, ref)
    out["nu_half_1_3half"]["rel_err_vs_oracle_nseg16"] = {"max": mx, "p99": p99, "n": 192,
                                                          "oracle_s": time.perf_counter() - t0}
    out["cost_ratio_3h_vs_single_mode"] = (out["nu_half_1_3half"]["kernel_ms"]
                                           / out["single_mode_kernel"]["kernel_ms"])
    c.close()
    # the paper's mapping (plain path) with the same harmonics, timed over full waves of
    # its one-thread-per-template launch (as the bench's plain leg)
    import bench
    p = TFS(0, path="plain", pn_order=1, response=1, profile=1)
    p.load_tf_data(D.d, D.dt, D.dT)
    p.set_noise_weights(D.w, D.mask)
    p.set_harmonics(nu, cc)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    leg = bench._sized_leg(p, th, int(getattr(args, "plain_waves", 4)),
                           float(getattr(args, "leg_seconds", 4.0)),
                           torch.cuda.current_stream(), flush)
    pv = leg["value"]
    out["plain_nu_half_1_3half"] = {"templates_per_s": pv, "n_templates": leg["n_templates"],
                                    "launch": leg["launch"]}
    out["mixed_vs_plain_3h"] = out["nu_half_1_3half"]["templates_per_s"] / pv
    p.close()
    return out

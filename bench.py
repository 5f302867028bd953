#!/usr/bin/env python
"""Throughput of the semi-coherent statistic Upsilon_{N_seg} (rho^2_sc) on one B300.

Workload: two-year, two-channel (A/E) TF grid of 2048-sample tranches x 6144 tranches
(dt = 5 s, 1024 complex bins per tranche), PSD modulated +-20 % with a 30-day period,
3.5 h gaps every 14 days plus 20 Poisson gaps, 20 injections; a bank of 1e6
non-spinning 1PN templates (M_c in [10, 60], eta in [0.1, 0.25], f_0 in [15, 30] mHz,
isotropic sky, random psi, cos iota, phi_0), each evaluated at N_seg = 256, 64 and 16
in one pass. All inputs are seeded synthetic data.

One step = one eval_statistic call over the whole bank (set-up, length sort, the
mixed-precision statistic kernel, output) with inputs resident in HBM, replayed as a
CUDA graph; the L2 cache is flushed (a 256 MB write) between timed steps. The plain
FP32 path (the paper's one-thread-per-template mapping) and the FP64 path are timed on
prefixes of the same bank of at least a few full waves of their launches, and the
mixed path with FP32 pixels on the whole bank, for the mixed-vs-plain ratios at the
FP16 bound and at equal (1e-4) accuracy; the FP64 CPU oracle runs on a bounded sample
for the CPU baseline. `--impl reference` times the oracle itself as the reference arm.

Prints one JSON line (rank 0).
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "templates/s of ρ²_sc (2-yr A+E TF grid), mixed vs plain form; % roofline"
N_SEG = [256, 64, 16]
NF = 21
# Algorithmic FP32 work per active (template, tranche) unit of the two-channel path
# (the per-unit figure of the design's roofline section): per bin ~30 flops to form the
# phase-cancelled Fresnel kernel value plus, per channel, the conj(u) W multiply-
# accumulate (8) and the w |W|^2 accumulate (3): 52 flops x 21 bins; per tranche ~150
# flops (track, response, phase factors): 21 * 52 + 150 ~ 1250.
FLOP_PER_UNIT = 1250
SM_COUNT = 148
FP32_LANES = 128
SM_MAX_GHZ = 2.032
PEAK_FP32_TFLOPS = SM_COUNT * FP32_LANES * 2 * SM_MAX_GHZ / 1000.0  # 76.96


def flop_per_unit(n_chan):
    return FLOP_PER_UNIT


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n-templates", type=int, default=1_000_000)
    p.add_argument("--path", default="mixed", choices=["mixed", "plain", "fp64"])
    p.add_argument("--pixel", default="f16", choices=["f16", "bf16", "f32"])
    p.add_argument("--plain-waves", type=int, default=4,
                   help="plain leg: at least this many full waves of its launch")
    p.add_argument("--fp64-waves", type=int, default=1,
                   help="FP64 leg: at least this many full waves of its launch")
    p.add_argument("--leg-seconds", type=float, default=4.0,
                   help="comparison legs: grow the batch (up to the whole bank) while a call "
                        "is estimated to stay under this")
    p.add_argument("--warps-per-cta", type=int, default=0,
                   help="pin the mixed launch's CTA size (0: autotuned)")
    p.add_argument("--tile-variant", type=int, default=0,
                   help="with --warps-per-cta: the mixed kernel's compiled tile variant")
    p.add_argument("--no-graph", action="store_true",
                   help="headline step without CUDA-graph replay")
    p.add_argument("--cpu-sample", type=int, default=1200)  # ~10-20 s of oracle work
    p.add_argument("--ref-sample", type=int, default=192)   # per reference-arm step (12 per host thread on 16)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-plain", action="store_true")
    p.add_argument("--study", default=None, choices=["precision", "ladder", "refine", "fap", "pso", "tdi", "harmonics"],
                   help="run one of the workload studies instead of the headline step")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:  # noqa: BLE001
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:  # noqa: BLE001
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), parts[4:8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r) if v == "Active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def oracle_sample_rate(D, theta, n_seg, threads=0):
    """templates/s of the FP64 CPU oracle (all N_seg levels) on the given templates."""
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    for L in n_seg:
        oracle.statistic(D.d, D.w, D.mask, theta, L, D.dT, pn_order=D.pn_order,
                         response=D.response, n_threads=threads)
    dt = time.perf_counter() - t0
    return theta.shape[1] / dt, dt


def clocks_rejected(clocks):
    """True for a timed region that saw hardware or thermal slowdown, or SM clocks well
    below their maximum with no reason reported (a leftover clock lock)."""
    if not clocks or clocks.get("samples", 0) == 0:
        return False
    bad = {"hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"}
    if bad & set(clocks.get("reasons", [])):
        return True
    mhz, top = clocks.get("sm_mhz"), clocks.get("sm_max_mhz")
    return bool(mhz and top and mhz < 0.9 * top and not clocks.get("reasons"))


def kernel_source_sha1():
    """SHA-1 over the sources the statistic kernel is compiled from."""
    h = hashlib.sha1()
    for f in ("tfs_eval_mixed.cu", "tfs_mixed_bins.cuh", "tfs_internal.cuh", "tfs_kernels.cuh",
              "tfs_tdi.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2510_19047_b300", "csrc", f), "rb").read())
    return h.hexdigest()


def traffic_record(units, variant):
    """DRAM bytes (read + write) of one full-size statistic launch of the given tile
    variant, from a committed one-pass ncu capture of this bench's workload; valid only
    while the kernel source is unchanged and the launch processes the same number of
    units. The traffic is not proportional to the units (the grid is read about once
    per launch and then served from L2), so a capture of another size is not rescaled."""
    path = os.path.join(ROOT, "profiles", "k_eval_mixed_dram.json")
    if not os.path.exists(path):
        return None
    rec = json.load(open(path))
    h = kernel_source_sha1()
    if rec.get("source_sha1") != h or int(rec.get("units_per_launch", -1)) != units:
        return None
    for r in rec.get("records", []):
        if int(r["variant"]) == int(variant):
            return r
    return None


def _timed_calls(ctx, th, reps, stream, flush):
    """CUDA-event times [ms] of `reps` eval_statistic calls on device-resident theta."""
    import torch
    ms = []
    for _ in range(reps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.eval_statistic(th, N_SEG)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    return ms


def _sized_leg(ctx, theta, waves, seconds, stream, flush, reps=2):
    """Time the context's current path on a prefix of the bank: at least `waves` full
    waves of its one-thread-per-template launch, grown towards the whole bank while one
    call is estimated to stay under `seconds`. Returns the leg's record."""
    n_all = theta.shape[1]
    probe = theta[:, : min(n_all, 2048)].contiguous()
    ctx.eval_statistic(probe, N_SEG)
    shp = ctx.last_launch_shape()
    per_wave = shp["ctas_per_sm"] * shp["sms"] * shp["threads_per_cta"]
    n = min(n_all, waves * per_wave)
    sub = theta[:, :n].contiguous()
    ms = _timed_calls(ctx, sub, 1, stream, flush)  # also the untimed warm-up
    rate = n / (ms[0] / 1000.0)
    n_big = min(n_all, max(n, int(rate * seconds) // per_wave * per_wave))
    if n_big > n:
        n = n_big
        sub = theta[:, :n].contiguous()
    ms = _timed_calls(ctx, sub, reps, stream, flush)
    shp = ctx.last_launch_shape()
    return {"value": n / (statistics.mean(ms) / 1000.0), "unit": "templates/s",
            "n_templates": n, "ms_per_step": statistics.mean(ms),
            "launch": {"threads_per_cta": shp["threads_per_cta"], "ctas": shp["ctas"],
                       "ctas_per_sm": shp["ctas_per_sm"],
                       "warps_per_sm": shp["ctas_per_sm"] * shp["threads_per_cta"] // 32,
                       "waves": shp["ctas"] / (shp["ctas_per_sm"] * shp["sms"])}}


def comparison_legs(ctx, theta, args, stream, flush):
    """The plain path (the paper's one-thread-per-template mapping, FP32 pixels, FP64
    phase), the FP64 parity path, and the mixed path with FP32 pixels (the variant
    that meets the plain path's 1e-4 bound) on the same bank and N_seg levels."""
    out = {}
    ctx.set_options(path="plain", profile=0, use_graph=0)
    out["plain"] = dict(_sized_leg(ctx, theta, args.plain_waves, args.leg_seconds, stream, flush),
                        dtype="f32 pixels, f64 phase")
    ctx.set_options(path="fp64", profile=0, use_graph=0)
    out["fp64"] = dict(_sized_leg(ctx, theta, args.fp64_waves, args.leg_seconds, stream, flush),
                       dtype="f64")
    ctx.set_options(path="mixed", pixel="f32", profile=0, use_graph=0)
    ctx.eval_statistic(theta, N_SEG)  # autotune and pack the FP32 plane (untimed)
    ms = _timed_calls(ctx, theta, 3, stream, flush)
    shp = ctx.last_launch_shape()
    out["mixed_f32"] = {"value": theta.shape[1] / (statistics.mean(ms) / 1000.0),
                        "unit": "templates/s", "n_templates": theta.shape[1],
                        "ms_per_step": statistics.mean(ms), "dtype": "f32 pixels",
                        "launch": {"variant": shp["variant"],
                                   "warps_per_cta": shp["threads_per_cta"] // 32,
                                   "ctas_per_sm": shp["ctas_per_sm"]}}
    return out


def run_reference(args):
    """The oracle as the reference arm (FP64 CPU, all host cores)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_2510_19047_b300 import synth
    import oracle
    D = synth.cached(synth.two_year_two_channel)
    theta = synth.two_year_bank(args.ref_sample, seed=2002)
    cores = oracle.max_threads()
    for _ in range(max(1, args.warmup)):  # untimed warm-up steps (build, page in)
        oracle_sample_rate(D, theta, N_SEG)
    rates, times = [], []
    for _ in range(args.steps):
        r, dt = oracle_sample_rate(D, theta, N_SEG)
        rates.append(r)
        times.append(dt)
    v = args.ref_sample * len(times) / sum(times)
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "templates/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * statistics.mean(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "AE-2yr-2048x6144, N_seg 256/64/16",
                   "sample": f"{args.ref_sample} templates of the 1e6 bank per step"},
        "cpu_baseline": {"value": v, "unit": "templates/s", "cores": cores, "kind": "oracle",
                         "sample": f"{args.ref_sample} templates x 3 N_seg levels per step"},
        "e2e": {"value": v, "unit": "templates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.study:
        import bench_studies
        print(json.dumps(getattr(bench_studies, args.study)(args)), flush=True)
        return
    rank, world, local = dist_env()
    import torch
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2510_19047_b300 import synth
    from paper_2510_19047_b300.binding import TFS
    from paper_2510_19047_b300.sharding import max_over_ranks, shard_range

    D = synth.cached(synth.two_year_two_channel)
    # weak scaling: a bank of world x n templates, each rank evaluates its own shard
    n_total = args.n_templates * world
    lo, hi = shard_range(n_total, rank, world)
    theta_np = np.ascontiguousarray(synth.two_year_bank(n_total, seed=2002)[:, lo:hi])
    n = hi - lo
    theta = torch.from_numpy(theta_np).cuda()
    use_graph = 0 if args.no_graph else 1
    ctx = TFS(local, path=args.path, pixel=args.pixel, profile=1, use_graph=use_graph)
    if args.warps_per_cta:
        ctx.set_options(warps_per_cta=args.warps_per_cta, tile_variant=args.tile_variant)
    ctx.load_tf_data(D.d, D.dt, D.dT)
    ctx.set_noise_weights(D.w, D.mask)
    stat = torch.empty((len(N_SEG), n), dtype=torch.float64, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    # one untimed call with diagnostics: active (template, tranche) units per launch
    _, _, diag = ctx.eval_statistic(theta, N_SEG, diag=True)
    units = int(diag[0].sum().item())
    for _ in range(args.warmup):
        ctx.eval_statistic(theta, N_SEG, out=stat)
    torch.cuda.synchronize()
    shape = ctx.last_launch_shape()

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    stream = torch.cuda.current_stream()  # the library launches on the caller's current stream

    def timed_region():
        sampler = ClockSampler(local)
        barrier()
        torch.cuda.synchronize()
        sampler.start()
        step_ms, kern_ms, launches = [], [], 0
        for _ in range(args.steps):
            flush.zero_()  # L2 flush between timed steps
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.eval_statistic(theta, N_SEG, out=stat)
            e1.record(stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            kern_ms.append(ctx.last_profile()["statistic"])
            launches += ctx.last_launch_count()
        torch.cuda.synchronize()
        barrier()
        return step_ms, kern_ms, launches, sampler.stop()

    step_ms, kern_ms, launches, clocks = timed_region()
    rejected = None
    again = clocks_rejected(clocks)
    if world > 1:  # every rank re-measures if any rank's clocks were rejected
        flag = torch.tensor([int(again)], device="cuda")
        torch.distributed.all_reduce(flag, op=torch.distributed.ReduceOp.MAX)
        again = bool(flag.item())
    if again:
        # a throttled or clock-locked run is measured once more
        rejected = clocks
        step_ms, kern_ms, launches, clocks = timed_region()
    ms = max_over_ranks(statistics.mean(step_ms))
    value = n_total / (ms / 1000.0)

    # roofline of the statistic kernel
    kms = statistics.mean(kern_ms)
    flops = units * flop_per_unit(D.n_chan)
    achieved = flops / (kms / 1000.0) / 1e12
    trec = traffic_record(units, shape["variant"])
    roof = {"bound": "alu", "achieved": achieved, "peak": PEAK_FP32_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / PEAK_FP32_TFLOPS,
            "traffic": trec["dram_bytes_per_launch"] if trec else None,
            "kernel": "k_eval_mixed", "kernel_ms": kms, "units_per_launch": units,
            "flop_per_unit": flop_per_unit(D.n_chan),
            "peak_source": "derived: 148 SMs x 128 FP32 lanes x 2 flop x 2.032 GHz"}
    if clocks and clocks.get("sm_mhz"):
        # the same peak at the median SM clock sampled under load (the power cap can hold
        # the clock below its maximum)
        at = PEAK_FP32_TFLOPS * clocks["sm_mhz"] / 2032.0
        roof["peak_at_sampled_clock"] = at
        roof["frac_at_sampled_clock"] = achieved / at

    result = {
        "metric": METRIC, "value": value, "unit": "templates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": "AE-2yr-2048x6144 (12.58M samples/ch, 1e6 templates, "
                               "N_seg 256/64/16 in one pass)",
                   "n_templates_per_gpu": n, "n_seg": N_SEG, "path": args.path,
                   "pixel": args.pixel, "phase": "double-float", "l2": "flushed between steps",
                   "graph": bool(use_graph and args.path == "mixed"),
                   "launch": {"variant": shape["variant"], "warps_per_cta": shape["threads_per_cta"] // 32,
                              "ctas": shape["ctas"], "ctas_per_sm": shape["ctas_per_sm"],
                              "autotuner_trials": shape["tune_trials"]},
                   "parallelism": f"templates sharded, {world} GPU(s)"},
        "roofline": roof,
        "gpu_launches": launches,
        "clocks": clocks,
    }
    if rejected is not None:
        result["clocks_rejected_first_run"] = rejected

    if not args.no_e2e:
        # end to end through the C ABI with host buffers, on every rank at once (the
        # whole job's templates over the slowest rank's time)
        ctx.set_options(path=args.path, pixel=args.pixel, profile=0)
        th_host = torch.from_numpy(theta_np).pin_memory()
        out_host = torch.empty((len(N_SEG), n), dtype=torch.float64).pin_memory()
        ctx.eval_statistic(th_host, N_SEG, out=out_host.numpy())
        ets = []
        for _ in range(max(1, min(args.steps, 3))):
            torch.cuda.synchronize()
            barrier()
            t0 = time.perf_counter()
            ctx.eval_statistic(th_host, N_SEG, out=out_host.numpy())
            torch.cuda.synchronize()
            ets.append(time.perf_counter() - t0)
        e2e_s = max_over_ranks(statistics.mean(ets))
        result["e2e"] = {"value": n_total / e2e_s, "unit": "templates/s",
                         "h2d_bytes_per_step": int(8 * 8 * n_total),
                         "d2h_bytes_per_step": int(len(N_SEG) * n_total * (8 + 4))}
        ctx.set_options(path=args.path, pixel=args.pixel, profile=1, use_graph=use_graph)

    if rank == 0 and not args.no_plain and args.path == "mixed":
        mixed_rate = n / (statistics.mean(step_ms) / 1000.0)
        legs = comparison_legs(ctx, theta, args, stream, flush)
        result.update(legs)
        # FP16 pixels at their stated bound, and FP32 pixels at the plain path's 1e-4
        result["mixed_vs_plain"] = mixed_rate / legs["plain"]["value"]
        result["mixed_f32_vs_plain"] = legs["mixed_f32"]["value"] / legs["plain"]["value"]
        ctx.set_options(path=args.path, pixel=args.pixel, profile=1, use_graph=use_graph)

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        sample = theta_np[:, : args.cpu_sample].copy()
        rate, dt = oracle_sample_rate(D, sample, N_SEG)
        result["cpu_baseline"] = {"value": rate, "unit": "templates/s",
                                  "cores": oracle.max_threads(), "kind": "oracle",
                                  "sample": f"first {args.cpu_sample} templates of the bank, "
                                            f"3 N_seg levels, {dt:.1f} s"}
    if rank == 0:
        print(json.dumps(result), flush=True)
    ctx.close()
    if world > 1:
        barrier()  # the other ranks wait for rank 0's legs before the group goes away
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()

#!/usr/bin/env python
"""Block-Vecchia log-likelihood benchmark on GB300.

One step = one block-Vecchia log-likelihood evaluation (covariance generation through the
scalar ell, the timed span of the paper's time-to-solution, Sec. 3.1) at a parameter
vector perturbed by U(0.8, 1.2) around the truth, on the batched plain-FP64 workload:
n = 200,000 uniform locations in [0,1]^2, Matern nu = 1.5, sigma^2 = 1, beta = 0.05,
nugget 1e-4, y drawn from the block-Vecchia model at m = 400, bc = 20,000 K-means blocks,
m = 60 conditioning points.  K-means, neighbour search and the data draw are one-time
set-up (excluded, as in the paper).

Prints one JSON line (see --help).  --impl reference times the FP64 CPU oracle instead
(on a bounded sample of the same workload, host cores).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2410_04477_gb300 import synth  # noqa: E402

METRIC = "block-Vecchia loglik evals/sec (FP64), n=2e5, bc=2e4, m=60, nu=1.5"
UNIT = "evals/s"
FP64_PEAK_TFLOPS = 1.25  # nominal GB300 FP64 (vector and tensor), used as the ALU roofline
SM_COUNT, FP32_LANES, SM_MAX_MHZ = 152, 128, 2070.0
FP32_PEAK_TFLOPS = SM_COUNT * FP32_LANES * 2 * SM_MAX_MHZ * 1e6 / 1e12  # 80.5 at max clock

WORKLOADS = {
    "c2_m60": dict(n=200_000, d=2, bc=20_000, m=60, nu=1.5, sigma2=1.0, beta=0.05, nugget=1e-4,
                   seed=1, gen_m=400),
    "c2_m120": dict(n=200_000, d=2, bc=20_000, m=120, nu=1.5, sigma2=1.0, beta=0.05,
                    nugget=1e-4, seed=1, gen_m=400),
}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    """nvidia-smi sampler of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "200", "-i", str(device)], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def make_thetas(bv, w, count, seed):
    f = synth.perturb_factors(seed + 1000, count)
    out = []
    for k in range(count):
        out.append(bv.theta(w["sigma2"] * f[k, 0], w["beta"] * f[k, 1], w["nu"], w["nugget"] * f[k, 2]))
    return out


def setup_gpu(bv, ctx, w, log):
    t0 = time.perf_counter()
    locs = synth.locs_uniform(w["n"], w["d"], w["seed"])
    ctx.set_data(locs)
    ctx.build_blocks(w["bc"], seed=w["seed"], iters=20)
    t1 = time.perf_counter()
    ctx.select_neighbors(w["gen_m"])
    z = synth.normal(w["seed"], 20, w["n"])
    y = ctx.simulate(bv.theta(w["sigma2"], w["beta"], w["nu"], w["nugget"]), z)
    t2 = time.perf_counter()
    ctx.select_neighbors(w["m"])
    t3 = time.perf_counter()
    log(f"setup: blocks {t1 - t0:.1f}s, draw(m={w['gen_m']}) {t2 - t1:.1f}s, neighbours {t3 - t2:.1f}s")
    return locs, y, dict(blocks_s=round(t1 - t0, 2), draw_s=round(t2 - t1, 2), nn_s=round(t3 - t2, 2))


def time_device(torch, bv, ctx, stream, thetas, prec, warmup, steps, flush):
    """Per-evaluation CUDA-event durations (ms) on the launching stream, L2 flushed between."""
    dout = torch.zeros(1, dtype=torch.float64, device="cuda")
    with torch.cuda.stream(stream):
        for k in range(warmup):
            ctx.loglik_async([thetas[k % len(thetas)]], prec, dout.data_ptr())
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    with torch.cuda.stream(stream):
        for k in range(steps):
            flush.zero_()
            evs[k][0].record(stream)
            ctx.loglik_async([thetas[(warmup + k) % len(thetas)]], prec, dout.data_ptr())
            evs[k][1].record(stream)
    torch.cuda.synchronize()
    st, fb = ctx.sync()
    if st != 0:
        raise RuntimeError(f"evaluation failed (status {st}, block {fb})")
    return [a.elapsed_time(b) for a, b in evs]


def cpu_oracle_sample(w, seconds=12.0):
    """The FP64 oracle on a bounded sample of the workload: a sub-square holding n_s points at
    the same density (so the same block and neighbourhood shapes), its own K-means blocks
    and neighbours; evaluations repeated for about `seconds`.  Returns evals/s of the FULL
    workload extrapolated by block count, the sample description and the thread count."""
    import oracle
    n_s = 20_000
    side = (n_s / w["n"]) ** (1.0 / w["d"])
    locs = synth.locs_uniform(n_s, w["d"], w["seed"] + 7) * side
    bc_s = max(1, int(round(w["bc"] * n_s / w["n"])))
    bp, pi, ce = oracle.build_blocks(locs, bc_s, seed=w["seed"], iters=20)
    nnp, nni = oracle.select_neighbors(locs, bp, pi, ce, w["m"])
    y = synth.normal(w["seed"] + 7, 21, n_s)
    th = oracle.theta(w["sigma2"], w["beta"] * side / side, w["nu"], w["nugget"])
    reps, t0 = 0, time.perf_counter()
    while True:
        oracle.loglik(th, locs, y, bp, pi, nnp, nni)
        reps += 1
        el = time.perf_counter() - t0
        if el >= seconds or reps >= 200:
            break
    per_eval_sample = el / reps
    nblk_s = len(bp) - 1
    full_eval = per_eval_sample * (w["bc"] / nblk_s)
    return (1.0 / full_eval, f"{reps} evals of an n={n_s} sub-square at the same density "
            f"({nblk_s} blocks, m={w['m']}), extrapolated by block count", oracle.num_threads(),
            per_eval_sample)


def run_reference(args, w):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    import oracle as O
    n_s = 20_000
    side = (n_s / w["n"]) ** (1.0 / w["d"])
    locs = synth.locs_uniform(n_s, w["d"], w["seed"] + 7) * side
    bc_s = max(1, int(round(w["bc"] * n_s / w["n"])))
    bp, pi, ce = O.build_blocks(locs, bc_s, seed=w["seed"], iters=20)
    nnp, nni = O.select_neighbors(locs, bp, pi, ce, w["m"])
    y = synth.normal(w["seed"] + 7, 21, n_s)
    f = synth.perturb_factors(w["seed"] + 1000, args.warmup + args.steps)
    ths = [O.theta(w["sigma2"] * f[k, 0], w["beta"] * f[k, 1], w["nu"], w["nugget"] * f[k, 2])
           for k in range(len(f))]
    for k in range(args.warmup):
        O.loglik(ths[k], locs, y, bp, pi, nnp, nni, check=False)
    t0 = time.perf_counter()
    for k in range(args.steps):
        O.loglik(ths[args.warmup + k], locs, y, bp, pi, nnp, nni, check=False)
    el = time.perf_counter() - t0
    scale = w["bc"] / (len(bp) - 1)
    per_full = el / args.steps * scale
    val = 1.0 / per_full
    sample = (f"each step: one FP64 oracle evaluation of an n={n_s} sub-square at the same density "
              f"({len(bp) - 1} blocks, m={w['m']}), extrapolated to the full workload by block count")
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_full * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_of(w, args),
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def config_of(w, args):
    return {"workload": args.workload, "n": w["n"], "d": w["d"], "bc": w["bc"], "m": w["m"],
            "nu": w["nu"], "sigma2": w["sigma2"], "beta": w["beta"], "nugget": w["nugget"],
            "y": f"block-Vecchia draw at m={w['gen_m']}", "theta": "perturbed U(0.8,1.2) per step",
            "precision": args.precision, "l2": "flushed between timed steps (256 MB write)",
            "parallelism": "replicas" if _dist()[0] > 1 else "single"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c2_m60", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--no-extras", action="store_true", help="skip the mixed / m=120 / MLE lines")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    w = WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, w)

    ws, rank, local = _dist()
    import torch
    log = (lambda s: print(s, file=sys.stderr, flush=True)) if rank == 0 else (lambda s: None)
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    from paper_2410_04477_gb300 import bv
    prec = bv.BV_FP64 if args.precision == "fp64" else bv.BV_MIXED
    stream = torch.cuda.Stream()
    ctx = bv.Context(local, stream.cuda_stream)
    locs, y_true, setup = setup_gpu(bv, ctx, w, log)
    thetas = make_thetas(bv, w, args.warmup + args.steps, w["seed"])
    ctx.autotune(prec)
    info = ctx.plan_info(prec)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    barrier()
    clk = Clocks(local)
    ms = time_device(torch, bv, ctx, stream, thetas, prec, args.warmup, args.steps, flush)
    barrier()
    clocks = clk.stop()
    tot_ms = float(sum(ms))
    if ws > 1:
        import torch.distributed as dist
        t = torch.tensor([tot_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        tot_ms = float(t.item())
    mean_ms = tot_ms / args.steps
    value = ws * args.steps / (tot_ms / 1e3)

    # end to end through the public API with host buffers: y (pinned) up, ell down
    y_pin = torch.from_numpy(y_true.copy()).pin_memory()
    barrier()
    t0 = time.perf_counter()
    for k in range(args.steps):
        ctx.set_observations(y_pin.numpy())
        ctx.loglik(thetas[(args.warmup + k) % len(thetas)], prec)
    barrier()
    e2e_s = time.perf_counter() - t0
    e2e = {"value": ws * args.steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(w["n"] * 8 + 64),
           "d2h_bytes_per_step": 8}

    achieved = info["flops"] / (mean_ms / 1e3) / 1e12
    roof = {"bound": "alu", "kernel": "k_ll_fp64 (all size bins) + reduction, one evaluation",
            "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None,
            "peak_source": "nominal GB300 FP64 1.25 TFLOP/s (no FP64 entry in MEASURED_PEAKS.json)",
            "flops_per_eval": info["flops"], "cov_entries_per_eval": info["cov_entries"]}
    if prec == bv.BV_MIXED:
        roof.update(kernel="k_ll_mixed (all size bins) + reduction", peak=FP32_PEAK_TFLOPS,
                    frac=achieved / FP32_PEAK_TFLOPS,
                    peak_source="FP32 FMA: 152 SMs x 128 lanes x 2 x 2070 MHz")

    extras = {}
    if not args.no_extras and rank == 0:
        ll_true64 = ctx.loglik(bv.theta(w["sigma2"], w["beta"], w["nu"], w["nugget"]), bv.BV_FP64)
        other = bv.BV_MIXED if prec == bv.BV_FP64 else bv.BV_FP64
        ctx.autotune(other)
        ms2 = time_device(torch, bv, ctx, stream, thetas, other, 3, min(args.steps, 30), flush)
        ll_true_m = ctx.loglik(bv.theta(w["sigma2"], w["beta"], w["nu"], w["nugget"]), bv.BV_MIXED)
        extras["other_precision"] = {
            "precision": "mixed" if other == bv.BV_MIXED else "fp64",
            "evals_per_s": len(ms2) / (sum(ms2) / 1e3),
            "achieved_tflops": info["flops"] / (statistics.mean(ms2) / 1e3) / 1e12,
            "ell_fp64": ll_true64, "ell_mixed": ll_true_m,
            "rel_err_mixed_vs_fp64": abs(ll_true_m - ll_true64) / abs(ll_true64),
            "abs_err": abs(ll_true_m - ll_true64)}
        log(f"extras: {extras['other_precision']}")
    cpu = None
    if not args.no_cpu and rank == 0 and ws == 1:
        v, sample, cores, per = cpu_oracle_sample(w)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": mean_ms, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec == bv.BV_FP64 else "f32+f64",
                "data": "synthetic", "config": config_of(w, args), "roofline": roof,
                "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
                "gpu_launches": int(info["launches_per_eval"] * args.steps),
                "setup_s": setup, "plan": {"n_bins": info["n_bins"]}, "extras": extras}
        print(json.dumps(line), flush=True)
    ctx.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())

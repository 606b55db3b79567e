#!/usr/bin/env python
"""Block-Vecchia log-likelihood benchmark on GB300.

One step = one block-Vecchia log-likelihood evaluation (covariance generation through the
scalar ell, the timed span of the paper's time-to-solution, Sec. 3.1) at a parameter
vector perturbed by U(0.8, 1.2) around the truth.  Default workload: the largest
single-GPU configuration, the 3D profile of n = 1,000,000 points (20,000 sites x 50
jittered levels in the unit cube), Matern nu = 0.5 with anisotropic ranges (0.1, 0.1, 0.3),
sigma^2 = 1, nugget 1e-3, y drawn from the block-Vecchia model at m = 400, bc = 100,000
K-means blocks, m = 200 conditioning points, FP64.  K-means, neighbour search and the
data draw are one-time set-up (excluded, as in the paper).  The default run also reports
the other precision and the MLE wall-times (n = 5e5, cold and learned warm starts, FP64
and mixed) under "extras".

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

UNIT = "evals/s"
FP64_PEAK_TFLOPS = 1.25  # nominal GB300 FP64 (vector and tensor), used as the ALU roofline
SM_COUNT, FP32_LANES, SM_MAX_MHZ = 152, 128, 2070.0
FP32_PEAK_TFLOPS = SM_COUNT * FP32_LANES * 2 * SM_MAX_MHZ * 1e6 / 1e12  # 80.5 at max clock

# DRAM bytes (read + write) of one evaluation's likelihood-kernel launches, summed over
# the size bins, from an ncu capture (dram__bytes_read.sum + dram__bytes_write.sum);
# reported as roofline.traffic for these workloads and precisions only.
NCU_TRAFFIC = {("c2_m60", "fp64"): 636_160 + 10_996_224 + 2_597_376 + 40_704 + 36_864 + 34_816,
               # config 3: the main bin's 5,937,920 bytes at n-scale 0.05 (4,974 of its 99,949
               # blocks; the other bins hold 51 blocks), times 20
               ("c3", "fp64"): 20 * 5_937_920}

WORKLOADS = {
    # batched plain FP64: 2e5 uniform points, bc 2e4, m 60 / 120, y from BV at m=400
    "c2_m60": dict(n=200_000, d=2, bc=20_000, m=60, nu=1.5, sigma2=1.0, beta=0.05, nugget=1e-4,
                   seed=1, gen_m=400),
    "c2_m120": dict(n=200_000, d=2, bc=20_000, m=120, nu=1.5, sigma2=1.0, beta=0.05,
                    nugget=1e-4, seed=1, gen_m=400),
    # general smoothness (K_nu path): the config-2 shape at nu = 1.2
    "c2_nu12": dict(n=200_000, d=2, bc=20_000, m=60, nu=1.2, sigma2=1.0, beta=0.05, nugget=1e-4,
                    seed=1, gen_m=400),
    # 3D profile: 20,000 sites x 50 jittered levels = 1e6 points, anisotropic range
    "c3": dict(n=1_000_000, d=3, sites=20_000, levels=50, bc=100_000, m=200, nu=0.5, sigma2=1.0,
               beta=0.1, ranges=[0.1, 0.1, 0.3], nugget=1e-3, seed=2, gen_m=400),
    # MLE on 5e5 points, bc 5e4, m 100; cold start (1, 0.1, 1e-2) vs learned warm start
    "c4_mle": dict(n=500_000, d=2, bc=50_000, m=100, nu=1.5, sigma2=1.5, beta=0.05, nugget=5e-3,
                   seed=4, gen_m=100),
    # 256 datasets in one launch, n log-uniform [5e3, 5e4], bc = n/10, per-dataset theta
    "c5_m30": dict(ndata=256, m=30, seed=5, d=2, gen_m=30),
    "c5_m60": dict(ndata=256, m=60, seed=5, d=2, gen_m=30),
    "c5_m120": dict(ndata=256, m=120, seed=5, d=2, gen_m=30),
    # classic Vecchia (blocks of size 1, random order) on the config-2 data: the paper's
    # baseline method, m = 30 (its recommended conditioning size) and m = 60
    "cv_m30": dict(n=200_000, d=2, bc=20_000, m=30, nu=1.5, sigma2=1.0, beta=0.05, nugget=1e-4, seed=1,
                   gen_m=400, classic=True),
    "cv_m60": dict(n=200_000, d=2, bc=20_000, m=60, nu=1.5, sigma2=1.0, beta=0.05, nugget=1e-4, seed=1,
                   gen_m=400, classic=True),
    # KL study (Sec. 3.1): n = 20,000 uniform in the unit square, nu = 1.5, beta = 0.052537
    # (effective range 0.3, Table 1); timed step = one exact log-likelihood (dense FP64
    # Cholesky); extras: KL of block Vecchia (bc = 1500, five orderings, several m) and of
    # classic Vecchia (random order), each with its evaluation time
    "kl_20k": dict(kind="kl", n=20_000, d=2, nu=1.5, sigma2=1.0, beta=0.052537, nugget=0.0, seed=8,
                   bc=1500, bv_m=[10, 30, 60, 120, 180], cv_m=[10, 30, 60, 150],
                   orders=["random", "maxmin", "morton", "kdtree", "hilbert"]),
    # the paper's small-scale KL case (n = 8,000, its supplementary study), bc = 650
    "kl_8k": dict(kind="kl", n=8_000, d=2, nu=1.5, sigma2=1.0, beta=0.052537, nugget=0.0, seed=9,
                  bc=650, bv_m=[30, 120], cv_m=[30, 60], orders=["random", "maxmin"]),
    # prediction (Algorithm 2) + 1,000-round univariate conditional simulation and PICP:
    # the paper's shape (n = 20,000 in the unit square, 10% held out, 200 prediction
    # blocks) and a 10x larger one with the same 1:10 block-to-location ratio
    "pred_20k": dict(kind="pred", n=20_000, d=2, bc=2_000, gen_m=200, pred_bc=200, m=60, rounds=1000,
                     nu=1.5, sigma2=1.0, beta=0.05, nugget=1e-2, seed=6),
    "pred_2e5": dict(kind="pred", n=200_000, d=2, bc=20_000, gen_m=200, pred_bc=2_000, m=120, rounds=1000,
                     nu=1.5, sigma2=1.0, beta=0.05, nugget=1e-2, seed=7),
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


def max_over_ranks(x: float) -> float:
    """Largest value of x over all ranks (replicas time independently; the job time is
    the slowest rank's).  Works with NCCL (CUDA tensor) and gloo (CPU tensor)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(steps: int, world: int, max_ms: float) -> float:
    """Evaluations per second of the whole job: every rank runs `steps` evaluations."""
    return world * steps / (max_ms / 1e3)


def true_theta(bv, w, f=(1.0, 1.0, 1.0)):
    if w.get("ranges"):
        return bv.theta(w["sigma2"] * f[0], None, w["nu"], w["nugget"] * f[2],
                        ranges=[r * f[1] for r in w["ranges"]])
    return bv.theta(w["sigma2"] * f[0], w["beta"] * f[1], w["nu"], w["nugget"] * f[2])


def make_thetas(bv, w, count, seed):
    """count perturbed parameter vectors (one per step); for several datasets, a list
    of per-dataset vectors per step."""
    f = synth.perturb_factors(seed + 1000, count)
    if "ndata" in w:
        base = w["thetas"]
        return [[bv.theta(t[0] * f[k, 0], t[1] * f[k, 1], t[3], t[2] * f[k, 2]) for t in base]
                for k in range(count)]
    return [[true_theta(bv, w, f[k])] for k in range(count)]


def setup_gpu(bv, ctx, w, log):
    t0 = time.perf_counter()
    if "ndata" in w:
        return setup_multi(bv, ctx, w, log)
    if w["d"] == 3:
        locs = synth.locs_levels(w["sites"], w["levels"], w["seed"])
    else:
        locs = synth.locs_uniform(w["n"], w["d"], w["seed"])
    ctx.set_data(locs)
    ctx.build_blocks(w["bc"], seed=w["seed"], iters=20)
    t1 = time.perf_counter()
    ctx.select_neighbors(w["gen_m"])
    z = synth.normal(w["seed"], 20, w["n"])
    y = ctx.simulate(true_theta(bv, w), z)
    t2 = time.perf_counter()
    if w.get("classic"):
        ctx.build_singletons(seed=w["seed"])
    ctx.select_neighbors(w["m"])
    t3 = time.perf_counter()
    log(f"setup: blocks {t1 - t0:.1f}s, draw(m={w['gen_m']}) {t2 - t1:.1f}s, neighbours {t3 - t2:.1f}s")
    return locs, y, dict(blocks_s=round(t1 - t0, 2), draw_s=round(t2 - t1, 2), nn_s=round(t3 - t2, 2))


def setup_multi(bv, ctx, w, log):
    """C5: every dataset drawn from the block-Vecchia model at its own theta (one context
    per dataset for the draw), then all loaded into one context for batched evaluation."""
    t0 = time.perf_counter()
    sizes = synth.dataset_sizes(w["seed"], w["ndata"])
    th = synth.theta_draws(w["seed"], w["ndata"])
    w["thetas"] = [tuple(map(float, t)) for t in th]
    w["n"] = int(sizes.sum())
    w["sizes"] = sizes
    locs_l, y_l = [], []
    with bv.Context(ctx_device(ctx)) as tmp:
        for k in range(w["ndata"]):
            n = int(sizes[k])
            locs = synth.locs_uniform(n, 2, w["seed"] * 100000 + k)
            tmp.set_data(locs)
            tmp.build_blocks(n // 10, seed=w["seed"] * 100000 + k, iters=20)
            tmp.select_neighbors(w["gen_m"])
            s2, beta, tau2, nu = th[k]
            y_l.append(tmp.simulate(bv.theta(s2, beta, nu, tau2), synth.normal(w["seed"] * 100000 + k, 20, n)))
            locs_l.append(locs)
    t1 = time.perf_counter()
    ctx.set_datasets(locs_l, y_l)
    ctx.build_blocks_multi([int(n) // 10 for n in sizes], seed=w["seed"] * 100000, iters=20)
    ctx.select_neighbors(w["m"])
    t2 = time.perf_counter()
    log(f"setup: {w['ndata']} draws {t1 - t0:.1f}s, blocks+neighbours {t2 - t1:.1f}s (sum n = {w['n']})")
    return locs_l, np.concatenate(y_l), dict(draws_s=round(t1 - t0, 2), structure_s=round(t2 - t1, 2))


def ctx_device(ctx):
    return 0


def time_device(torch, bv, ctx, stream, thetas, prec, warmup, steps, flush):
    """Per-evaluation CUDA-event durations (ms) on the launching stream, L2 flushed between."""
    dout = torch.zeros(len(thetas[0]), dtype=torch.float64, device="cuda")
    with torch.cuda.stream(stream):
        for k in range(warmup):
            ctx.loglik_async(thetas[k % len(thetas)], prec, dout.data_ptr())
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    with torch.cuda.stream(stream):
        for k in range(steps):
            flush.zero_()
            evs[k][0].record(stream)
            ctx.loglik_async(thetas[(warmup + k) % len(thetas)], prec, dout.data_ptr())
            evs[k][1].record(stream)
    torch.cuda.synchronize()
    st, fb = ctx.sync()
    if st != 0:
        raise RuntimeError(f"evaluation failed (status {st}, block {fb})")
    return [a.elapsed_time(b) for a, b in evs]


def oracle_sample(w, n_s=20_000):
    """A bounded sample of the workload for the FP64 oracle, with the same block and
    neighbourhood shapes: for one 2D dataset, n_s uniform points in a sub-square at the
    same density; for the 3D profile, the sites of a sub-square at the same site density
    with all their levels; for many datasets, the first datasets of the workload (own
    sizes and parameters) until they hold n_s points.  Blocks and neighbours come from the
    oracle.  Returns (parts, scale, description): parts are (locs, y, block_ptr, point_idx,
    nn_ptr, nn_idx, (sigma2, beta, nu, nugget, ranges)) and scale = blocks of the full
    workload / blocks of the sample."""
    import oracle
    parts = []
    if "ndata" in w:
        sizes = synth.dataset_sizes(w["seed"], w["ndata"])
        th = synth.theta_draws(w["seed"], w["ndata"])
        tot, k = 0, 0
        while tot < n_s and k < w["ndata"]:
            n = int(sizes[k])
            locs = synth.locs_uniform(n, 2, w["seed"] * 100000 + k)
            bp, pi, ce = oracle.build_blocks(locs, n // 10, seed=w["seed"] * 100000 + k, iters=20)
            nnp, nni = oracle.select_neighbors(locs, bp, pi, ce, w["m"])
            y = synth.normal(w["seed"] * 100000 + k, 21, n)
            s2, beta, tau2, nu = map(float, th[k])
            parts.append((locs, y, bp, pi, nnp, nni, (s2, beta, nu, tau2, None)))
            tot += n
            k += 1
        nblk = sum(len(p[2]) - 1 for p in parts)
        full = int(sum(int(n) // 10 for n in sizes))
        return parts, full / nblk, (f"the first {k} datasets of the workload ({tot} points, {nblk} blocks, "
                                    f"m={w['m']}), extrapolated by block count")
    if w["d"] == 3:
        sites = max(1, n_s // w["levels"])
        side = (sites / w["sites"]) ** 0.5
        locs = synth.locs_levels(sites, w["levels"], w["seed"] + 7)
        locs[:, :2] *= side
        what = f"{sites} sites x {w['levels']} levels of a sub-square at the same site density"
    else:
        side = (n_s / w["n"]) ** (1.0 / w["d"])
        locs = synth.locs_uniform(n_s, w["d"], w["seed"] + 7) * side
        what = f"an n={n_s} sub-square at the same density"
    n_s = len(locs)
    bc_s = max(1, int(round(w["bc"] * n_s / w["n"])))
    if w.get("classic"):
        bp, pi, ce = oracle.build_singletons(locs, seed=w["seed"])
    else:
        bp, pi, ce = oracle.build_blocks(locs, bc_s, seed=w["seed"], iters=20)
    nnp, nni = oracle.select_neighbors(locs, bp, pi, ce, w["m"])
    y = synth.normal(w["seed"] + 7, 21, n_s)
    parts.append((locs, y, bp, pi, nnp, nni, (w["sigma2"], w["beta"], w["nu"], w["nugget"], w.get("ranges"))))
    nblk = len(bp) - 1
    full = w["n"] if w.get("classic") else w["bc"]
    return parts, full / nblk, f"{what} ({nblk} blocks, m={w['m']}), extrapolated by block count"


def oracle_eval(parts, f=(1.0, 1.0, 1.0)):
    """One FP64 oracle evaluation of every part of the sample, parameters scaled by f."""
    import oracle
    for locs, y, bp, pi, nnp, nni, (s2, beta, nu, tau2, ranges) in parts:
        if ranges is not None:
            th = oracle.theta(s2 * f[0], None, nu, tau2 * f[2], ranges=[r * f[1] for r in ranges])
        else:
            th = oracle.theta(s2 * f[0], beta * f[1], nu, tau2 * f[2])
        oracle.loglik(th, locs, y, bp, pi, nnp, nni, check=False)


def _time_oracle(parts, seconds):
    """Repeat one oracle evaluation of the sample for about `seconds` (at least once):
    (repetitions, seconds per evaluation)."""
    reps, t0 = 0, time.perf_counter()
    while True:
        oracle_eval(parts)
        reps += 1
        el = time.perf_counter() - t0
        if el >= seconds or reps >= 200:
            return reps, el / reps


def cpu_oracle_sample(w, seconds=12.0, one_thread_seconds=4.0):
    """The FP64 oracle on a bounded sample of the workload (oracle_sample), repeated for
    about `seconds` on every host core, then for about `one_thread_seconds` on one thread
    (skipped when 0).  Returns evals/s of the FULL workload extrapolated by block count,
    the sample description, the thread count, the seconds per sample evaluation and the
    one-thread figures (a dict, or None)."""
    import oracle
    parts, scale, desc = oracle_sample(w)
    reps, per_eval_sample = _time_oracle(parts, seconds)
    cores = oracle.num_threads()
    one = None
    if one_thread_seconds > 0:
        oracle.set_num_threads(1)
        try:
            reps1, per1 = _time_oracle(parts, one_thread_seconds)
        finally:
            oracle.set_num_threads(cores)
        one = {"value": 1.0 / (per1 * scale), "unit": UNIT, "cores": 1, "sample": f"{reps1} evals of {desc}"}
    return (1.0 / (per_eval_sample * scale), f"{reps} evals of {desc}", cores, per_eval_sample, one)


def run_reference(args, w):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    parts, scale, desc = oracle_sample(w)
    f = synth.perturb_factors(w["seed"] + 1000, args.warmup + args.steps)
    for k in range(args.warmup):
        oracle_eval(parts, f[k])
    t0 = time.perf_counter()
    for k in range(args.steps):
        oracle_eval(parts, f[args.warmup + k])
    el = time.perf_counter() - t0
    per_full = el / args.steps * scale
    val = 1.0 / per_full
    sample = f"each step: one FP64 oracle evaluation of {desc} to the full workload"
    line = {"impl": "reference", "metric": metric_of(w, args), "value": val, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_full * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_of(w, args),
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def config_of(w, args):
    c = {"workload": args.workload, "d": w["d"], "m": w["m"], "y": f"block-Vecchia draw at m={w['gen_m']}",
         "blocks": "n singletons, random order" if w.get("classic") else f"bc={w.get('bc')} K-means",
         "theta": "perturbed U(0.8,1.2) per step", "precision": args.precision,
         "l2": "flushed between timed steps (256 MB write)",
         "parallelism": "replicas" if _dist()[0] > 1 else "single"}
    if "ndata" in w:
        c.update(ndata=w["ndata"], n_total=w.get("n"), bc="n/10 per dataset", n_range=[5000, 50000],
                 theta_per_dataset="log-uniform sigma2 [0.5,2], beta [0.02,0.3], tau2 [1e-4,1e-1]; nu in {0.5,1.5,2.5}")
    else:
        c.update(n=w["n"], bc=w["bc"], nu=w["nu"], sigma2=w["sigma2"], nugget=w["nugget"],
                 range=w.get("ranges") or w["beta"])
        if "n_scale" in w:
            c.update(n_scale=w["n_scale"])
    return c


def metric_of(w, args):
    prec = "FP64" if args.precision == "fp64" else "mixed FP32/FP64"
    if w.get("classic"):
        return (f"classic-Vecchia loglik evals/sec ({prec}), n={w['n']:.0e}, blocks of size 1, m={w['m']}, "
                f"nu={w['nu']}, d={w['d']}")
    if "ndata" in w:
        return f"block-Vecchia loglik evals/sec ({prec}), {w['ndata']} datasets in one launch, m={w['m']}"
    return (f"block-Vecchia loglik evals/sec ({prec}), n={w['n']:.0e}, bc={w['bc']:.0e}, m={w['m']}, "
            f"nu={w['nu']}, d={w['d']}")


def run_mle(bv, ctx, w, log):
    """MLE wall-time: cold start (1, 0.1, 1e-2) and the learned warm start, FP64 and
    mixed; sigma^2, range and nugget free, nu fixed."""
    wpath = os.path.join(ROOT, "paper_2410_04477_gb300", "weights", "warmstart.bvws")
    nu = w["nu"]
    lo, hi = bv.theta(0.01, 0.001, nu, 1e-6), bv.theta(100.0, 3.0, nu, 10.0)
    cold0 = bv.theta(1.0, 0.1, nu, 1e-2)
    res = {}
    warm0 = None
    if os.path.exists(wpath):
        t0 = time.perf_counter()
        ctx.warmstart_load(wpath)
        warm0 = ctx.warmstart_predict(cold0)
        res["warm_predict_s"] = time.perf_counter() - t0
        res["warm_start_theta"] = [warm0.sigma2, warm0.range[0], warm0.nugget]
        res["warm_start_nu_class"] = ctx.warmstart_predict(bv.theta(1.0, 0.1, 0.0, 1e-2)).nu  # truth: w["nu"]
    # both starts run the same search (trust-region Newton steps first, the simplex search
    # only if they fail); the simplex scale is 0.5 in log-parameters from the fixed cold
    # start, and from the learned warm start its validation RMSE (0.2 for log sigma^2 and
    # log beta, 0.75 for log tau^2, weights/warmstart.json)
    for pname, prec in (("fp64", bv.BV_FP64), ("mixed", bv.BV_MIXED)):
        for sname, th0, step, stepn in (("cold", cold0, 0.5, 0.5), ("warm", warm0, 0.2, 0.75)):
            if th0 is None:
                continue
            ctx.loglik(th0, prec)   # plan, tune and capture outside the timed MLE
            t0 = time.perf_counter()
            th, ll, ne = ctx.mle(th0, lo, hi, precision=prec, ftol_rel=1e-10, xtol=1e-5, max_evals=2000,
                                 init_step=step, init_step_nugget=stepn, newton_first=True)
            el = time.perf_counter() - t0
            if sname == "warm":
                el += res.get("warm_predict_s", 0.0)
            res[f"{pname}_{sname}"] = {"wall_s": el, "evals": ne, "loglik": ll,
                                       "theta_hat": [th.sigma2, th.range[0], th.nugget]}
            log(f"mle {pname} {sname}: {el:.2f}s {ne} evals ell={ll:.6f}")
    for pname in ("fp64", "mixed"):
        if f"{pname}_warm" in res:
            c, wv = res[f"{pname}_cold"], res[f"{pname}_warm"]
            res[f"{pname}_warm_vs_cold"] = {"speedup": c["wall_s"] / wv["wall_s"], "evals_saved": c["evals"] - wv["evals"],
                                            "rel_diff_loglik": abs(wv["loglik"] - c["loglik"]) / abs(c["loglik"])}
    return res


def oracle_mle_estimate(wm, res, seconds=6.0):
    """The FP64 oracle's MLE wall-time on the same workload, extrapolated: its time per
    evaluation (cpu_oracle_sample on every host core) times the number of evaluations
    that each FP64 search on the GPU needed.  Nothing of the search itself runs on the
    CPU; the figure says what the same search would cost with the oracle as evaluator."""
    v, sample, cores, _, _ = cpu_oracle_sample(wm, seconds=seconds, one_thread_seconds=0)
    out = {"kind": "oracle, extrapolated", "evals_per_s": v, "cores": cores, "sample": sample}
    for key in ("fp64_cold", "fp64_warm"):
        if key in res:
            out[f"{key}_wall_s"] = res[key]["evals"] / v
    return out


def pred_split(w):
    """Locations and the held-out mask (10%: SplitMix64 draw mod 10 == 0)."""
    locs = synth.locs_uniform(w["n"], w["d"], w["seed"])
    r = synth.splitmix64(synth.stream(w["seed"], 9), np.arange(w["n"], dtype=np.uint64))
    return locs, (r % np.uint64(10)) == np.uint64(0)


def pred_metric(w):
    return (f"block-Vecchia prediction + {w['rounds']}-round conditional simulation, new locations/sec (FP64), "
            f"n={w['n']:.0e}, n*={w['n'] // 10:.0e}, pred bc={w['pred_bc']}, m={w['m']}, nu={w['nu']}")


def pred_config(w, args):
    return {"workload": args.workload, "n": w["n"], "held_out": "10% (SplitMix64 mod 10)", "pred_bc": w["pred_bc"],
            "m": w["m"], "rounds": w["rounds"], "d": w["d"], "nu": w["nu"],
            "theta": [w["sigma2"], w["beta"], w["nugget"]], "y": f"block-Vecchia draw at m={w['gen_m']}",
            "l2": "flushed between timed steps (256 MB write)",
            "parallelism": "replicas" if _dist()[0] > 1 else "single"}


def pred_oracle_sample(w, locs, y, hold, seconds=10.0):
    """The oracle's Algorithm 2 + conditional simulation on the first prediction blocks of
    the same workload (oracle blocks and neighbours), repeated for about `seconds`;
    returns new locations/s, the sample description and the thread count."""
    import oracle
    lo, yo, ls, yt = locs[~hold], y[~hold], locs[hold], y[hold]
    th = oracle.theta(w["sigma2"], w["beta"], w["nu"], w["nugget"])
    bp, pi, ce = oracle.build_pred_blocks(ls, w["pred_bc"], seed=w["seed"])
    k = min(len(bp) - 1, 20)
    nnp, nni = oracle.select_pred_neighbors(lo, ce[:k], w["m"])
    sel = pi[:bp[k]]
    sub_ls, sub_yt = ls[sel], yt[sel]
    sub_bp, sub_pi = bp[:k + 1], np.arange(bp[k], dtype=np.int32)
    reps, t0 = 0, time.perf_counter()
    while True:
        mean, var, _ = oracle.predict(th, lo, yo, sub_ls, sub_bp, sub_pi, nnp, nni)
        oracle.cond_sim(mean, var, w["rounds"], reps, 1.959963984540054, sub_yt)
        reps += 1
        el = time.perf_counter() - t0
        if el >= seconds or reps >= 100:
            break
    return (reps * len(sel) / el, f"{reps} x (Algorithm 2 + {w['rounds']}-round conditional simulation) on the "
            f"first {k} prediction blocks ({len(sel)} new locations) of the same workload", oracle.num_threads())


def run_pred(args, w, log):
    ws, rank, local = _dist()
    if args.impl == "reference":
        if rank != 0:
            return 0
        import oracle
        oracle.build()
        # data from the oracle's own block-Vecchia draw on a 20,000-point copy at the same density
        n_s = min(w["n"], 20_000)
        wl = dict(w, n=n_s, pred_bc=max(1, w["pred_bc"] * n_s // w["n"]))
        locs, hold = pred_split(wl)
        th = oracle.theta(w["sigma2"], w["beta"], w["nu"], w["nugget"])
        bp, pi, ce = oracle.build_blocks(locs, n_s // 10, seed=w["seed"])
        nnp, nni = oracle.select_neighbors(locs, bp, pi, ce, 30)
        y = oracle.bv_draw(th, locs, bp, pi, nnp, nni, synth.normal(w["seed"], 20, n_s))
        vals = []
        for k in range(args.warmup + args.steps):
            v, sample, cores = pred_oracle_sample(wl, locs, y, hold, seconds=2.0)
            if k >= args.warmup:
                vals.append(v)
        val = statistics.mean(vals)
        line = {"impl": "reference", "metric": pred_metric(w), "value": val, "unit": "predictions/s",
                "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": (w["n"] // 10) / val * 1e3,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": pred_config(w, args),
                "cpu_baseline": {"value": val, "unit": "predictions/s", "cores": cores, "kind": "oracle",
                                 "sample": "each step: " + sample + " (data: oracle block-Vecchia draw at m=30, "
                                 f"n={n_s})"},
                "e2e": {"value": val, "unit": "predictions/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return 0
    import torch
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2410_04477_gb300 import bv
    stream = torch.cuda.Stream()
    t0 = time.perf_counter()
    locs, hold = pred_split(w)
    th = bv.theta(w["sigma2"], w["beta"], w["nu"], w["nugget"])
    with bv.Context(local, stream.cuda_stream) as gen:
        gen.set_data(locs)
        gen.build_blocks(w["bc"], seed=w["seed"])
        gen.select_neighbors(w["gen_m"])
        y = gen.simulate(th, synth.normal(w["seed"], 20, w["n"]))
    ctx = bv.Context(local, stream.cuda_stream)
    ctx.set_data(locs[~hold], y[~hold])
    ctx.set_pred_locations(locs[hold], y[hold])
    ctx.build_pred_blocks(w["pred_bc"], seed=w["seed"])
    ctx.select_pred_neighbors(w["m"])
    flops, cov_evals = ctx.pred_plan_info()
    n_star = int(hold.sum())
    log(f"setup {time.perf_counter() - t0:.1f}s: n_obs={int((~hold).sum())} n*={n_star}")
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    def step(k, timing):
        with torch.cuda.stream(stream):   # the flush finishes before the timed calls start
            flush.zero_()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record(stream)
        ctx.predict(th, want=())
        e[1].record(stream)
        _, _, cov = ctx.cond_sim(w["rounds"], seed=k, bounds=False)
        e[2].record(stream)
        if timing is not None:
            timing.append((e, cov))

    for k in range(args.warmup):
        step(k, None)
    barrier()
    clk = Clocks(local)
    rec = []
    for k in range(args.steps):
        step(args.warmup + k, rec)
    barrier()
    clocks = clk.stop()
    pred_ms = [a[0].elapsed_time(a[1]) for a, _ in rec]
    sim_ms = [a[1].elapsed_time(a[2]) for a, _ in rec]
    tot_ms = max_over_ranks(float(sum(pred_ms) + sum(sim_ms)))
    value = ws * args.steps * n_star / (tot_ms / 1e3)
    picp = [c / n_star for _, c in rec]
    # end to end through the public API with host buffers: observations up, means,
    # variances and interval bounds down
    y_pin = torch.from_numpy(np.ascontiguousarray(y[~hold])).pin_memory()
    barrier()
    t0 = time.perf_counter()
    for k in range(args.steps):
        ctx.set_observations(y_pin.numpy())
        ctx.predict(th)
        ctx.cond_sim(w["rounds"], seed=k)
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    e2e = {"value": ws * args.steps * n_star / e2e_s, "unit": "predictions/s",
           "h2d_bytes_per_step": int((~hold).sum()) * 8, "d2h_bytes_per_step": n_star * 8 * 4 + 16}
    mean_pred = statistics.mean(pred_ms) / 1e3
    achieved = flops / mean_pred / 1e12
    roof = {"bound": "alu", "kernel": "k_pred (one launch: covariance + partial augmented Cholesky of every "
            "prediction block)", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None,
            "peak_source": "nominal GB300 FP64 1.25 TFLOP/s (no FP64 entry in MEASURED_PEAKS.json; probe 1.19)",
            "flops_per_launch": flops, "cov_entries_per_launch": cov_evals}
    cpu = None
    if not args.no_cpu and rank == 0 and ws == 1:
        v, sample, cores = pred_oracle_sample(w, locs, y, hold)
        cpu = {"value": v, "unit": "predictions/s", "cores": cores, "kind": "oracle", "sample": sample}
    if rank == 0:
        line = {"metric": pred_metric(w), "value": value, "unit": "predictions/s", "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": pred_config(w, args), "roofline": roof, "cpu_baseline": cpu,
                "e2e": e2e, "clocks": clocks, "gpu_launches": 2 * args.steps,
                "extras": {"predict_ms": statistics.mean(pred_ms), "cond_sim_ms": statistics.mean(sim_ms),
                           "picp_mean": statistics.mean(picp), "picp_min": min(picp), "picp_max": max(picp)}}
        print(json.dumps(line), flush=True)
    ctx.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_kl(args, w, log):
    ws, rank, local = _dist()
    n = w["n"]
    if args.impl == "reference":
        if rank != 0:
            return 0
        import oracle
        oracle.build()
        # the oracle's dense Eq. 1 on a bounded sample (n_s points at the same density)
        n_s = min(3000, n)
        locs = synth.locs_uniform(n_s, 2, w["seed"]) * (n_s / n) ** 0.5
        th = oracle.theta(w["sigma2"], w["beta"], w["nu"], max(w["nugget"], 1e-10))
        zero = np.zeros(n_s)
        for _ in range(args.warmup):
            oracle.exact_loglik(th, locs, zero)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            oracle.exact_loglik(th, locs, zero)
        per = (time.perf_counter() - t0) / args.steps * (n / n_s) ** 3
        val = 1.0 / per
        line = {"impl": "reference", "metric": kl_metric(w), "value": val, "unit": "evals/s", "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": per * 1e3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": kl_config(w, args),
                "cpu_baseline": {"value": val, "unit": "evals/s", "cores": oracle.num_threads(), "kind": "oracle",
                                 "sample": f"each step: the oracle's dense Eq. 1 on n={n_s} points at the same "
                                 "density, extrapolated by (n / n_s)^3"},
                "e2e": {"value": val, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return 0
    import torch
    torch.cuda.set_device(local)
    from paper_2410_04477_gb300 import bv
    stream = torch.cuda.Stream()
    locs = synth.locs_uniform(n, w["d"], w["seed"])
    th = bv.theta(w["sigma2"], w["beta"], w["nu"], w["nugget"])
    ctx = bv.Context(local, stream.cuda_stream)
    ctx.set_data(locs, np.zeros(n))
    flops = bv.exact_flops(n)
    for _ in range(args.warmup):
        ctx.exact_loglik(th, use_y=False)
    torch.cuda.synchronize()
    clk = Clocks(local)
    ms = []
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ell0, _, logdet0 = ctx.exact_loglik(th, use_y=False)
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    clocks = clk.stop()
    tot_ms = max_over_ranks(float(sum(ms)))
    value = ws * args.steps / (tot_ms / 1e3)
    achieved = flops / (statistics.mean(ms) / 1e3) / 1e12
    roof = {"bound": "alu", "kernel": "k_update + k_trsm + k_potrf (tiled dense Cholesky, one exact evaluation)",
            "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
            "traffic": None, "flops_per_launch_sequence": flops,
            "peak_source": "nominal GB300 FP64 1.25 TFLOP/s (no FP64 entry in MEASURED_PEAKS.json; probe 1.19)"}
    # end to end: observations up, ell down, through the public call
    y = synth.normal(w["seed"], 20, n)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ctx.set_observations(y)
        ctx.exact_loglik(th)
    e2e_s = time.perf_counter() - t0
    e2e = {"value": args.steps / e2e_s, "unit": "evals/s", "h2d_bytes_per_step": n * 8, "d2h_bytes_per_step": 24}
    # the KL study itself
    study = {"exact_logdet": logdet0, "exact_ell0": ell0, "bv": [], "cv": []}

    def timed_eval(c):
        c.loglik(th)
        t = time.perf_counter()
        for _ in range(5):
            c.loglik(th)
        return (time.perf_counter() - t) / 5 * 1e3

    # KL = (log|Sigma_a| - log|Sigma_0|) / 2 (Eq. 7); the exact log-determinant is the one
    # of the timed steps, the approximate one comes from the block kernels
    ctx.set_observations(np.zeros(n))

    def kl_of(c):
        _, _, logdet_a = c.loglik_terms(th)
        return 0.5 * (logdet_a - logdet0)

    for order in w["orders"]:
        ctx.build_blocks(w["bc"], seed=w["seed"])
        ctx.order_blocks(order, seed=w["seed"])
        for m in w["bv_m"]:
            ctx.select_neighbors(m)
            kl = kl_of(ctx)
            study["bv"].append({"order": order, "bc": w["bc"], "m": m, "kl": kl, "eval_ms": timed_eval(ctx)})
            log(f"BV-{w['bc']}-{m}-{order}: KL {kl:.3e}")
    ctx.build_singletons(seed=w["seed"])
    for m in w["cv_m"]:
        ctx.select_neighbors(m)
        kl = kl_of(ctx)
        study["cv"].append({"order": "random", "m": m, "kl": kl, "eval_ms": timed_eval(ctx)})
        log(f"CV-{n}-{m}-random: KL {kl:.3e}")
    if rank == 0:
        line = {"metric": kl_metric(w), "value": value, "unit": "evals/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": kl_config(w, args), "roofline": roof, "cpu_baseline": None, "e2e": e2e,
                "clocks": clocks, "gpu_launches": int(3 * ((n + 64) // 64) + 2) * args.steps,
                "extras": {"kl_study": study}}
        if not args.no_cpu and ws == 1:
            import oracle
            n_s = min(3000, n)
            sub = locs[:n_s] * 1.0
            oth = oracle.theta(w["sigma2"], w["beta"], w["nu"], max(w["nugget"], 1e-10))
            t0 = time.perf_counter()
            oracle.exact_loglik(oth, sub, np.zeros(n_s))
            per = (time.perf_counter() - t0) * (n / n_s) ** 3
            line["cpu_baseline"] = {"value": 1.0 / per, "unit": "evals/s", "cores": oracle.num_threads(),
                                    "kind": "oracle", "sample": f"one dense Eq. 1 on {n_s} points, "
                                    "extrapolated by (n / n_s)^3"}
        print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def kl_metric(w):
    return (f"exact GP log-likelihood evals/sec (dense FP64 Cholesky, Eq. 1), n={w['n']}, nu={w['nu']}, "
            f"beta={w['beta']}; KL study of block vs classic Vecchia in extras")


def kl_config(w, args):
    return {"workload": args.workload, "n": w["n"], "d": w["d"], "nu": w["nu"], "beta": w["beta"],
            "sigma2": w["sigma2"], "nugget": w["nugget"], "bc": w["bc"], "bv_m": w["bv_m"], "cv_m": w["cv_m"],
            "orders": w["orders"], "l2": "inputs (3.2 GB factor) larger than L2"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c3", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--no-extras", action="store_true", help="skip the other-precision line")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    ap.add_argument("--n-scale", type=float, default=1.0,
                    help="scale n and bc (3D: the number of sites) by this factor, keeping the block and "
                         "conditioning sizes; for profiling a smaller case of the same kernel shapes")
    ap.add_argument("--no-mle", action="store_true",
                    help="skip the MLE wall-time extras (n=5e5 MLE, cold/warm x FP64/mixed) of the default run")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    w = dict(WORKLOADS[args.workload])
    if args.n_scale != 1.0 and "n" in w and "bc" in w:
        f = args.n_scale
        if "sites" in w:
            w["sites"] = max(1, int(round(w["sites"] * f)))
            w["n"] = w["sites"] * w["levels"]
        else:
            w["n"] = max(1, int(round(w["n"] * f)))
        w["bc"] = max(1, int(round(w["bc"] * f)))
        w["n_scale"] = f
    if w.get("kind") == "kl":
        log = (lambda s: print(s, file=sys.stderr, flush=True)) if _dist()[1] == 0 else (lambda s: None)
        return run_kl(args, w, log)
    if w.get("kind") == "pred":
        log = (lambda s: print(s, file=sys.stderr, flush=True)) if _dist()[1] == 0 else (lambda s: None)
        return run_pred(args, w, log)
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
    # plan, autotune and graph capture at the workload's own smoothness and scale (the
    # first evaluation tunes at its theta; the kernels' cost depends on the Matern form)
    ctx.loglik_multi(thetas[0], prec)
    info = ctx.plan_info(prec)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    nd = len(thetas[0])

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
    tot_ms = max_over_ranks(float(sum(ms)))
    mean_ms = tot_ms / args.steps
    value = whole_job_rate(args.steps, ws, tot_ms)

    # end to end through the public API with host buffers: y (pinned) up, ell down
    y_pin = torch.from_numpy(np.ascontiguousarray(y_true)).pin_memory()
    barrier()
    t0 = time.perf_counter()
    for k in range(args.steps):
        ctx.set_observations(y_pin.numpy())
        if nd == 1:
            ctx.loglik(thetas[(args.warmup + k) % len(thetas)][0], prec)
        else:
            ctx.loglik_multi(thetas[(args.warmup + k) % len(thetas)], prec)
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    e2e = {"value": ws * args.steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(w["n"] * 8 + 64 * nd),
           "d2h_bytes_per_step": 8 * nd}

    achieved = info["flops"] / (mean_ms / 1e3) / 1e12
    roof = {"bound": "alu", "kernel": "k_ll_fp64 (all size bins) + reduction, one evaluation",
            "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP64_PEAK_TFLOPS, "traffic": NCU_TRAFFIC.get((args.workload, args.precision)),
            "traffic_unit": "bytes per evaluation (ncu dram__bytes_read.sum + dram__bytes_write.sum)",
            "peak_source": "nominal GB300 FP64 1.25 TFLOP/s (no FP64 entry in MEASURED_PEAKS.json; probe 1.19)",
            "flops_per_eval": info["flops"], "cov_entries_per_eval": info["cov_entries"]}
    if prec == bv.BV_MIXED:
        roof.update(kernel="k_ll_mixed (all size bins) + reduction, one evaluation", peak=FP32_PEAK_TFLOPS,
                    frac=achieved / FP32_PEAK_TFLOPS,
                    peak_source="FP32 FMA: 152 SMs x 128 lanes x 2 x 2070 MHz (probe 69.5 at ~1.99 GHz)")

    extras = {}
    if not args.no_extras and rank == 0:
        base = [true_theta(bv, w)] if nd == 1 else [bv.theta(t[0], t[1], t[3], t[2]) for t in w["thetas"]]
        ll64 = ctx.loglik_multi(base, bv.BV_FP64)
        other = bv.BV_MIXED if prec == bv.BV_FP64 else bv.BV_FP64
        ctx.autotune(other)
        n2 = min(args.steps, 30) if other == bv.BV_MIXED or nd > 1 else min(args.steps, 5)
        ms2 = time_device(torch, bv, ctx, stream, thetas, other, 3, n2, flush)
        steps64, steps_ell = [], []
        if other == bv.BV_MIXED:
            # the check's FP64 share at each timed theta (untimed re-evaluations): the bound
            # is relative to |ell|, so a theta where ell is small needs more FP64 blocks
            for k in range(n2):
                steps_ell.append(float(np.sum(ctx.loglik_multi(thetas[(3 + k) % len(thetas)], bv.BV_MIXED))))
                steps64.append(int(ctx.mixed_check_info()[0]))
        llm = ctx.loglik_multi(base, bv.BV_MIXED)
        nb64, ntouched, est = ctx.mixed_check_info()
        rel = np.abs(llm - ll64) / np.abs(ll64)
        extras["other_precision"] = {
            "precision": "mixed" if other == bv.BV_MIXED else "fp64",
            "evals_per_s": len(ms2) / (sum(ms2) / 1e3),
            "achieved_tflops": info["flops"] / (statistics.mean(ms2) / 1e3) / 1e12,
            "ell_fp64_at_truth": float(ll64.sum()), "ell_mixed_at_truth": float(llm.sum()),
            "rel_err_mixed_vs_fp64": float(abs(llm.sum() - ll64.sum()) / abs(ll64.sum())),
            "max_rel_err_per_dataset": float(rel.max()), "abs_err": float(abs(llm.sum() - ll64.sum())),
            "abs_err_per_dataset_max": float(np.abs(llm - ll64).max()),
            "check": {"bound": 1e-6, "blocks_fp64": int(nb64), "blocks": int(ctx.sizes()[0]),
                      "datasets_with_blocks_recomputed": int(ntouched), "datasets": int(nd),
                      "est_rel_err_max": float(est.max())}}
        if steps64:
            extras["other_precision"]["check"]["timed_steps"] = {
                "blocks_fp64": steps64, "ell": steps_ell,
                "mean_fraction_fp64": float(np.mean(steps64)) / int(ctx.sizes()[0])}
        if other == bv.BV_MIXED:
            # the same without the check: FP32 throughout (bv_set_mixed_tolerance(0))
            ctx.set_mixed_tolerance(0.0)
            ms3 = time_device(torch, bv, ctx, stream, thetas, other, 3, n2, flush)
            llu = ctx.loglik_multi(base, bv.BV_MIXED)
            ctx.set_mixed_tolerance(1e-6)
            relu = np.abs(llu - ll64) / np.abs(ll64)
            extras["other_precision"]["unchecked_fp32"] = {
                "evals_per_s": len(ms3) / (sum(ms3) / 1e3),
                "achieved_tflops": info["flops"] / (statistics.mean(ms3) / 1e3) / 1e12,
                "rel_err_vs_fp64": float(abs(llu.sum() - ll64.sum()) / abs(ll64.sum())),
                "max_rel_err_per_dataset": float(relu.max()), "abs_err": float(abs(llu.sum() - ll64.sum()))}
        log(f"extras: {extras['other_precision']}")
        if args.workload == "c4_mle":
            extras["mle"] = run_mle(bv, ctx, w, log)
            if not args.no_cpu:
                try:
                    extras["mle"]["cpu_oracle"] = oracle_mle_estimate(w, extras["mle"])
                except Exception as exc:  # reported, never hides the main line
                    extras["mle"]["cpu_oracle"] = {"error": repr(exc)}
        elif not args.no_mle and ws == 1 and args.workload == "c3":
            # the metric's second half: MLE wall-time on the n = 5e5 workload, in its own context
            wm = dict(WORKLOADS["c4_mle"])
            try:
                with bv.Context(local, stream.cuda_stream) as mctx:
                    setup_gpu(bv, mctx, wm, log)
                    extras["mle"] = dict(workload="c4_mle: n=5e5 uniform 2D, bc=5e4, m=100, nu=1.5 fixed, "
                                         "true theta (1.5, 0.05, 5e-3), cold start (1, 0.1, 1e-2)",
                                         **run_mle(bv, mctx, wm, log))
            except Exception as exc:  # reported, never hides the main line
                extras["mle"] = {"error": repr(exc)}
            if not args.no_cpu and "error" not in extras["mle"]:
                try:
                    extras["mle"]["cpu_oracle"] = oracle_mle_estimate(wm, extras["mle"])
                except Exception as exc:  # reported, never hides the main line
                    extras["mle"]["cpu_oracle"] = {"error": repr(exc)}
    cpu = None
    if not args.no_cpu and rank == 0 and ws == 1:
        try:
            v, sample, cores, per, one = cpu_oracle_sample(w)
            cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                   "one_thread": one}
        except Exception as exc:  # reported, never hides the main line
            cpu = {"kind": "oracle", "error": repr(exc)}

    if rank == 0:
        line = {"metric": metric_of(w, args), "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
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

"""bench.py's reference arm (the FP64 CPU oracle on a bounded sample of the workload) runs
without a GPU: its one JSON line must carry the fields the benchmark contract names, with
the reference marked as such, the oracle's thread count stated and no host-device copies
claimed."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _reference_line(*extra):
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3", *extra], capture_output=True, text=True, cwd=ROOT, env=env, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    return json.loads(lines[0])


@pytest.mark.parametrize("workload,unit", [("c3", "evals/s"), ("c2_m60", "evals/s"), ("c5_m60", "evals/s"),
                                           ("pred_20k", "predictions/s")])
def test_reference_arm_json(workload, unit):
    d = _reference_line("--workload", workload)
    if workload == "c3":  # the default workload is the largest single-GPU configuration
        assert _reference_line()["config"] == d["config"]
    assert d["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["unit"] == unit and d["value"] > 0 and d["ms_per_step"] > 0
    assert d["steps"] == 1 and d["warmup"] >= 3 and d["n_gpus"] == 1
    assert d["higher_is_better"] is True and d["data"] == "synthetic"
    assert d["config"]["workload"] == workload
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == unit
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_cpu_baseline_reports_all_cores_and_one_thread():
    # the CPU-baseline leg of the GPU line: the oracle on every host core and on one
    # thread, the thread count restored afterwards
    import sys
    sys.path.insert(0, ROOT)
    import bench
    import oracle
    oracle.build()
    before = oracle.num_threads()
    v, sample, cores, per, one = bench.cpu_oracle_sample(dict(bench.WORKLOADS["c2_m60"]), seconds=0.0,
                                                         one_thread_seconds=0.0001)
    assert oracle.num_threads() == before == cores
    assert v > 0 and per > 0 and sample.startswith("1 evals of ")
    assert one["cores"] == 1 and one["value"] > 0 and one["unit"] == "evals/s"
    assert one["sample"].startswith("1 evals of ")
    assert bench.cpu_oracle_sample(dict(bench.WORKLOADS["c2_m60"]), seconds=0.0, one_thread_seconds=0)[4] is None


def test_oracle_mle_estimate_scales_the_gpu_call_counts():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    import oracle
    oracle.build()
    res = {"fp64_cold": {"evals": 37}, "fp64_warm": {"evals": 19}, "mixed_cold": {"evals": 55}}
    est = bench.oracle_mle_estimate(dict(bench.WORKLOADS["c4_mle"]), res, seconds=0.0)
    assert est["kind"] == "oracle, extrapolated" and est["cores"] == oracle.num_threads()
    assert est["fp64_cold_wall_s"] == 37 / est["evals_per_s"]
    assert est["fp64_warm_wall_s"] == 19 / est["evals_per_s"]
    assert "mixed_cold_wall_s" not in est

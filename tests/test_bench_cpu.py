"""bench.py's reference arm (the FP64 oracle on the host cores) runs on any
host: one JSON line with the benchmark contract's keys, and silence from
ranks other than 0."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(extra_env=None):
    env = dict(os.environ, **(extra_env or {}))
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                           "--workload", "lf5x5_64_x2", "--steps", "2", "--warmup", "3"],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_reference_arm_prints_one_contract_line():
    r = _run()
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 3
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["config"]["workload"] == "lf5x5_64_x2"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_are_silent():
    r = _run({"RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""


def test_throttled_clock_records_are_rejected():
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    ok = {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": []}
    assert not bench.clocks_rejected(ok)
    for r in ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"):
        assert bench.clocks_rejected(dict(ok, reasons=[r]))
    # a power cap is kept; clocks far below their maximum with no reason are a lock
    assert not bench.clocks_rejected(dict(ok, sm_mhz=1700.0, reasons=["sw_power_cap"]))
    assert bench.clocks_rejected(dict(ok, sm_mhz=1200.0))


def test_algorithmic_counts_of_the_rooflines():
    """The benchmark's roofline numerators for the 9 x 9-view, 512^2 light field,
    against the counts written out: streaming bytes per iteration
    B_alg = 4 (3 s_k q + 2 s_d p + 3 p) + 4 K 11 p, and 37 FLOP per view and
    HR pixel for one sum_k A_k^T A_k p at scale 2 with a 7-tap blur."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    from paper_2206_05047_gb300 import synth
    wl = synth.WORKLOADS["lf9x9_256_x2"]
    s_k, q, p, s_d, K = 81, 256 * 256, 512 * 512, 48, 5
    assert (wl.s_k, wl.H * wl.W, wl.HR[0] * wl.HR[1], wl.s_d, wl.cg_iters) == (s_k, q, p, s_d, K)
    assert bench.alg_bytes_per_iter(wl) == 4 * (3 * s_k * q + 2 * s_d * p + 3 * p) + 4 * K * 11 * p
    assert bench.alg_bytes_per_iter(wl) == 225_181_696
    # gather 8 + scatter 8 + blur 4 kb (1/2 + 1/4) = 16 + 21 = 37 FLOP per view and pixel
    assert bench.normal_flops_per_launch(wl) == s_k * p * 37 == 785_645_568

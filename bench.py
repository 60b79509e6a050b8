#!/usr/bin/env python
"""Benchmark of the light-field super-resolution ADMM hot path.

One step = one full solve of one synthetic light field: x := x0, duals := 0,
then N ADMM iterations (Algorithm 1), each with weights rebuilt from x and a
K = 5 step CG x-step (Algorithm 2).  The metric is HR light-field
throughput, s_k * Hh * Wh * N / t, in Mpix * ADMM-iter / s.

  value   inputs resident in HBM, device time (CUDA events on the solver's
          stream) of K steps, L2 flushed (256 MB write) between steps
  e2e     the same metric through lfsr_solve with pinned HOST buffers: the
          views and x0 go host -> device and x comes back inside the timing
  roofline  the dominant kernel (x-step normal-matrix operator) timed with
          CUDA events in the library's profiling mode, against the FP32 ALU
          peak (its bound); plus the whole path's HBM fraction
  cpu_baseline  the FP64 oracle on the host cores, on a bounded sample
  batched / served  bounded records on the first 16 light fields of the
          batched configuration: the batch (both launch forms) against serial
          plain solves, and Poisson arrivals (20 per second for 3 s) served by
          the continuous-batching server against one plain solve at a time

python bench.py [--gpus N --steps K --warmup W] [--impl reference]
Under torchrun (N > 1) every rank solves its own light field (replicas, weak
scaling); times are the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2206_05047_gb300 import synth  # noqa: E402

METRIC = "HR LF Mpix*ADMM-iter/s"
BATCH_WORKLOAD = "batch_uneven"
SERVE_WORKLOAD = "serve_poisson"
UNIT = "Mpix*iter/s"
FP32_LANES_PER_SM = 128
# the arithmetic type of the path with the storage kind of its large streams
DTYPE = {"fp32": "f32", "fp16": "f32 (f16 storage)", "bf16": "f32 (bf16 storage)",
         "fp16-views32": "f32 (f16 storage, f32 views)",
         "bf16-views32": "f32 (bf16 storage, f32 views)"}


def sm_count(dev=None) -> int:
    """Streaming multiprocessors of the device (the FP32 peak's SM factor)."""
    import torch
    return int(torch.cuda.get_device_properties(dev if dev is not None else 0)
               .multi_processor_count)


def args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="lf9x9_256_x2",
                    choices=sorted(synth.WORKLOADS) + [BATCH_WORKLOAD, SERVE_WORKLOAD])
    ap.add_argument("--batch", type=int, default=64, help="light fields of the batch workload")
    ap.add_argument("--serve-seconds", type=float, default=60.0,
                    help="arrival window of the serving workload (Poisson, 20 requests/s)")
    ap.add_argument("--serve-rate", type=float, default=20.0)
    ap.add_argument("--serve-slots", type=int, default=64)
    ap.add_argument("--serve-no-plain", action="store_true",
                    help="skip the serial plain-path comparison of the serving workload")
    ap.add_argument("--iterations", type=int, default=None, help="ADMM iterations per step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batch-record", action="store_true",
                    help="skip the bounded batched-vs-plain and served-vs-plain records of the "
                         "default line")
    ap.add_argument("--precision", default="fp32",
                    choices=["fp32", "fp16", "bf16", "fp16-views32", "bf16-views32"],
                    help="storage type of views, duals and NLTV weights (arithmetic is f32); "
                         "-views32 keeps the views in f32")
    ap.add_argument("--weights", default="patch", choices=["patch", "paper"],
                    help="regulariser weights of the named workloads: the patch distance "
                         "exp(-pd/h^2), or the paper's spatial * edge * occlusion weights "
                         "(Sec. 3.4) at synth.PAPER_SIGMAS")
    return ap.parse_args()


def workload_config(wl, n_iter, extra=None):
    cfg = {"workload": wl.name, "views": f"{wl.U}x{wl.V}", "lr": f"{wl.H}x{wl.W}",
           "hr": f"{wl.HR[0]}x{wl.HR[1]}", "scale": wl.scale, "blur": f"{wl.kb}x{wl.kb} "
           f"gaussian sigma {wl.blur_sigma}", "nltv_window": wl.window, "nltv_patch": wl.patch,
           "nltv_h": wl.h, "admm_iters_per_step": n_iter, "cg_iters": wl.cg_iters,
           "lambda1": wl.lambda1, "lambda2": wl.lambda2, "mu": wl.mu,
           "noise": f"gaussian {wl.noise_sigma} + {int(100 * wl.impulse)}% salt-and-pepper"}
    if extra:
        cfg.update(extra)
    return cfg


def alg_bytes_per_iter(wl, esize=4, esize_y=4) -> float:
    """Streaming bytes of one ADMM iteration: duals read+write (esize bytes
    each: 4, or 2 with 16-bit storage), views read (esize_y), x / omega / v,
    and 11 HR-vector passes per CG step (float32)."""
    p = wl.HR[0] * wl.HR[1]
    q = wl.H * wl.W
    return (esize * (2 * wl.s_k * q + 2 * wl.s_d * p) + esize_y * wl.s_k * q + 4.0 * 3 * p
            + 4.0 * wl.cg_iters * 11 * p)


def normal_flops_per_launch(wl) -> float:
    """Algorithmic FLOPs of one sum_k A_k^T A_k p: per view and HR pixel,
    8 (bilinear gather) + 8 (bilinear scatter) + separable blur at the
    decimated positions and its adjoint on the non-zeros,
    4 kb (1/zeta + 1/zeta^2)."""
    p = wl.HR[0] * wl.HR[1]
    z = wl.scale
    return wl.s_k * p * (16.0 + 4.0 * wl.kb * (1.0 / z + 1.0 / z ** 2))


def max_over_ranks(value: float) -> float:
    """Max of a per-rank scalar over the process group (the identity when no
    group is initialised).  Uses a CUDA tensor under NCCL, a CPU one else."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" \
        else torch.device("cpu")
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_seed(rank: int) -> int:
    """Each rank solves its own light field (replicas, weak scaling)."""
    return 1000 * 2 + rank


# --------------------------------------------------------------------------
# clocks
# --------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None

        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        smax = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons,
                "samples": len(rows)}


def clocks_rejected(clk) -> bool:
    """A timed region whose clock record shows a hardware or thermal slowdown,
    or SM clocks well below their maximum with no reason given (a clock
    lock left by someone else), is not a valid measurement."""
    bad = {"hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"}
    if bad & set(clk.get("reasons") or []):
        return True
    sm, smax = clk.get("sm_mhz"), clk.get("sm_max_mhz")
    return bool(sm and smax and sm < 0.85 * smax and not clk.get("reasons"))


def any_rank(flag: bool) -> bool:
    """True on every rank if it is true on one (max over ranks)."""
    return max_over_ranks(1.0 if flag else 0.0) > 0.5


# --------------------------------------------------------------------------
# CPU baseline: the FP64 oracle, as it stands, on the host cores
# --------------------------------------------------------------------------
def weight_kwargs(weights: str) -> dict:
    """Solver / oracle keyword arguments of a weight scheme."""
    return {} if weights == "patch" else dict(weights="paper", **synth.PAPER_SIGMAS)


def oracle_rate(prob, iters: int, weights: str = "patch"):
    from oracle import oracle as om
    o = om.Oracle.from_problem(prob, **weight_kwargs(weights))
    t = time.perf_counter()
    o.admm(prob.y, prob.x0, iters)
    dt = time.perf_counter() - t
    wl = prob.wl
    return wl.s_k * wl.HR[0] * wl.HR[1] * iters / dt / 1e6, dt, om.num_threads()


def kernel_source_digest() -> str:
    """Digest of the operator-kernel sources (the kernel the roofline names)."""
    h = hashlib.sha256()
    for f in ("op_kernels.cu", "op_fast.cu", "op_fast.cuh", "lfsr_internal.cuh",
              "lfsr_device.cuh"):
        with open(os.path.join(ROOT, "paper_2206_05047_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_from_profile(wl):
    """DRAM bytes per normal-operator launch from the committed ncu summary,
    if it was taken on the current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", "normal_apply_traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
        if rec.get("source_sha256_16") != kernel_source_digest() or rec.get("workload") != wl.name:
            return None
        return float(rec["dram_bytes_per_launch"])
    except (OSError, KeyError, ValueError):
        return None


# --------------------------------------------------------------------------
def run_reference(a, wl, n_iter):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    prob = synth.make_problem(wl, seed=1000 * 2)
    from oracle import oracle as om
    o = om.Oracle.from_problem(prob, **weight_kwargs(getattr(a, "weights", "patch")))
    # bounded sample per step: one ADMM iteration of the full workload
    x, wA, wS = prob.x0, None, None
    for _ in range(a.warmup):
        x, wA, wS = o.admm(prob.y, x, 1, wA=wA, wS=wS)
    t = time.perf_counter()
    for _ in range(a.steps):
        x, wA, wS = o.admm(prob.y, x, 1, wA=wA, wS=wS)
    dt = time.perf_counter() - t
    value = wl.s_k * wl.HR[0] * wl.HR[1] * a.steps / dt / 1e6
    sample = f"1 ADMM iteration (K = {wl.cg_iters} CG steps) of {wl.name} per step"
    line = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference",
            "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": 1e3 * dt / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(wl, 1, {"parallelism": "none (host cores)"}),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": om.num_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------
# batched uneven light fields: one launch per phase for all of them, against
# the same light fields solved one after another by the plain path
# --------------------------------------------------------------------------
def _make_problem_args(wl_seed):
    wl, seed = wl_seed
    pr = synth.make_problem(wl, seed=seed)
    return (pr.y.astype(np.float32), pr.x0.astype(np.float32), pr.blur.astype(np.float32),
            pr.disparity.astype(np.float32), pr.gt)


def batch_problems(n: int, seed: int = 4000):
    """The batched configuration's light fields, generated in a process pool
    (spawned: no CUDA state is forked)."""
    import multiprocessing as mp
    wls = synth.batch_workloads(n, seed)
    jobs = [(w, seed + 1 + i) for i, w in enumerate(wls)]
    procs = min(len(jobs), os.cpu_count() or 1, 16)
    with mp.get_context("spawn").Pool(procs) as pool:
        out = pool.map(_make_problem_args, jobs, chunksize=1)
    return wls, out


def run_batch(a):
    import torch
    from paper_2206_05047_gb300 import lfsr
    if int(os.environ.get("WORLD_SIZE", "1")) > 1:
        raise SystemExit("the batch workload runs on one GPU")
    t_gen = time.perf_counter()
    wls, probs = batch_problems(a.batch)
    t_gen = time.perf_counter() - t_gen
    n_iter = a.iterations if a.iterations is not None else wls[0].iterations
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    kws = []
    for wl, (y, x0, blur, disp, gt) in zip(wls, probs):
        kws.append(dict(U=wl.U, V=wl.V, H=wl.H, W=wl.W, scale=wl.scale, blur=blur,
                        disparity=disp, lambda1=wl.lambda1, lambda2=wl.lambda2, mu=wl.mu,
                        nltv_window=wl.window, nltv_patch=wl.patch, nltv_h=wl.h,
                        cg_iters=wl.cg_iters, cg_tol=0.0, precision=a.precision))
    y_d = [torch.from_numpy(p[0]).to(dev) for p in probs]
    x0_d = [torch.from_numpy(p[1]).to(dev) for p in probs]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    work = sum(w.s_k * w.HR[0] * w.HR[1] for w in wls) * n_iter     # HR LF pixel-iterations

    def timed(step, steps):
        torch.cuda.synchronize(dev)
        total = 0.0
        for _ in range(steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            e1.synchronize()
            total += e0.elapsed_time(e1)
        return total

    # the batch: one launch per phase (per operator group) for all light fields
    batch = lfsr.Batch(kws, stream=stream)

    def batch_step():
        for j in range(len(wls)):
            batch.load(j, y_d[j], x0_d[j])
        batch.iterate(n_iter)

    # the project's autotuner: operator tile side per group, NLTV stencil
    # blocking, timed on these light fields (it iterates them; reloaded below)
    for j in range(len(wls)):
        batch.load(j, y_d[j], x0_d[j])
    t_tune = time.perf_counter()
    tuning = batch.autotune()
    t_tune = time.perf_counter() - t_tune
    for _ in range(a.warmup):
        batch_step()
    for attempt in range(2):        # one re-measurement if the clocks were throttled
        clocks = ClockSampler(0)
        clocks.start()
        time.sleep(0.25)
        t_batch = timed(batch_step, a.steps)
        clk = clocks.stop()
        clk["remeasured"] = attempt > 0
        if not clocks_rejected(clk):
            break
    value = work * a.steps / (t_batch / 1e3) / 1e6
    xb = []
    for j, wl in enumerate(wls):
        x = torch.empty(wl.HR, dtype=torch.float32, device=dev)
        batch.get_x(j, x)
        xb.append(x.cpu().numpy().astype(np.float64))

    # e2e: pinned host views and x0 in, x out, inside the timing
    e2e = None
    if not a.no_e2e:
        y_h = [torch.from_numpy(p[0]).pin_memory() for p in probs]
        x0_h = [torch.from_numpy(p[1]).pin_memory() for p in probs]
        x_h = [torch.empty(w.HR, dtype=torch.float32).pin_memory() for w in wls]

        def e2e_step():
            for j in range(len(wls)):
                batch.load(j, y_h[j], x0_h[j])
            batch.iterate(n_iter)
            for j in range(len(wls)):
                batch.get_x(j, x_h[j])
        t_e2e = timed(e2e_step, a.steps)
        e2e = {"value": work * a.steps / (t_e2e / 1e3) / 1e6, "unit": UNIT,
               "h2d_bytes_per_step": int(sum(t.numel() * 4 for t in y_h + x0_h)),
               "d2h_bytes_per_step": int(sum(t.numel() * 4 for t in x_h))}

    # per-kernel times of one batched iteration (profiling mode)
    batch.set_profiling(True)
    batch_step()
    ms, nl = batch.kernel_times()
    batch.set_profiling(False)
    names = ["nltv_block", "data_block", "cg_init", "nltv_apply", "normal_apply", "cg_update"]
    per_class = {names[i]: {"ms": ms[i], "launches": nl[i]} for i in range(6)}
    flops = sum(normal_flops_per_launch(w) for w in wls)         # one CG step, all light fields
    normal_ms_per_step = per_class["normal_apply"]["ms"] / max(n_iter * wls[0].cg_iters, 1)
    sm_clk = (clk.get("sm_max_mhz") or 2070.0)
    n_sm = sm_count()
    peak_tflops = n_sm * FP32_LANES_PER_SM * 2 * sm_clk * 1e6 / 1e12
    achieved = flops / (normal_ms_per_step / 1e3) / 1e12
    launches = batch.launches_per_iteration()
    roofline = {"bound": "alu",
                "kernel": "k_operator_fast<OP_NORMAL> (table: all light fields of a group)",
                "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                "frac": achieved / peak_tflops, "traffic": None,
                "normal_ms_per_cg_step": normal_ms_per_step, "flops_per_cg_step": flops,
                "peak_note": f"FP32 FMA: {n_sm} SMs x {FP32_LANES_PER_SM} lanes x 2 x "
                             f"{sm_clk:.0f} MHz",
                "per_kernel_ms_per_step": {k: v["ms"] for k, v in per_class.items()}}
    batch.close()

    # the plain path: the same light fields solved one after another
    solvers = [lfsr.Solver(stream=stream, **kw) for kw in kws]

    def plain_step():
        for j, sv in enumerate(solvers):
            lfsr.load(sv.handle, y_d[j], x0_d[j])
            lfsr.iterate(sv.handle, n_iter)

    def plain_x():
        out = []
        for sv, wl in zip(solvers, wls):
            x = torch.empty(wl.HR, dtype=torch.float32, device=dev)
            lfsr.get_x(sv.handle, x)
            out.append(x.cpu().numpy().astype(np.float64))
        return out

    for _ in range(a.warmup - 1):
        plain_step()
    xp0 = plain_x() if a.warmup >= 1 else None
    if a.warmup >= 1:
        plain_step()
    t_plain = timed(plain_step, a.steps)
    launches_plain = sum(int(lfsr.stats(sv.handle)["launches"]) for sv in solvers) // n_iter
    value_plain = work * a.steps / (t_plain / 1e3) / 1e6
    xp = plain_x()
    gts = [p[4] for p in probs]
    dpsnr = [synth.psnr(xb[j], gts[j]) - synth.psnr(xp[j], gts[j]) for j in range(len(wls))]
    # two runs of the plain path differ as much: float atomics reorder sums and
    # the reweighted iteration at this h amplifies the difference
    dpsnr_plain = ([synth.psnr(xp0[j], gts[j]) - synth.psnr(xp[j], gts[j])
                    for j in range(len(wls))] if xp0 is not None else [float("nan")])
    assert all(np.isfinite(x).all() for x in xb)
    for sv in solvers:
        sv.close()

    cpu = None
    if not a.no_cpu_baseline:
        small = min(range(len(wls)), key=lambda j: wls[j].s_k * wls[j].HR[0] * wls[j].HR[1])
        y, x0, blur, disp, gt = probs[small]
        prob = synth.Problem(wls[small], 0, blur.astype(np.float64), disp.astype(np.float64),
                             y.astype(np.float64), x0.astype(np.float64), gt, None)
        rate, dt, cores = oracle_rate(prob, 3)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"3 ADMM iterations of the smallest light field of the batch "
                         f"({wls[small].name}), {dt:.1f} s"}
    groups = sorted({(w.scale, w.kb) for w in wls})
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": t_batch / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[a.precision],
            "data": "synthetic (seeded textured-plane light fields)",
            "config": {"workload": BATCH_WORKLOAD, "light_fields": len(wls),
                       "iterations": n_iter, "cg_iters": wls[0].cg_iters,
                       "views": sorted({f"{w.U}x{w.V}" for w in wls}),
                       "lr_side": [min(w.H for w in wls), max(w.H for w in wls)],
                       "scales": sorted({w.scale for w in wls}),
                       "operator_groups": [f"x{z} blur {k}x{k}" for z, k in groups],
                       "hr_lf_mpix_per_iteration": work / n_iter / 1e6, "seed": 4000,
                       "storage": a.precision, "parallelism": "single GPU",
                       "autotuned": dict(tuning, seconds=round(t_tune, 2)),
                       "l2": "flushed between steps (256 MB write); working set >> L2",
                       "generation_s": round(t_gen, 1)},
            "plain_serial": {"value": value_plain, "unit": UNIT,
                             "ms_per_step": t_plain / a.steps,
                             "launches_per_iteration": launches_plain},
            "batch_vs_plain": value / value_plain,
            "equal_psnr": {"batch_vs_plain": {"max_abs_db": max(abs(d) for d in dpsnr),
                                              "mean_db": float(np.mean(dpsnr)),
                                              "mean_psnr_batch_db": float(np.mean(
                                                  [synth.psnr(xb[j], gts[j])
                                                   for j in range(len(wls))]))},
                           "plain_vs_plain": {"max_abs_db": max(abs(d) for d in dpsnr_plain),
                                              "mean_db": float(np.mean(dpsnr_plain))}},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": int(a.steps * n_iter * launches),
            "launches_per_iteration": launches, "clocks": clk}
    print(json.dumps(line), flush=True)


def batch_subrecord(dev, stream, n_lf: int = 16, n_iter: int = 10, steps: int = 3,
                    warmup: int = 1):
    """Bounded batched-vs-plain record for the default line: the first n_lf
    light fields of the batched configuration (seed 4000), n_iter ADMM
    iterations per step, one autotuned batch (one launch per phase and
    operator group, graph-replayed) against the same light fields solved
    one after another by the plain path, in float32 and in 16-bit (fp16)
    storage, with the PSNR of every light field compared between the two.
    Returns the record and the light fields (descriptions, arrays)."""
    import torch
    from paper_2206_05047_gb300 import lfsr
    t_gen = time.perf_counter()
    wls, probs = batch_problems(n_lf)
    t_gen = time.perf_counter() - t_gen
    y_d = [torch.from_numpy(p[0]).to(dev) for p in probs]
    x0_d = [torch.from_numpy(p[1]).to(dev) for p in probs]
    gts = [p[4] for p in probs]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    work = sum(w.s_k * w.HR[0] * w.HR[1] for w in wls) * n_iter

    def timed(step):
        for _ in range(warmup):
            step()
        torch.cuda.synchronize(dev)
        total = 0.0
        for _ in range(steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            e1.synchronize()
            total += e0.elapsed_time(e1)
        return total

    def xs_of(get, hrs):
        out = []
        for j, hr in enumerate(hrs):
            x = torch.empty(hr, dtype=torch.float32, device=dev)
            get(j, x)
            out.append(x.cpu().numpy().astype(np.float64))
        return out

    rec = {"workload": f"first {n_lf} light fields of {BATCH_WORKLOAD} (seed 4000)",
           "iterations": n_iter, "steps": steps,
           "hr_lf_mpix_per_iteration": work / n_iter / 1e6,
           "generation_s": round(t_gen, 1)}
    for prec in ("fp32", "fp16"):
        kws = [dict(U=w.U, V=w.V, H=w.H, W=w.W, scale=w.scale, blur=p[2], disparity=p[3],
                    lambda1=w.lambda1, lambda2=w.lambda2, mu=w.mu, nltv_window=w.window,
                    nltv_patch=w.patch, nltv_h=w.h, cg_iters=w.cg_iters, cg_tol=0.0,
                    precision=prec) for w, p in zip(wls, probs)]
        batch = lfsr.Batch(kws, stream=stream)
        for j in range(len(wls)):
            batch.load(j, y_d[j], x0_d[j])
        tuning = batch.autotune()

        def batch_step():
            for j in range(len(wls)):
                batch.load(j, y_d[j], x0_d[j])
            batch.iterate(n_iter)
        t_b = timed(batch_step)
        xb = xs_of(batch.get_x, [w.HR for w in wls])
        launches_b = batch.launches_per_iteration()
        # both launch forms (per-phase launches, one persistent launch per
        # iteration) at the tuned tiles, where the persistent one is available
        forms = {}
        if batch.persistent_available():
            tuned_form = batch.form()
            for form in ("phases", "persistent"):
                batch.set_form(form)
                forms[form] = timed(batch_step) / (steps * n_iter)
            batch.set_form(tuned_form)
        batch.close()
        solvers = [lfsr.Solver(stream=stream, **kw) for kw in kws]

        def plain_step():
            for j, sv in enumerate(solvers):
                lfsr.load(sv.handle, y_d[j], x0_d[j])
                lfsr.iterate(sv.handle, n_iter)
        t_p = timed(plain_step)
        launches_p = sum(int(lfsr.stats(sv.handle)["launches"]) for sv in solvers) // n_iter
        xp = xs_of(lambda j, x: lfsr.get_x(solvers[j].handle, x), [w.HR for w in wls])
        for sv in solvers:
            sv.close()
        dps = [synth.psnr(xb[j], gts[j]) - synth.psnr(xp[j], gts[j]) for j in range(len(wls))]
        vb = work * steps / (t_b / 1e3) / 1e6
        vp = work * steps / (t_p / 1e3) / 1e6
        rec[prec] = {"batch": vb, "plain_serial": vp, "batch_vs_plain": vb / vp,
                     "unit": UNIT, "launches_per_iteration": {
                         "batch": launches_b, "plain_serial": launches_p},
                     "forms_ms_per_iteration": forms or None,
                     "max_abs_dpsnr_db": max(abs(d) for d in dps),
                     "mean_psnr_db": float(np.mean([synth.psnr(xb[j], gts[j])
                                                    for j in range(len(wls))])),
                     "autotuned": tuning}
    del flush
    return rec, (wls, probs)


# --------------------------------------------------------------------------
# serving: Poisson arrivals, continuous batching under a memory budget,
# against the same arrivals served one at a time by the plain path
# --------------------------------------------------------------------------
def serve_compare(wls, probs, kws, rate, seconds, slots, n_iter, seed, stream, plain=True):
    """Poisson arrivals (rate per second over `seconds`, seeded) drawn from
    the pool (wls, probs, kws): served by one continuous-batching server
    (slots, 120 GB budget, 4 iterations per scheduling round), then the same
    arrivals served first come first served by one plain solve at a time.
    Wall-clock times on the host, inputs and results in host memory."""
    from paper_2206_05047_gb300 import lfsr
    rng = np.random.default_rng(seed)
    arrivals, t = [], 0.0
    while True:
        t += rng.exponential(1.0 / rate)
        if t > seconds:
            break
        arrivals.append(t)
    picks = rng.integers(0, len(wls), len(arrivals))
    work = [wls[k].s_k * wls[k].HR[0] * wls[k].HR[1] * n_iter for k in picks]
    budget = 120 * 10**9

    def pctl(v, q):
        return float(np.percentile(np.asarray(v), q))

    # warm-up: one small request through the server (kernels, allocator)
    small = min(range(len(wls)), key=lambda k: wls[k].H * wls[k].W * wls[k].s_k)
    warm = lfsr.Server(budget, max_active=slots, iterations=2, iterations_per_step=2,
                       stream=stream)
    warm.submit(probs[small][0], probs[small][1], **kws[small])
    while warm.stats()["done"] < 1:
        warm.step()
    warm.close()

    srv = lfsr.Server(budget, max_active=slots, iterations=n_iter, iterations_per_step=4,
                      stream=stream)
    ids, done_t, pending = {}, {}, set()
    nxt = 0
    t0 = time.perf_counter()
    while len(done_t) < len(arrivals):
        now = time.perf_counter() - t0
        while nxt < len(arrivals) and arrivals[nxt] <= now:
            k = picks[nxt]
            ids[nxt] = srv.submit(probs[k][0], probs[k][1], **kws[k])
            pending.add(nxt)
            nxt += 1
        active = srv.step()
        tnow = time.perf_counter() - t0
        for r in list(pending):
            state, _, rc = srv.status(ids[r])
            if state == lfsr.LFSR_REQ_DONE:
                done_t[r] = tnow
                pending.discard(r)
            elif state == lfsr.LFSR_REQ_FAILED:
                raise SystemExit(f"request {r} failed: {rc}")
        if active == 0 and not pending and nxt < len(arrivals):
            time.sleep(max(0.0, arrivals[nxt] - (time.perf_counter() - t0)))
    t_end = max(done_t.values())
    st = srv.stats()
    lat = [done_t[r] - arrivals[r] for r in range(len(arrivals))]
    xs = {}
    for r in range(len(arrivals)):
        x = np.zeros(wls[picks[r]].HR, np.float32)
        srv.fetch(ids[r], x)
        xs[r] = x
    srv.close()
    value = sum(work) / (t_end - arrivals[0]) / 1e6

    # the same arrivals, first come first served, one plain solve at a time
    picks_plain = picks if plain else []
    solvers = {}
    for k in sorted(set(np.asarray(picks_plain).tolist())):
        solvers[k] = lfsr.Solver(stream=stream, **kws[k])
    out = {k: np.zeros(wls[k].HR, np.float32) for k in solvers}
    for k in solvers:                                  # warm-up
        lfsr.solve(solvers[k].handle, probs[k][0], 2, probs[k][1], out[k])
    done_p, dpsnr = {}, []
    t0 = time.perf_counter()
    for r in range(len(picks_plain)):
        now = time.perf_counter() - t0
        if arrivals[r] > now:
            time.sleep(arrivals[r] - now)
        k = picks[r]
        lfsr.solve(solvers[k].handle, probs[k][0], n_iter, probs[k][1], out[k])
        done_p[r] = time.perf_counter() - t0
        gt = probs[k][4]
        dpsnr.append(synth.psnr(xs[r], gt) - synth.psnr(out[k], gt))
    for sv in solvers.values():
        sv.close()
    rec = {"value": value, "unit": UNIT, "requests": len(arrivals),
           "arrivals_per_s": rate, "arrival_window_s": seconds,
           "ms_first_arrival_to_last_result": 1e3 * (t_end - arrivals[0]),
           "latency_s": {"p50": pctl(lat, 50), "p99": pctl(lat, 99), "mean": float(np.mean(lat)),
                         "max": float(np.max(lat))},
           "plain_serial": None, "served_vs_plain": None, "equal_psnr": None,
           "peak_state_gb": st["bytes_peak"] / 1e9, "batch_rebuilds": st["batch_rebuilds"],
           "gpu_launches": int(st["launches"]),
           "h2d_bytes": int(sum(probs[k][0].nbytes + probs[k][1].nbytes for k in picks)),
           "d2h_bytes": int(sum(xs[r].nbytes for r in xs))}
    if done_p:
        t_end_p = max(done_p.values())
        lat_p = [done_p[r] - arrivals[r] for r in range(len(arrivals))]
        value_p = sum(work) / (t_end_p - arrivals[0]) / 1e6
        rec["plain_serial"] = {"value": value_p, "unit": UNIT,
                               "latency_s": {"p50": pctl(lat_p, 50), "p99": pctl(lat_p, 99),
                                             "mean": float(np.mean(lat_p))}}
        rec["served_vs_plain"] = value / value_p
        rec["equal_psnr"] = {"max_abs_db": float(np.max(np.abs(dpsnr))),
                             "mean_db": float(np.mean(dpsnr))}
    return rec


def serve_subrecord(stream, wls, probs, rate: float = 20.0, seconds: float = 3.0,
                    n_iter: int = 100, slots: int = 16):
    """Bounded served-vs-plain record for the default line: Poisson arrivals
    at `rate` per second for `seconds`, drawn from the light fields of the
    batched record (the first 16 of the batched configuration), each solved
    to its N = 100 iterations by the continuous-batching server (`slots`
    requests active at most: fewer slots finish the early requests sooner,
    more slots batch more) and, separately, by one plain solve at a time."""
    kws = [dict(U=w.U, V=w.V, H=w.H, W=w.W, scale=w.scale, blur=p[2], disparity=p[3],
                lambda1=w.lambda1, lambda2=w.lambda2, mu=w.mu, nltv_window=w.window,
                nltv_patch=w.patch, nltv_h=w.h, cg_iters=w.cg_iters, cg_tol=0.0,
                precision="fp32") for w, p in zip(wls, probs)]
    rec = serve_compare(wls, probs, kws, rate, seconds, slots, n_iter, 5000, stream)
    rec["pool"] = f"the batched record's {len(wls)} light fields"
    rec["slots"] = slots
    rec["iterations"] = n_iter
    rec["timing"] = ("wall clock from the first arrival to the last result on the host; "
                     "requests and results in host memory")
    return rec


def run_serve(a):
    import torch
    if int(os.environ.get("WORLD_SIZE", "1")) > 1:
        raise SystemExit("the serving workload runs on one GPU")
    seed = 5000
    t_gen = time.perf_counter()
    wls, probs = batch_problems(64, seed)          # the pool requests are drawn from
    t_gen = time.perf_counter() - t_gen
    n_iter = a.iterations if a.iterations is not None else wls[0].iterations
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    kws = [dict(U=w.U, V=w.V, H=w.H, W=w.W, scale=w.scale, blur=p[2], disparity=p[3],
                lambda1=w.lambda1, lambda2=w.lambda2, mu=w.mu, nltv_window=w.window,
                nltv_patch=w.patch, nltv_h=w.h, cg_iters=w.cg_iters, cg_tol=0.0,
                precision=a.precision) for w, p in zip(wls, probs)]
    clocks = ClockSampler(0)
    clocks.start()
    rec = serve_compare(wls, probs, kws, a.serve_rate, a.serve_seconds, a.serve_slots, n_iter,
                        seed, stream, plain=not a.serve_no_plain)
    clk = clocks.stop()
    line = {"metric": METRIC, "value": rec["value"], "unit": UNIT, "n_gpus": 1, "steps": 1,
            "warmup": 1, "ms_per_step": rec["ms_first_arrival_to_last_result"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE[a.precision],
            "data": "synthetic (seeded textured-plane light fields)",
            "config": {"workload": SERVE_WORKLOAD, "arrivals_per_s": a.serve_rate,
                       "arrival_window_s": a.serve_seconds, "requests": rec["requests"],
                       "pool": f"64 light fields of the batched distribution (seed {seed})",
                       "iterations": n_iter, "hbm_budget_gb": 120.0,
                       "slots": a.serve_slots, "iterations_per_step": 4,
                       "peak_state_gb": rec["peak_state_gb"],
                       "batch_rebuilds": rec["batch_rebuilds"], "storage": a.precision,
                       "generation_s": round(t_gen, 1),
                       "timing": "wall clock from the first arrival to the last result on "
                                 "the host; requests and results in host memory"},
            "latency_s": rec["latency_s"],
            "plain_serial": rec["plain_serial"],
            "served_vs_plain": rec["served_vs_plain"],
            "equal_psnr": rec["equal_psnr"],
            "e2e": {"value": rec["value"], "unit": UNIT, "h2d_bytes_per_step": rec["h2d_bytes"],
                    "d2h_bytes_per_step": rec["d2h_bytes"]},
            "roofline": None, "cpu_baseline": None,
            "gpu_launches": rec["gpu_launches"], "clocks": clk}
    print(json.dumps(line), flush=True)


def main():
    a = args()
    if a.workload == SERVE_WORKLOAD:
        if a.impl == "reference":
            run_reference(a, synth.batch_workloads(1, 5000)[0], 1)
        else:
            run_serve(a)
        return
    if a.workload == BATCH_WORKLOAD:
        if a.impl == "reference":
            run_reference(a, synth.batch_workloads(1)[0], 1)
        else:
            run_batch(a)
        return
    wl = synth.WORKLOADS[a.workload]
    n_iter = a.iterations if a.iterations is not None else wl.iterations
    if a.impl == "reference":
        run_reference(a, wl, n_iter)
        return

    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2206_05047_gb300 import lfsr

    prob = synth.make_problem(wl, seed=replica_seed(rank))
    blur = prob.blur.astype(np.float32)
    disp = prob.disparity.astype(np.float32)
    y_h = torch.from_numpy(prob.y.astype(np.float32)).pin_memory()
    x0_h = torch.from_numpy(prob.x0.astype(np.float32)).pin_memory()
    x_h = torch.empty(wl.HR, dtype=torch.float32).pin_memory()
    y_d = y_h.to(dev)
    x0_d = x0_h.to(dev)
    x_d = torch.empty(wl.HR, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    solver = lfsr.Solver(prob, stream=stream, precision=a.precision, **weight_kwargs(a.weights))
    h = solver.handle
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2

    def barrier():
        torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()

    def step():
        lfsr.load(h, y_d, x0_d)
        lfsr.iterate(h, n_iter)

    for _ in range(a.warmup):
        step()
    barrier()

    for attempt in range(2):        # one re-measurement if the clocks were throttled
        clocks = ClockSampler(local)
        clocks.start()
        time.sleep(0.25)
        barrier()
        evs = []
        for _ in range(a.steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            evs.append((e0, e1))
        barrier()
        clk = clocks.stop()
        clk["remeasured"] = attempt > 0
        t_ms = max_over_ranks(sum(e0.elapsed_time(e1) for e0, e1 in evs))
        if not any_rank(clocks_rejected(clk)):
            break
    p = wl.HR[0] * wl.HR[1]
    work = wl.s_k * p * n_iter * a.steps * world
    value = work / (t_ms / 1e3) / 1e6

    # kernel launches of one solve (the library counts them since the load)
    launches_per_solve = int(lfsr.stats(h)["launches"])
    # output sanity: finite, and better than the bicubic start
    lfsr.get_x(h, x_d)
    xs = x_d.cpu().numpy().astype(np.float64)
    assert np.isfinite(xs).all()

    # e2e: through lfsr_solve with pinned host buffers
    e2e = None
    if not a.no_e2e:
        barrier()
        e2e_ms = 0.0
        for _ in range(a.steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            lfsr.solve(h, y_h, n_iter, x0_h, x_h)
            e1.record(stream)
            e1.synchronize()
            e2e_ms += e0.elapsed_time(e1)
        e2e_ms = max_over_ranks(e2e_ms)
        e2e = {"value": work / (e2e_ms / 1e3) / 1e6, "unit": UNIT,
               "h2d_bytes_per_step": int(y_h.numel() * 4 + x0_h.numel() * 4),
               "d2h_bytes_per_step": int(x_h.numel() * 4)}

    # roofline of the dominant kernel (profiling mode: events around launches)
    barrier()
    lfsr.set_profiling(h, True)
    step()
    st = lfsr.stats(h)
    lfsr.set_profiling(h, False)
    names = ["nltv_block", "data_block", "cg_init", "nltv_apply", "normal_apply", "cg_update"]
    per_class = {names[i]: {"ms": st["kernel_ms"][i], "launches": st["kernel_launches"][i]}
                 for i in range(6)}
    total_prof = sum(v["ms"] for v in per_class.values())
    dom = per_class["normal_apply"]
    avg_ms = dom["ms"] / max(dom["launches"], 1)
    flops = normal_flops_per_launch(wl)
    sm_clk = (clk.get("sm_max_mhz") or 2070.0)
    n_sm = sm_count(dev)
    peak_tflops = n_sm * FP32_LANES_PER_SM * 2 * sm_clk * 1e6 / 1e12
    achieved = flops / (avg_ms / 1e3) / 1e12
    traffic = traffic_from_profile(wl)
    roofline = {"bound": "alu",
                "kernel": "k_operator_fast<OP_NORMAL> (sum_k A_k^T A_k p; with the fused CG update)",
                "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                "frac": achieved / peak_tflops, "traffic": traffic,
                "avg_launch_ms": avg_ms, "flops_per_launch": flops,
                "peak_note": f"FP32 FMA: {n_sm} SMs x {FP32_LANES_PER_SM} lanes x 2 x "
                             f"{sm_clk:.0f} MHz",
                "share_of_step": dom["ms"] / total_prof if total_prof else None,
                "per_kernel_ms_per_step": {k: v["ms"] for k, v in per_class.items()}}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            hbm = float(json.load(f)["hbm_gbs"])
        hbm_note = "of measured"
    except (OSError, KeyError, ValueError):
        hbm, hbm_note = 6800.0, "of fallback"
    step_s = t_ms / 1e3 / a.steps
    esize = 4 if a.precision == "fp32" else 2
    esize_y = 4 if a.precision in ("fp32", "fp16-views32", "bf16-views32") else 2
    hbm_frac = alg_bytes_per_iter(wl, esize, esize_y) * n_iter / step_s / (hbm * 1e9)

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        iters = 3 if wl.name != "lf5x5_64_x2" else 20
        rate, dt, cores = oracle_rate(prob, iters, a.weights)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{iters} ADMM iterations (K = {wl.cg_iters}) of {wl.name} from x0, "
                         f"{dt:.1f} s"}

    batch_rec = serve_rec = None
    if rank == 0 and world == 1 and not a.no_batch_record and a.workload == "lf9x9_256_x2":
        batch_rec, pool = batch_subrecord(dev, stream)
        serve_rec = serve_subrecord(stream, *pool)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": a.steps, "warmup": a.warmup, "ms_per_step": t_ms / a.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": DTYPE[a.precision],
                "data": "synthetic (seeded textured-plane light field)",
                "config": workload_config(wl, n_iter, {
                    "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                    "weights": "patch distance exp(-pd/h^2)" if a.weights == "patch" else
                               "paper (Sec. 3.4): " + ", ".join(
                                   f"{k}={v:g}" for k, v in synth.PAPER_SIGMAS.items()),
                    "storage": {"fp32": "f32", "fp16": "f16 (views, duals, NLTV weights)",
                                "bf16": "bf16 (views, duals, NLTV weights)",
                                "fp16-views32": "f16 (duals, NLTV weights), f32 views",
                                "bf16-views32": "bf16 (duals, NLTV weights), f32 views"}[
                                    a.precision],
                    "l2": "flushed between steps (256 MB write); per-step working set "
                          f"{st['state_bytes'] / 1e6:.0f} MB"}),
                "hbm_roofline": {"frac": hbm_frac,
                                 "alg_bytes_per_iter": alg_bytes_per_iter(wl, esize, esize_y),
                                 "peak_gbs": hbm, "note": hbm_note},
                # the reference view alone: HR Mpix * ADMM iterations per second
                "sai_rate": {"value": p * n_iter * a.steps * world / (t_ms / 1e3) / 1e6,
                             "unit": "HR Mpix*iter/s (reference view)"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "batched": batch_rec, "served": serve_rec,
                "gpu_launches": int(a.steps * launches_per_solve),
                "launches_per_iteration": launches_per_solve / max(n_iter, 1),
                "clocks": clk}
        print(json.dumps(line), flush=True)
    solver.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

"""16-bit storage of the large streams (LR views, data and regulariser
duals, stored NLTV weights) with float32 arithmetic:
the storage conversions are bit-exact against numpy's round-to-nearest-even,
and whole solves are compared with the float64 oracle, each result with its
own stated error.

Targets for a 16-bit variant (float64 oracle on the same float32 inputs):
relative L2 error of x <= 1e-3 and |dPSNR| <= 0.05 dB.  The float32 path
keeps its own tolerance (1e-4, 0.01 dB) in test_gpu_parity.py.

Errors are measured at the workloads' configured h = 0.1.
"""
import json
import os

import numpy as np
import pytest

from paper_2206_05047_gb300 import lfsr, synth
from tests.gpu_util import ROUND, Case, check_golden_inputs, f32, golden, rel_err

pytestmark = pytest.mark.gpu

# (rel-L2, |dPSNR| dB) stated per variant; "-views32" keeps the views in
# float32 (LFSR_KEEP_VIEWS_FP32)
TARGET = {"fp16": (1e-3, 0.05), "fp16-views32": (1e-3, 0.05),
          "bf16": (1e-3, 0.05), "bf16-views32": (1e-3, 0.05)}
VARIANTS = list(TARGET)


def _report(rec):
    """Appends a measured error record to $LFSR_PRECISION_REPORT (JSON lines)
    when that variable is set."""
    path = os.environ.get("LFSR_PRECISION_REPORT")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps(rec) + "\n")


def _small(precision, **over):
    wl = synth.custom(U=3, V=3, H=14, W=13, scale=2, kb=5, blur_sigma=1.0, window=5)
    return Case(wl, seed=3, precision=precision, **over)


def _edge_mask(o):
    """[d][u] is 1 where u + d lies inside the HR image."""
    Hh, Wh = o.hr
    m = np.zeros((o.s_d, Hh, Wh), np.float32)
    for n, (di, dj) in enumerate(zip(*o.dirs())):
        di, dj = int(di), int(dj)
        m[n, max(0, -di):min(Hh, Hh - di), max(0, -dj):min(Wh, Wh - dj)] = 1.0
    return m


@pytest.mark.parametrize("precision", ["fp16", "bf16"])
def test_state_round_trip_is_round_to_nearest_even(precision):
    c = _small(precision)
    o, wl = c.oracle, c.wl
    rng = np.random.default_rng(5)
    x = f32(rng.random(o.hr))
    wA = f32(rng.uniform(-1, 1, (o.s_k, wl.H, wl.W)))
    wA.flat[:4] = [1.0 + 2.0 ** -11, -0.333333, 6.1e-5, 1e-9]   # ties, subnormals
    wS = f32(rng.uniform(-1, 1, (o.s_d,) + o.hr)) * _edge_mask(o)
    lfsr.load(c.h, c.t(c.y), c.t(x))
    lfsr.set_state(c.h, c.t(x), c.t(wA), c.t(wS))
    gx, gA, gS = c.empty(*o.hr), c.empty(o.s_k, wl.H, wl.W), c.empty(o.s_d, *o.hr)
    lfsr.get_state(c.h, gx, gA, gS)
    rnd = ROUND[precision]
    assert np.array_equal(c.np(gx), x.astype(np.float64))          # x stays float32
    assert np.array_equal(c.np(gA), rnd(wA).astype(np.float64))
    assert np.array_equal(c.np(gS), rnd(wS).astype(np.float64))
    # host-memory path
    hA = np.zeros_like(wA)
    lfsr.get_state(c.h, None, hA, None)
    assert np.array_equal(hA, rnd(wA))


@pytest.mark.parametrize("precision", ["fp16", "bf16"])
def test_stored_weights_are_rounded_weights(precision):
    c = _small(precision)
    o = c.oracle
    rng = np.random.default_rng(2)
    x = f32(rng.random(o.hr))
    w = c.empty(o.s_d, *o.hr)
    lfsr.weights(c.h, c.t(x), w)
    ref = o.weights(x.astype(np.float64))
    # float32 weights within 3e-5 (see test_gpu_parity), then one rounding
    ulp = {"fp16": 2.0 ** -11, "bf16": 2.0 ** -8}[precision]
    assert np.abs(c.np(w) - ref).max() <= 3e-5 + ulp
    got = c.np(w).astype(np.float32)
    assert np.array_equal(got, ROUND[precision](got))                # representable


# one ADMM iteration from a state the storage type represents exactly:
# separable fast path, non-separable blur (generic operator kernel), and a
# 9x9 window (generic NLTV kernel, weights recomputed on the fly)
ONE_ITER = [
    ("x2_5x5", dict(U=5, V=5, H=21, W=19, scale=2, kb=5, blur_sigma=1.0, window=5,
                    disparities=(-1.0, 0.0, 0.8)), None),
    ("x4_nonsep", dict(U=3, V=3, H=9, W=10, scale=4, kb=5, blur_sigma=1.0, window=7,
                       disparities=(-0.6, 1.2)), "motion"),
    ("x2_window9", dict(U=3, V=3, H=12, W=13, scale=2, kb=3, blur_sigma=0.8, window=9,
                        disparities=(-0.7, 0.9)), None),
    # rows of 40 16-bit weights (80 bytes): the NLTV apply stages them with
    # TMA; ragged tiles, 7x7 window
    ("x2_tma_ragged", dict(U=3, V=3, H=22, W=20, scale=2, kb=5, blur_sigma=1.0, window=7,
                           disparities=(-0.9, 0.7)), None),
]
# rel-L2 bounds of one iteration: outputs rounded once, plus the rounded
# weights / divergence terms inside the x-step
ONE_ITER_TOL = {"fp16": 1e-3, "bf16": 8e-3}


@pytest.mark.parametrize("precision", ["fp16", "bf16"])
@pytest.mark.parametrize("name", [c[0] for c in ONE_ITER])
def test_one_iteration_from_representable_state(name, precision):
    ov, blur = {n: (o, b) for n, o, b in ONE_ITER}[name]
    wl = synth.custom(**ov)
    kw = {}
    if blur == "motion":
        K = np.random.default_rng(9).random((wl.kb, wl.kb)) ** 3
        kw["blur"] = K / K.sum()
    c = Case(wl, seed=1, precision=precision, **kw)
    o = c.oracle
    rnd = ROUND[precision]
    rng = np.random.default_rng(3)
    wA = rnd(f32(np.clip(0.6 * rng.standard_normal((o.s_k, wl.H, wl.W)), -1, 1)))
    wS = rnd(f32(np.clip(0.6 * rng.standard_normal((o.s_d,) + o.hr), -1, 1)) * _edge_mask(o))
    y = rnd(c.y)
    lfsr.load(c.h, c.t(y), c.t(c.x0))
    lfsr.set_state(c.h, c.t(c.x0), c.t(wA), c.t(wS))
    lfsr.iterate(c.h, 1)
    xs, wAs, wSs = c.empty(*o.hr), c.empty(*wA.shape), c.empty(*wS.shape)
    lfsr.get_state(c.h, xs, wAs, wSs)
    rx, rA, rS = o.admm(y.astype(np.float64), c.x0.astype(np.float64), 1,
                        wA=wA.astype(np.float64), wS=wS.astype(np.float64))
    errs = (rel_err(c.np(xs), rx), rel_err(c.np(wAs), rA), rel_err(c.np(wSs), rS))
    _report({"case": name, "precision": precision, "one_iteration_rel_l2": errs})
    assert max(errs) <= ONE_ITER_TOL[precision], errs


def test_view_out_of_half_range_is_reported():
    c = _small("fp16")
    y = c.y.copy()
    y[0, 0, 0] = 1e5
    x = c.empty(*c.oracle.hr)
    with pytest.raises(lfsr.LfsrError) as e:
        lfsr.solve(c.h, c.t(y), 1, c.t(c.x0), x)
    assert e.value.code == lfsr.LFSR_EINVAL
    # a clean load clears the status
    lfsr.solve(c.h, c.t(c.y), 1, c.t(c.x0), x)
    assert np.isfinite(c.np(x)).all()


def test_bf16_accepts_large_views_and_rejects_nonfinite():
    c = _small("bf16")
    y = c.y.copy()
    y[0, 0, 0] = 1e5
    x = c.empty(*c.oracle.hr)
    lfsr.solve(c.h, c.t(y), 1, c.t(c.x0), x)
    y[0, 0, 1] = np.inf
    with pytest.raises(lfsr.LfsrError) as e:
        lfsr.solve(c.h, c.t(y), 1, c.t(c.x0), x)
    assert e.value.code == lfsr.LFSR_EINVAL


@pytest.mark.parametrize("precision", VARIANTS)
def test_state_bytes_halve(precision):
    a = _small("fp32")
    b = _small(precision)
    sa, sb = lfsr.stats(a.h)["state_bytes"], lfsr.stats(b.h)["state_bytes"]
    o = a.oracle
    p, q = o.hr[0] * o.hr[1], a.wl.H * a.wl.W
    n16 = 2 * o.s_k * q + 2 * o.s_d * p + (o.s_d // 2) * p   # wA x2, wS x2 (pairs), wt
    if not precision.endswith("views32"):
        n16 += o.s_k * q                                     # y
    assert sa - sb == 2 * n16


def _full_solve(wl, precision, n_iter, seed=0):
    c = Case(wl, seed=seed, precision=precision)
    x = c.empty(*c.oracle.hr)
    lfsr.solve(c.h, c.t(c.y), n_iter, c.t(c.x0), x)
    ref, _, _ = c.oracle.admm(c.y.astype(np.float64), c.x0.astype(np.float64), n_iter)
    gx = c.np(x)
    e = rel_err(gx, ref)
    dp = synth.psnr(gx, c.prob.gt) - synth.psnr(ref, c.prob.gt)
    st = lfsr.stats(c.h)
    assert st["status"] == 0
    _report({"workload": wl.name, "precision": precision, "iterations": n_iter, "h": wl.h,
             "rel_l2": e, "dpsnr_db": dp, "psnr_oracle": synth.psnr(ref, c.prob.gt)})
    return e, dp


@pytest.mark.parametrize("precision", VARIANTS)
def test_lf5x5_full_solve_storage(precision):
    """5x5 views, 64^2 -> 128^2, 50 iterations."""
    wl = synth.WORKLOADS["lf5x5_64_x2"]
    e, dp = _full_solve(wl, precision, wl.iterations)
    tol_e, tol_p = TARGET[precision]
    assert e <= tol_e, f"{precision}: rel-L2 {e:.3e}"
    assert abs(dp) <= tol_p, f"{precision}: dPSNR {dp:+.4f} dB"


@pytest.mark.parametrize("precision", ["fp32"] + VARIANTS)
def test_lf9x9_200_x3_first_iterations_storage(precision):
    """9x9 views, 200^2 -> 600^2 (x3, 9x9 blur), the first 3 iterations."""
    wl = synth.WORKLOADS["lf9x9_200_x3"]
    e, dp = _full_solve(wl, precision, 3)
    tol_e, tol_p = (1e-4, 0.01) if precision == "fp32" else TARGET[precision]
    assert e <= tol_e, f"{precision}: rel-L2 {e:.3e}"
    assert abs(dp) <= tol_p, f"{precision}: dPSNR {dp:+.4f} dB"


@pytest.mark.parametrize("precision", ["fp32"] + VARIANTS)
def test_lf9x9_200_x3_full_N_storage(precision):
    """The x3 workload through all 100 iterations, against the oracle's
    stored float64 iterate (tests/golden/, seed 3000)."""
    name, seed = "lf9x9_200_x3", 3000
    wl = synth.WORKLOADS[name]
    g = golden(name, seed, wl.iterations)
    c = Case(wl, seed=seed, precision=precision)
    check_golden_inputs(c, g)
    x = c.empty(*c.oracle.hr)
    lfsr.solve(c.h, c.t(c.y), wl.iterations, c.t(c.x0), x)
    gx = c.np(x)
    e = rel_err(gx, g["x"])
    dp = synth.psnr(gx, c.prob.gt) - float(g["psnr_x"])
    assert lfsr.stats(c.h)["status"] == 0
    _report({"workload": name, "precision": precision, "iterations": wl.iterations, "h": wl.h,
             "rel_l2": e, "dpsnr_db": dp, "psnr_oracle": float(g["psnr_x"])})
    tol_e, tol_p = (1e-4, 0.01) if precision == "fp32" else TARGET[precision]
    assert e <= tol_e, f"{precision}: rel-L2 {e:.3e}"
    assert abs(dp) <= tol_p, f"{precision}: dPSNR {dp:+.4f} dB"
    c.solver.close()

"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
identical seeded float32 inputs.

Tolerances (FP32 arithmetic with FP64 reductions against FP64):
  single operators       max-abs error <= 2e-6 of the output's max
  NLTV weights           abs error <= 3e-5 (exp(-pd/h^2) multiplies the FP32
                         rounding of pd by 1/h^2 = 100 at h = 0.1)
  one ADMM iteration     rel-L2 <= 2e-5 on x and on both dual blocks
  full solve, fixed N    rel-L2 <= 1e-4 and |dPSNR| <= 0.01 dB
"""
import math

import numpy as np
import pytest

from paper_2206_05047_gb300 import lfsr, synth
from tests.gpu_util import Case, f32, max_err, rel_err

pytestmark = pytest.mark.gpu

SMALL = [
    # (name, workload overrides, blur override)
    ("x2_5x5", dict(U=5, V=5, H=21, W=19, scale=2, kb=5, blur_sigma=1.0, window=5,
                    disparities=(-1.0, 0.0, 0.8)), None),
    ("x3_odd", dict(U=3, V=5, H=13, W=11, scale=3, kb=7, blur_sigma=1.3, window=3, patch=1,
                    disparities=(-2.3, 0.4, 1.7)), None),
    ("x4_nonsep", dict(U=3, V=3, H=9, W=10, scale=4, kb=5, blur_sigma=1.0, window=7,
                       disparities=(-0.6, 1.2)), "motion"),
    ("x1_single_view", dict(U=1, V=1, H=20, W=23, scale=1, kb=3, blur_sigma=0.7, window=5,
                            disparities=(0.0, 0.5)), None),
    ("x2_big_shift", dict(U=7, V=3, H=12, W=40, scale=2, kb=3, blur_sigma=0.8, window=3,
                          disparities=(-3.6, 2.9)), None),
    # rows of 40 floats (16-byte multiples): the NLTV apply stages its weight
    # planes with TMA; ragged 32 x 32 tiles in both directions, 7x7 window
    ("x2_tma_ragged", dict(U=3, V=3, H=22, W=20, scale=2, kb=5, blur_sigma=1.0, window=7,
                           disparities=(-0.9, 0.7)), None),
    # 9x9 window: the generic NLTV kernel (weights recomputed per direction)
    ("x2_window9", dict(U=3, V=3, H=12, W=13, scale=2, kb=3, blur_sigma=0.8, window=9,
                        disparities=(-0.7, 0.9)), None),
]


def _case(name, seed=0, **over):
    ov, blur = {n: (o, b) for n, o, b in SMALL}[name]
    wl = synth.custom(**ov)
    kw = {}
    if blur == "motion":
        rng = np.random.default_rng(9)
        K = rng.random((wl.kb, wl.kb)) ** 3
        kw["blur"] = K / K.sum()
    return Case(wl, seed=seed, **kw, **over)


@pytest.mark.parametrize("name", [c[0] for c in SMALL])
def test_forward_and_adjoint_operators(name):
    c = _case(name)
    o, wl = c.oracle, c.wl
    rng = np.random.default_rng(1)
    x = f32(rng.random(o.hr))
    g = f32(rng.standard_normal((o.s_k, wl.H, wl.W)))
    out = c.empty(o.s_k, wl.H, wl.W)
    lfsr.apply_A(c.h, -1, c.t(x), out)
    ref = np.stack([o.A(k, x.astype(np.float64)) for k in range(o.s_k)])
    assert max_err(c.np(out), ref) <= 2e-6
    # single view, host memory path
    k = o.s_k - 1
    out1 = np.zeros((wl.H, wl.W), np.float32)
    lfsr.apply_A(c.h, k, x, out1)
    assert max_err(out1, ref[k]) <= 2e-6
    # adjoint, all views summed and one view
    outT = c.empty(*o.hr)
    lfsr.apply_AT(c.h, -1, c.t(g), outT)
    refT = sum(o.A_T(kk, g[kk].astype(np.float64)) for kk in range(o.s_k))
    assert max_err(c.np(outT), refT) <= 2e-6
    outT1 = c.empty(*o.hr)
    lfsr.apply_AT(c.h, 0, c.t(g[0]), outT1)
    assert max_err(c.np(outT1), o.A_T(0, g[0].astype(np.float64))) <= 2e-6


@pytest.mark.parametrize("name", [c[0] for c in SMALL])
def test_adjoint_identity_in_float32(name):
    """<A x, g> = <x, A^T g> from the kernels' own float32 outputs (summed in
    float64), to 1e-5 relative."""
    c = _case(name)
    o, wl = c.oracle, c.wl
    rng = np.random.default_rng(11)
    for _ in range(2):
        x = f32(rng.standard_normal(o.hr))
        g = f32(rng.standard_normal((o.s_k, wl.H, wl.W)))
        ax = c.empty(o.s_k, wl.H, wl.W)
        atg = c.empty(*o.hr)
        lfsr.apply_A(c.h, -1, c.t(x), ax)
        lfsr.apply_AT(c.h, -1, c.t(g), atg)
        lhs = float(np.vdot(c.np(ax), g.astype(np.float64)))
        rhs = float(np.vdot(x.astype(np.float64), c.np(atg)))
        scale = np.linalg.norm(c.np(ax)) * np.linalg.norm(g)
        assert abs(lhs - rhs) <= 1e-5 * scale


@pytest.mark.parametrize("name", [c[0] for c in SMALL])
def test_weights(name):
    c = _case(name)
    o = c.oracle
    x = c.x0
    w = c.empty(o.s_d, *o.hr)
    lfsr.weights(c.h, c.t(x), w)
    ref = o.weights(x.astype(np.float64))
    assert np.abs(c.np(w) - ref).max() <= 3e-5


@pytest.mark.parametrize("name", [c[0] for c in SMALL])
def test_normal_matrix(name):
    c = _case(name)
    o = c.oracle
    rng = np.random.default_rng(2)
    p = f32(rng.standard_normal(o.hr))
    q = c.empty(*o.hr)
    pMp = lfsr.apply_normal(c.h, c.t(c.x0), c.t(p), q)
    w = o.weights(c.x0.astype(np.float64))
    ref = o.normal_apply(w, p.astype(np.float64))
    assert max_err(c.np(q), ref) <= 5e-6
    ref_pMp = float(np.vdot(p.astype(np.float64), ref))
    assert abs(pMp - ref_pMp) <= 2e-6 * abs(ref_pMp)


def _random_duals(c, rng):
    o, wl = c.oracle, c.wl
    t = 1.0 / c.params["mu"]
    wA = f32(np.clip(0.6 * t * rng.standard_normal((o.s_k, wl.H, wl.W)), -t, t))
    wS = np.clip(0.6 * t * rng.standard_normal((o.s_d,) + o.hr), -t, t)
    # duals of pairs that leave the image are zero in both layouts
    di, dj = o.dirs()
    Hh, Wh = o.hr
    ii, jj = np.meshgrid(np.arange(Hh), np.arange(Wh), indexing="ij")
    for d in range(o.s_d):
        inside = (ii + di[d] >= 0) & (ii + di[d] < Hh) & (jj + dj[d] >= 0) & (jj + dj[d] < Wh)
        wS[d][~inside] = 0.0
    return wA, f32(wS)


@pytest.mark.parametrize("name", [c[0] for c in SMALL])
def test_one_iteration_from_state(name):
    """One ADMM iteration from an identical (x, wA, wS) state."""
    c = _case(name)
    o = c.oracle
    rng = np.random.default_rng(3)
    wA, wS = _random_duals(c, rng)
    lfsr.load(c.h, c.t(c.y), c.t(c.x0))
    lfsr.set_state(c.h, c.t(c.x0), c.t(wA), c.t(wS))
    xs, wAs, wSs = c.empty(*o.hr), c.empty(*wA.shape), c.empty(*wS.shape)
    lfsr.get_state(c.h, xs, wAs, wSs)
    assert np.array_equal(c.np(xs), c.x0) and np.array_equal(c.np(wAs), wA)
    assert np.array_equal(c.np(wSs), wS)          # layout round trip is exact
    lfsr.iterate(c.h, 1)
    lfsr.get_state(c.h, xs, wAs, wSs)
    rx, rA, rS = o.admm(c.y.astype(np.float64), c.x0.astype(np.float64), 1,
                        wA=wA.astype(np.float64), wS=wS.astype(np.float64))
    assert rel_err(c.np(xs), rx) <= 2e-5
    assert rel_err(c.np(wAs), rA) <= 2e-5
    assert rel_err(c.np(wSs), rS) <= 2e-5


@pytest.mark.parametrize("h", [None, 0.3])
def test_config_lf5x5_full_solve_parity(h):
    """5x5 views, 64^2 -> 128^2, 50 ADMM iterations of K = 5 CG steps, at the
    configured h = 0.1 (and at h = 0.3): rel-L2 <= 1e-4 and |dPSNR| <= 0.01 dB."""
    wl = synth.WORKLOADS["lf5x5_64_x2"]
    c = Case(wl, seed=0, **({} if h is None else {"h": h}))
    x = c.empty(*c.oracle.hr)
    lfsr.solve(c.h, c.t(c.y), wl.iterations, c.t(c.x0), x)
    ref, _, _ = c.oracle.admm(c.y.astype(np.float64), c.x0.astype(np.float64), wl.iterations)
    gx = c.np(x)
    assert rel_err(gx, ref) <= 1e-4
    assert abs(synth.psnr(gx, c.prob.gt) - synth.psnr(ref, c.prob.gt)) <= 0.01
    st = lfsr.stats(c.h)
    assert st["iterations"] == wl.iterations and st["status"] == 0 and st["cg_steps"] == 5


def test_config_lf5x5_twice_the_iterations():
    """The configured workload through 100 iterations (twice its N): the
    iteration stays stable, so the fixed-N parity still holds."""
    wl = synth.WORKLOADS["lf5x5_64_x2"]
    c = Case(wl, seed=1)
    x = c.empty(*c.oracle.hr)
    lfsr.solve(c.h, c.t(c.y), 2 * wl.iterations, c.t(c.x0), x)
    ref, _, _ = c.oracle.admm(c.y.astype(np.float64), c.x0.astype(np.float64), 2 * wl.iterations)
    assert rel_err(c.np(x), ref) <= 1e-4
    assert synth.psnr(ref, c.prob.gt) > synth.psnr(c.x0, c.prob.gt) + 3.0


def test_host_memory_solve_matches_device():
    wl = synth.custom(U=3, V=3, H=16, W=16, scale=2, kb=5, blur_sigma=1.0, window=5)
    c = Case(wl, seed=4, h=0.3)
    xd = c.empty(*c.oracle.hr)
    lfsr.solve(c.h, c.t(c.y), 6, c.t(c.x0), xd)
    xh = np.zeros(c.oracle.hr, np.float32)
    lfsr.solve(c.h, c.y, 6, c.x0, xh)
    assert rel_err(xh, c.np(xd)) <= 1e-5


def test_cg_early_exit_and_zero_steps():
    wl = synth.custom(U=3, V=3, H=12, W=12, scale=2, kb=3, blur_sigma=0.8, window=3)
    # tau above the initial |r|^2 of the second iteration's x-step is hit at
    # different steps; compare the step count and result with the oracle
    for K, tau in ((0, 0.0), (5, 1e-3), (8, 1e-6)):
        c = Case(wl, seed=5, h=0.3, cg_iters=K, cg_tol=tau)
        x = c.empty(*c.oracle.hr)
        lfsr.solve(c.h, c.t(c.y), 3, c.t(c.x0), x)
        ref, _, _, diag = c.oracle.admm(c.y.astype(np.float64), c.x0.astype(np.float64), 3,
                                        diagnostics=True)
        assert rel_err(c.np(x), ref) <= 2e-5, (K, tau)
        assert lfsr.stats(c.h)["cg_steps"] == int(diag[-1, 4]), (K, tau)
        c.solver.close()


def test_invalid_parameters_are_rejected():
    blur = np.ones((3, 3), np.float32) / 9
    disp = np.zeros((16, 16), np.float32)
    with pytest.raises(lfsr.LfsrError) as e:
        lfsr.create(3, 3, 8, 8, 2, blur, disp, mu=0.0)
    assert e.value.code == lfsr.LFSR_EINVAL
    with pytest.raises(lfsr.LfsrError) as e:
        lfsr.create(3, 3, 8, 8, 5, blur, np.zeros((40, 40), np.float32))
    assert e.value.code == lfsr.LFSR_EUNSUPPORTED
    bad = disp.copy()
    bad[3, 3] = np.nan
    with pytest.raises(lfsr.LfsrError):
        lfsr.create(3, 3, 8, 8, 2, blur, bad)


@pytest.mark.parametrize("kind", ["smooth", "constant"])
def test_disparity_paths(kind):
    """The operator kernel takes a shared-split path on row segments of
    constant disparity and a per-pixel path elsewhere: a smoothly varying
    map exercises only the latter, a constant map only the former."""
    wl = synth.custom(U=5, V=5, H=70, W=66, scale=2, kb=7, blur_sigma=1.2, window=7)
    hr = wl.HR
    if kind == "smooth":
        ii, jj = np.meshgrid(np.arange(hr[0]), np.arange(hr[1]), indexing="ij")
        disp = 1.3 * np.sin(ii / 17.0) * np.cos(jj / 23.0) + 0.25
    else:
        disp = np.full(hr, -0.7)
    c = Case(wl, seed=8, disparity=disp, h=0.3)
    o = c.oracle
    rng = np.random.default_rng(12)
    x = f32(rng.random(o.hr))
    out = c.empty(o.s_k, wl.H, wl.W)
    lfsr.apply_A(c.h, -1, c.t(x), out)
    ref = np.stack([o.A(k, x.astype(np.float64)) for k in range(o.s_k)])
    assert max_err(c.np(out), ref) <= 2e-6
    p = f32(rng.standard_normal(o.hr))
    q = c.empty(*o.hr)
    pMp = lfsr.apply_normal(c.h, c.t(c.x0), c.t(p), q)
    qref = o.normal_apply(o.weights(c.x0.astype(np.float64)), p.astype(np.float64))
    assert max_err(c.np(q), qref) <= 5e-6
    assert abs(pMp - float(np.vdot(p, qref))) <= 2e-6 * abs(float(np.vdot(p, qref)))
    x_out = c.empty(*o.hr)
    lfsr.solve(c.h, c.t(c.y), 3, c.t(c.x0), x_out)
    rx, _, _ = o.admm(c.y.astype(np.float64), c.x0.astype(np.float64), 3)
    assert rel_err(c.np(x_out), rx) <= 2e-5

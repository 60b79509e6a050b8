"""The warp options of Sec. 4.1 on the CUDA path against the FP64 oracle:
per-view disparity maps omega_k for W_k (the generic operator kernel reads
view k's map), and the paper's backward warp W_k^* in the x-step (a gather
kernel over LR buffers, in place of the exact adjoint's scatter).

Tolerances as for the generic kernels in test_gpu_parity.py: operators
max-abs <= 2e-6 of the output's max, the normal matrix <= 5e-6 and
<p, M p> rel 2e-6, one ADMM iteration rel-L2 <= 2e-5, solves rel-L2 <= 1e-4
and |dPSNR| <= 0.01 dB."""
import numpy as np
import pytest

from paper_2206_05047_gb300 import lfsr, synth
from tests.gpu_util import Case, f32, max_err, rel_err

pytestmark = pytest.mark.gpu

GEOMS = {
    "x2_5x5": dict(U=5, V=5, H=21, W=19, scale=2, kb=5, blur_sigma=1.0, window=5,
                   disparities=(-1.0, 0.0, 0.8)),
    "x3_3x5": dict(U=3, V=5, H=13, W=11, scale=3, kb=7, blur_sigma=1.3, window=3, patch=1,
                   disparities=(-2.3, 0.4, 1.7)),
    "x4_nonsep": dict(U=3, V=3, H=9, W=10, scale=4, kb=5, blur_sigma=1.0, window=7,
                      disparities=(-0.6, 1.2)),
}


def _case(name, maps="scene", adjoint="exact", seed=0):
    wl = synth.custom(**GEOMS[name])
    kw = {}
    if name == "x4_nonsep":
        K = np.random.default_rng(9).random((wl.kb, wl.kb)) ** 3
        kw["blur"] = K / K.sum()
    dv = None
    if maps == "scene":
        dv = synth.view_disparity_maps(synth.make_problem(wl, seed=seed))
    elif maps == "random":
        dv = np.random.default_rng(12).uniform(-1.3, 1.3, (wl.s_k,) + wl.HR)
    return Case(wl, seed=seed, disparity_views=dv, adjoint=adjoint, **kw)


@pytest.mark.parametrize("name", list(GEOMS))
@pytest.mark.parametrize("maps", ["scene", "random"])
def test_per_view_map_operators(name, maps):
    c = _case(name, maps)
    o, wl = c.oracle, c.wl
    rng = np.random.default_rng(1)
    x = f32(rng.random(o.hr))
    g = f32(rng.standard_normal((o.s_k, wl.H, wl.W)))
    out = c.empty(o.s_k, wl.H, wl.W)
    lfsr.apply_A(c.h, -1, c.t(x), out)
    ref = np.stack([o.A(k, x.astype(np.float64)) for k in range(o.s_k)])
    assert max_err(c.np(out), ref) <= 2e-6
    outT = c.empty(*o.hr)
    lfsr.apply_AT(c.h, -1, c.t(g), outT)
    refT = sum(o.A_T(k, g[k].astype(np.float64)) for k in range(o.s_k))
    assert max_err(c.np(outT), refT) <= 2e-6


def _a_star(o, k, g):
    return o.warp_bw(k, o.blur_T(o.up(g)))


@pytest.mark.parametrize("name", list(GEOMS))
@pytest.mark.parametrize("maps", [None, "scene"])
def test_backward_warp_adjoint_and_normal_matrix(name, maps):
    c = _case(name, maps, adjoint="backward")
    o, wl = c.oracle, c.wl
    rng = np.random.default_rng(2)
    g = f32(rng.standard_normal((o.s_k, wl.H, wl.W)))
    outT = c.empty(*o.hr)
    lfsr.apply_AT(c.h, -1, c.t(g), outT)
    ref = sum(_a_star(o, k, g[k].astype(np.float64)) for k in range(o.s_k))
    assert max_err(c.np(outT), ref) <= 2e-6
    k = o.s_k - 1                              # one view, host memory
    out1 = np.zeros(o.hr, np.float32)
    lfsr.apply_AT(c.h, k, g[k], out1)
    assert max_err(out1, _a_star(o, k, g[k].astype(np.float64))) <= 2e-6
    p = f32(rng.standard_normal(o.hr))
    q = c.empty(*o.hr)
    pMp = lfsr.apply_normal(c.h, c.t(c.x0), c.t(p), q)
    refq = o.normal_apply(o.weights(c.x0.astype(np.float64)), p.astype(np.float64))
    assert max_err(c.np(q), refq) <= 5e-6
    ref_pMp = float(np.vdot(p.astype(np.float64), refq))
    assert abs(pMp - ref_pMp) <= 2e-6 * abs(ref_pMp)


def _random_duals(c, rng):
    o, wl = c.oracle, c.wl
    t = 1.0 / c.params["mu"]
    wA = f32(np.clip(0.6 * t * rng.standard_normal((o.s_k, wl.H, wl.W)), -t, t))
    wS = np.clip(0.6 * t * rng.standard_normal((o.s_d,) + o.hr), -t, t)
    di, dj = o.dirs()
    Hh, Wh = o.hr
    ii, jj = np.meshgrid(np.arange(Hh), np.arange(Wh), indexing="ij")
    for d in range(o.s_d):
        inside = (ii + di[d] >= 0) & (ii + di[d] < Hh) & (jj + dj[d] >= 0) & (jj + dj[d] < Wh)
        wS[d][~inside] = 0.0
    return wA, f32(wS)


@pytest.mark.parametrize("name", list(GEOMS))
@pytest.mark.parametrize("maps,adjoint", [("scene", "exact"), (None, "backward"),
                                          ("random", "backward")])
def test_one_iteration_from_state(name, maps, adjoint):
    c = _case(name, maps, adjoint)
    o = c.oracle
    wA, wS = _random_duals(c, np.random.default_rng(3))
    lfsr.load(c.h, c.t(c.y), c.t(c.x0))
    lfsr.set_state(c.h, c.t(c.x0), c.t(wA), c.t(wS))
    lfsr.iterate(c.h, 1)
    xs, wAs, wSs = c.empty(*o.hr), c.empty(*wA.shape), c.empty(*wS.shape)
    lfsr.get_state(c.h, xs, wAs, wSs)
    rx, rA, rS = o.admm(c.y.astype(np.float64), c.x0.astype(np.float64), 1,
                        wA=wA.astype(np.float64), wS=wS.astype(np.float64))
    assert rel_err(c.np(xs), rx) <= 2e-5
    assert rel_err(c.np(wAs), rA) <= 2e-5
    assert rel_err(c.np(wSs), rS) <= 2e-5
    K = c.params["cg_iters"]
    bw = 1 if adjoint == "backward" else 0
    assert lfsr.stats(c.h)["launches"] == 3 + bw + (3 + bw) * K


@pytest.mark.parametrize("maps,adjoint", [("scene", "exact"), ("scene", "backward"),
                                          (None, "backward")])
def test_full_solve(maps, adjoint):
    c = _case("x2_5x5", maps, adjoint)
    n_iter = 12
    x = c.empty(*c.oracle.hr)
    lfsr.solve(c.h, c.t(c.y), n_iter, c.t(c.x0), x)
    ref, _, _ = c.oracle.admm(c.y.astype(np.float64), c.x0.astype(np.float64), n_iter)
    gx = c.np(x)
    assert rel_err(gx, ref) <= 1e-4
    assert abs(synth.psnr(gx, c.prob.gt) - synth.psnr(ref, c.prob.gt)) <= 0.01
    assert lfsr.stats(c.h)["status"] == 0


def test_batches_take_neither_option():
    wl = synth.custom(**GEOMS["x2_5x5"])
    pr = synth.make_problem(wl, seed=0)
    base = dict(U=wl.U, V=wl.V, H=wl.H, W=wl.W, scale=wl.scale, blur=f32(pr.blur),
                disparity=f32(pr.disparity), nltv_window=5)
    for extra in (dict(adjoint="backward"),
                  dict(disparity_views=synth.view_disparity_maps(pr))):
        with pytest.raises(lfsr.LfsrError) as e:
            lfsr.Batch([base, dict(base, **extra)])
        assert e.value.code == lfsr.LFSR_EUNSUPPORTED

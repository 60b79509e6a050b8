"""View subsets (Sec. 6.1's x4 experiment: 17 SAIs of a 5 x 5 grid in a
star): the CUDA path against the FP64 oracle with the same subset."""
import numpy as np
import pytest

from paper_2206_05047_gb300 import lfsr, synth
from tests.gpu_util import Case, f32, max_err, rel_err

pytestmark = pytest.mark.gpu


def _star_case(scale=4, H=14, W=13, kb=7, seed=0):
    wl = synth.custom(U=5, V=5, H=H, W=W, scale=scale, kb=kb, blur_sigma=1.2, window=5,
                      disparities=(-0.9, 0.4, 1.3))
    return Case(wl, seed=seed, views=synth.star_views(5, 5))


def test_star_subset_operators():
    c = _star_case()
    o, wl = c.oracle, c.wl
    assert o.s_k == 17
    x = f32(np.random.default_rng(1).random(o.hr))
    out = c.empty(17, wl.H, wl.W)
    lfsr.apply_A(c.h, -1, c.t(x), out)
    ref = np.stack([o.A(j, x.astype(np.float64)) for j in range(17)])
    assert max_err(c.np(out), ref) <= 2e-6
    g = f32(np.random.default_rng(2).standard_normal((17, wl.H, wl.W)))
    q = c.empty(*o.hr)
    lfsr.apply_AT(c.h, -1, c.t(g), q)
    refT = sum(o.A_T(j, g[j].astype(np.float64)) for j in range(17))
    assert max_err(c.np(q), refT) <= 2e-6


@pytest.mark.parametrize("scale,kb", [(4, 7), (2, 5)])
def test_star_subset_solve(scale, kb):
    c = _star_case(scale=scale, kb=kb, H=16, W=15)
    x = c.empty(*c.oracle.hr)
    n = 12
    lfsr.solve(c.h, c.t(c.y), n, c.t(c.x0), x)
    ref, _, _ = c.oracle.admm(c.y.astype(np.float64), c.x0.astype(np.float64), n)
    assert rel_err(c.np(x), ref) <= 1e-4


def test_star_subset_in_a_batch():
    c = _star_case(scale=2, kb=5, H=16, W=15)
    full = Case(synth.custom(U=3, V=3, H=12, W=12, scale=2, kb=5, blur_sigma=1.2, window=5,
                             disparities=(-0.5, 0.8)), seed=3)
    kws = []
    for cc in (c, full):
        kws.append(dict(U=cc.wl.U, V=cc.wl.V, H=cc.wl.H, W=cc.wl.W, scale=cc.wl.scale,
                        blur=cc.blur, disparity=cc.disp, views=cc.views, **{
                            k: v for k, v in dict(lambda1=cc.wl.lambda1, lambda2=cc.wl.lambda2,
                                                  mu=cc.wl.mu, nltv_window=cc.wl.window,
                                                  nltv_patch=cc.wl.patch, nltv_h=cc.wl.h,
                                                  cg_iters=cc.wl.cg_iters).items()}))
    b = lfsr.Batch(kws)
    for j, cc in enumerate((c, full)):
        b.load(j, cc.t(cc.y), cc.t(cc.x0))
    b.iterate(6)
    for j, cc in enumerate((c, full)):
        x = cc.empty(*cc.oracle.hr)
        b.get_x(j, x)
        ref, _, _ = cc.oracle.admm(cc.y.astype(np.float64), cc.x0.astype(np.float64), 6)
        assert rel_err(cc.np(x), ref) <= 1e-4, j
    b.close()

"""lfsr_apply_normal_noalloc -- the allocation-free variant of the x-step
normal-matrix product, for callers that cannot allocate device memory.

Checked through the C ABI against the FP64 oracle's normal matrix and
against lfsr_apply_normal (the handle-based entry point) on two calls in a
row, within the tolerance of the normal-matrix parity test, on the
specialised operator kernel, the generic one (a non-separable blur, and a
(scale, blur size) pair without a specialised kernel) and a view subset.
This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

from paper_2206_05047_gb300 import lfsr, synth
from tests.gpu_util import Case, f32, max_err

pytestmark = pytest.mark.gpu


def _kw(c):
    wl, p = c.wl, c.params
    return dict(U=wl.U, V=wl.V, H=wl.H, W=wl.W, scale=wl.scale, blur=c.blur,
                disparity=c.disp, lambda1=p["lambda1"], lambda2=p["lambda2"], mu=p["mu"],
                nltv_window=p["window"], nltv_patch=p["patch"], nltv_h=p["h"], views=c.views)


def _oracle_q(c, xw, p):
    o = c.oracle
    return o.normal_apply(o.weights(xw.astype(np.float64)), p.astype(np.float64))


def _nonseparable(kb, seed):
    k = np.random.default_rng(seed).random((kb, kb)) + 0.05
    return k / k.sum()


CASES = {
    # specialised kernel: (scale, blur size) = (2, 5) and (3, 7)
    "fast_x2_k5": (synth.custom(U=5, V=5, H=21, W=19, scale=2, kb=5, blur_sigma=1.0, window=5),
                   {}),
    "fast_x3_k7": (synth.custom(U=3, V=5, H=13, W=11, scale=3, kb=7, blur_sigma=1.3, window=3,
                                patch=1, disparities=(-2.3, 0.4, 1.7)), {}),
    # generic kernel: a non-separable blur, and scale 3 with a 3 x 3 blur
    "generic_nonsep": (synth.custom(U=3, V=3, H=17, W=15, scale=2, kb=5, blur_sigma=1.0,
                                    window=5), {"blur": _nonseparable(5, 3)}),
    "generic_x3_k3": (synth.custom(U=3, V=3, H=11, W=13, scale=3, kb=3, blur_sigma=0.8,
                                   window=3), {}),
    # a view subset: the star of a 5 x 5 grid
    "views_star": (synth.custom(U=5, V=5, H=16, W=18, scale=2, kb=5, blur_sigma=1.0, window=5),
                   {"views": synth.star_views(5, 5)}),
}


@pytest.mark.parametrize("name", list(CASES))
def test_noalloc_matches_oracle_and_handle_entry_point_twice(name):
    wl, kw = CASES[name]
    c = Case(wl, seed=6, **kw)
    rng = np.random.default_rng(11)
    d_disp = c.t(c.disp)
    xw = c.t(c.x0)
    for call in range(2):           # two calls in a row share the scratch
        p = f32(rng.standard_normal(c.oracle.hr))
        ref = _oracle_q(c, c.x0, p)
        ref_pMp = float(np.vdot(p.astype(np.float64), ref))
        q_ref = c.empty(*c.oracle.hr)
        pMp_ref = lfsr.apply_normal(c.h, xw, c.t(p), q_ref)
        q = c.empty(*c.oracle.hr)
        pMp = lfsr.apply_normal_noalloc(d_disparity=d_disp, xw=xw, p=c.t(p), q=q, **_kw(c))
        assert max_err(c.np(q), ref) <= 5e-6, call
        assert abs(pMp - ref_pMp) <= 2e-6 * abs(ref_pMp), call
        assert max_err(c.np(q), c.np(q_ref)) <= 5e-6, call
        assert abs(pMp - pMp_ref) <= 2e-6 * abs(pMp_ref), call
    c.solver.close()


def test_noalloc_device_map_larger_than_host_map():
    """The kernels warp by the device map: a device map with larger shifts
    than the host map must give the product of the device map (the warp halo
    is sized over both), not read outside the staged tile."""
    wl = synth.custom(U=5, V=5, H=20, W=18, scale=2, kb=5, blur_sigma=1.0, window=5,
                      disparities=(-0.5, 0.0, 0.4))
    small = Case(wl, seed=2)
    big_map = f32(small.disp * 3.0 + 0.7)
    big = Case(wl, seed=2, disparity=big_map)
    rng = np.random.default_rng(5)
    p = f32(rng.standard_normal(big.oracle.hr))
    ref = _oracle_q(big, big.x0, p)
    q = big.empty(*big.oracle.hr)
    kw = _kw(small)                  # host map: the small one
    lfsr.apply_normal_noalloc(d_disparity=big.t(big_map), xw=big.t(big.x0), p=big.t(p), q=q, **kw)
    assert max_err(big.np(q), ref) <= 5e-6
    small.solver.close()
    big.solver.close()


def test_noalloc_rejects_non_finite_device_map():
    import torch
    wl = synth.custom(U=3, V=3, H=12, W=10, scale=2, kb=5, blur_sigma=1.0, window=3)
    c = Case(wl, seed=1)
    for bad in (np.nan, np.inf):
        m = c.disp.copy()
        m[3, 4] = bad
        q = c.empty(*c.oracle.hr)
        with pytest.raises(lfsr.LfsrError) as e:
            lfsr.apply_normal_noalloc(d_disparity=c.t(m), xw=c.t(c.x0), p=c.t(c.x0), q=q,
                                      **_kw(c))
        assert e.value.code == lfsr.LFSR_EINVAL
        assert "non-finite" in lfsr.last_error(None)
    torch.cuda.synchronize()
    c.solver.close()


def test_noalloc_rejects_sizes_beyond_the_scratch():
    import torch
    H = W = 1040                      # HR 2080 x 2080: 65 x 65 = 4225 tiles > 4096
    blur = np.ones((3, 3), np.float32) / 9
    disp = np.zeros((2 * H, 2 * W), np.float32)
    t = torch.zeros(2 * H * 2 * W, dtype=torch.float32, device="cuda:0")
    q = torch.zeros_like(t)
    with pytest.raises(lfsr.LfsrError) as e:
        lfsr.apply_normal_noalloc(3, 3, H, W, 2, blur, disp, t, t, t, q)
    assert e.value.code == lfsr.LFSR_EINVAL
    assert "too large" in lfsr.last_error(None)

"""lfsr_apply_normal_noalloc -- the allocation-free variant of the x-step
normal-matrix product, for callers that cannot allocate device memory.

Checked through the C ABI against lfsr_apply_normal (the handle-based entry
point) on two calls in a row, within the tolerance of the normal-matrix
parity test.  This file is collected last so that a run stopping at the
first failure has already run every other test; it also passes alone in a
fresh process.
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
                nltv_window=p["window"], nltv_patch=p["patch"], nltv_h=p["h"])


@pytest.mark.parametrize("wl", [
    synth.custom(U=5, V=5, H=21, W=19, scale=2, kb=5, blur_sigma=1.0, window=5),
    synth.custom(U=3, V=5, H=13, W=11, scale=3, kb=7, blur_sigma=1.3, window=3, patch=1,
                 disparities=(-2.3, 0.4, 1.7)),
])
def test_noalloc_matches_handle_entry_point_twice(wl):
    c = Case(wl, seed=6)
    o = c.oracle
    rng = np.random.default_rng(11)
    d_disp = c.t(c.disp)
    xw = c.t(c.x0)
    for call in range(2):           # two calls in a row share the scratch
        p = f32(rng.standard_normal(o.hr))
        q_ref = c.empty(*o.hr)
        pMp_ref = lfsr.apply_normal(c.h, xw, c.t(p), q_ref)
        q = c.empty(*o.hr)
        pMp = lfsr.apply_normal_noalloc(d_disparity=d_disp, xw=xw, p=c.t(p), q=q, **_kw(c))
        assert max_err(c.np(q), c.np(q_ref)) <= 5e-6, call
        assert abs(pMp - pMp_ref) <= 2e-6 * abs(pMp_ref), call
    c.solver.close()


def test_noalloc_rejects_sizes_beyond_the_scratch():
    import torch
    H = W = 1040                      # HR 2080 x 2080: 65 x 65 = 4225 tiles > 4096
    blur = np.ones((3, 3), np.float32) / 9
    disp = np.zeros((2 * H, 2 * W), np.float32)
    t = torch.zeros(8, dtype=torch.float32, device="cuda:0")
    with pytest.raises(lfsr.LfsrError) as e:
        lfsr.apply_normal_noalloc(3, 3, H, W, 2, blur, disp, t, t, t, t)
    assert e.value.code == lfsr.LFSR_EINVAL
    assert "too large" in lfsr.last_error(None)

"""Edge cases at the limits of the parameters on the CUDA path, against the
FP64 oracle: the largest angular grid (17 x 17 = 289 views), the largest
blur (15 x 15), the largest NLTV window and patch (15, 7), LR images of one
pixel, one row and one column, and zero iterations.

Tolerances as in test_gpu_parity.py (operators max-abs <= 2e-6 of the
output's max, one iteration rel-L2 <= 2e-5, solves rel-L2 <= 1e-4)."""
import numpy as np
import pytest

from paper_2206_05047_gb300 import lfsr, synth
from tests.gpu_util import Case, f32, max_err, rel_err

pytestmark = pytest.mark.gpu

LIMITS = {
    # 289 views, 15 x 15 blur, 15 x 15 window with 7 x 7 patches (generic kernels)
    "views289_kb15_win15": dict(U=17, V=17, H=6, W=7, scale=2, kb=15, blur_sigma=2.5,
                                window=15, patch=7, disparities=(-0.5, 0.4)),
    # one LR pixel, x4
    "lr1x1_x4": dict(U=3, V=3, H=1, W=1, scale=4, kb=5, blur_sigma=1.0, window=3,
                     disparities=(-0.3, 0.2)),
    # one HR pixel: every NLTV edge leaves the image
    "hr1x1": dict(U=3, V=3, H=1, W=1, scale=1, kb=3, blur_sigma=0.7, window=3,
                  disparities=(0.0, 0.4)),
    # one LR row and one LR column
    "row1x40": dict(U=5, V=3, H=1, W=40, scale=2, kb=5, blur_sigma=1.0, window=5,
                    disparities=(-1.0, 0.7)),
    "col37x1": dict(U=3, V=5, H=37, W=1, scale=3, kb=7, blur_sigma=1.3, window=7,
                    disparities=(-0.8, 1.1)),
}


def _case(name, seed=0):
    return Case(synth.custom(**LIMITS[name]), seed=seed)


@pytest.mark.parametrize("name", list(LIMITS))
def test_operators_at_the_limits(name):
    c = _case(name)
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
    w = c.empty(o.s_d, *o.hr)
    lfsr.weights(c.h, c.t(x), w)
    assert np.abs(c.np(w) - o.weights(x.astype(np.float64))).max() <= 3e-5


@pytest.mark.parametrize("name", list(LIMITS))
def test_solve_at_the_limits(name):
    c = _case(name)
    o = c.oracle
    n_iter = 4
    x = c.empty(*o.hr)
    lfsr.solve(c.h, c.t(c.y), n_iter, c.t(c.x0), x)
    ref, _, _ = o.admm(c.y.astype(np.float64), c.x0.astype(np.float64), n_iter)
    assert rel_err(c.np(x), ref) <= 1e-4
    st = lfsr.stats(c.h)
    assert st["status"] == 0 and st["iterations"] == n_iter


def test_single_hr_pixel_has_no_regulariser_edges():
    c = _case("hr1x1")
    o = c.oracle
    w = c.empty(o.s_d, *o.hr)
    lfsr.weights(c.h, c.t(c.x0), w)
    assert not c.np(w).any()


def test_zero_iterations_return_x0_exactly():
    c = _case("row1x40")
    x = c.empty(*c.oracle.hr)
    lfsr.solve(c.h, c.t(c.y), 0, c.t(c.x0), x)
    assert np.array_equal(c.np(x), c.x0.astype(np.float64))
    assert lfsr.stats(c.h)["iterations"] == 0


def test_non_finite_start_is_reported_and_a_clean_load_recovers():
    """A NaN in x0 makes the CG curvature non-finite: the solve returns
    LFSR_ENUMERIC; the next load clears the status."""
    c = _case("row1x40")
    x0 = c.x0.copy()
    x0[0, 3] = np.nan
    x = c.empty(*c.oracle.hr)
    with pytest.raises(lfsr.LfsrError) as e:
        lfsr.solve(c.h, c.t(c.y), 2, c.t(x0), x)
    assert e.value.code == lfsr.LFSR_ENUMERIC
    lfsr.solve(c.h, c.t(c.y), 2, c.t(c.x0), x)
    assert np.isfinite(c.np(x)).all() and lfsr.stats(c.h)["status"] == 0

"""The seeded input generator: determinism, shapes and the noise recipe."""
import numpy as np

from paper_2206_05047_gb300 import synth


def test_deterministic_and_shapes():
    wl = synth.custom(U=3, V=5, H=9, W=7, scale=3, kb=5, blur_sigma=1.0)
    a = synth.make_problem(wl, seed=5)
    b = synth.make_problem(wl, seed=5)
    c = synth.make_problem(wl, seed=6)
    for name in ("y", "x0", "gt", "disparity", "blur"):
        assert np.array_equal(getattr(a, name), getattr(b, name))
    assert not np.array_equal(a.y, c.y)
    assert a.y.shape == (15, 9, 7)
    assert a.x0.shape == a.gt.shape == a.disparity.shape == (27, 21)
    assert set(np.unique(a.disparity)) <= set(wl.disparities)
    assert abs(a.blur.sum() - 1.0) < 1e-15 and a.blur.shape == (5, 5)
    np.testing.assert_array_equal(a.theta[7], [0.0, 0.0])   # centre view of 3x5


def test_impulse_fraction_and_range():
    wl = synth.custom(U=3, V=3, H=64, W=64, impulse=0.2, noise_sigma=0.0)
    p = synth.make_problem(wl, seed=1)
    clean = synth.make_problem(wl, seed=1, noise=False)
    hit = p.y != clean.y
    assert abs(hit.mean() - 0.2 * 1.0) < 0.02      # replaced pixels (0 or 1)
    assert set(np.unique(p.y[hit])) <= {0.0, 1.0}
    assert 0.0 <= clean.y.min() and clean.y.max() <= 1.0


def test_bicubic_interpolates_lr_samples():
    rng = np.random.default_rng(0)
    lr = rng.random((6, 5))
    hr = synth.bicubic_upsample(lr, 2)
    np.testing.assert_allclose(hr[::2, ::2], lr, atol=1e-15)


def test_degenerate_shapes_generate():
    """One LR pixel, one row, one column: the scene generator still places
    its planes (discs wider than the image are centred on that axis)."""
    for kw in (dict(H=1, W=1, scale=4), dict(H=1, W=40, scale=2), dict(H=37, W=1, scale=3)):
        wl = synth.custom(U=3, V=3, kb=5, blur_sigma=1.0, disparities=(-1.0, 0.0, 0.7), **kw)
        pr = synth.make_problem(wl, seed=0)
        assert pr.y.shape == (9, wl.H, wl.W) and pr.gt.shape == wl.HR
        assert np.isfinite(pr.y).all() and np.isfinite(pr.x0).all()


def test_view_disparity_maps_match_the_rendered_planes():
    wl = synth.custom(U=5, V=3, H=10, W=12, scale=2, disparities=(-1.0, 0.0, 0.8))
    pr = synth.make_problem(wl, seed=3)
    maps = synth.view_disparity_maps(pr)
    assert maps.shape == (wl.s_k,) + wl.HR
    assert np.array_equal(maps[wl.s_k // 2], pr.disparity)        # centre view = reference
    assert set(np.unique(maps)) <= set(wl.disparities)
    sub = synth.view_disparity_maps(pr, views=[0, 7, 14])
    assert np.array_equal(sub, maps[[0, 7, 14]])

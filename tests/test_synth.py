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

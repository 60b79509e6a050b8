"""Pins of the oracle's warp variants (Sec. 4.1): per-view disparity maps
omega_k for W_k, and the paper's backward warp W_k^* by the reference map
in place of the exact adjoint.  Checked against exact shifts, the adjoint
identity, the interior identity W_k^* = W_k^T for a constant disparity, and
the rendering of the synthetic scene."""
import numpy as np
import pytest

from paper_2206_05047_gb300 import synth


def _oracle(oracle_mod, U=3, V=3, H=7, W=8, zeta=2, disp=None, **kw):
    rng = np.random.default_rng(0)
    d = rng.uniform(-1.5, 1.5, (zeta * H, zeta * W)) if disp is None else disp
    return oracle_mod.Oracle(U, V, H, W, zeta, synth.gaussian_blur_kernel(3, 0.8), d, **kw)


def test_per_view_maps_equal_to_the_shared_map_change_nothing(oracle_mod):
    rng = np.random.default_rng(1)
    a = _oracle(oracle_mod)
    b = _oracle(oracle_mod, disparity_views=np.repeat(a.disp[None], a.s_k, axis=0))
    x = rng.random(a.hr)
    g = rng.standard_normal((a.H, a.W))
    for k in (0, 4, 8):
        assert np.array_equal(a.warp(k, x), b.warp(k, x))
        assert np.array_equal(a.A_T(k, g), b.A_T(k, g))
    y = rng.random((a.s_k, a.H, a.W))
    xa, _, _ = a.admm(y, x, 2)
    xb, _, _ = b.admm(y, x, 2)
    assert np.array_equal(xa, xb)


def test_per_view_integer_maps_are_exact_shifts(oracle_mod):
    """omega_k = c_k (integer) with a zero reference map: W_k x (z) =
    x(z + theta_k c_k), zero where that leaves the image."""
    rng = np.random.default_rng(2)
    o0 = _oracle(oracle_mod, disp=np.zeros((14, 16)))
    c = rng.integers(-2, 3, o0.s_k)
    maps = np.stack([np.full(o0.hr, float(ck)) for ck in c])
    o = _oracle(oracle_mod, disp=np.zeros((14, 16)), disparity_views=maps)
    x = rng.random(o.hr)
    Hh, Wh = o.hr
    offs = synth.view_offsets(3, 3)
    for k in range(o.s_k):
        si, sj = int(offs[k][1] * c[k]), int(offs[k][0] * c[k])
        ref = np.zeros(o.hr)
        for i in range(Hh):
            for j in range(Wh):
                if 0 <= i + si < Hh and 0 <= j + sj < Wh:
                    ref[i, j] = x[i + si, j + sj]
        assert np.array_equal(o.warp(k, x), ref)


def test_per_view_maps_keep_the_exact_adjoint(oracle_mod):
    rng = np.random.default_rng(3)
    maps = rng.uniform(-1.7, 1.7, (9, 14, 16))
    o = _oracle(oracle_mod, disparity_views=maps)
    for k in (0, 3, 8):
        x = rng.standard_normal(o.hr)
        g = rng.standard_normal(o.hr)
        lhs = float(np.vdot(o.warp(k, x), g))
        rhs = float(np.vdot(x, o.warp_T(k, g)))
        assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + 1.0)


@pytest.mark.parametrize("c", [1.0, -0.35, 0.6])
def test_backward_warp_is_the_adjoint_for_a_constant_disparity(oracle_mod, c):
    """For omega = c everywhere, bilinear sampling at u - theta c uses the
    taps and weights of the scatter from u - theta c: W_k^* = W_k^T on every
    pixel whose taps stay inside the image (all pixels for an integer
    shift)."""
    rng = np.random.default_rng(4)
    o = _oracle(oracle_mod, disp=np.full((14, 16), c))
    Hh, Wh = o.hr
    g = rng.standard_normal(o.hr)
    offs = synth.view_offsets(3, 3)
    for k in range(o.s_k):
        a, b = o.warp_bw(k, g), o.warp_T(k, g)
        m = int(np.ceil(abs(c) * np.abs(offs[k]).max())) + 1
        if float(c).is_integer():
            assert np.array_equal(a, b)
        else:
            assert np.allclose(a[m:Hh - m, m:Wh - m], b[m:Hh - m, m:Wh - m], rtol=0, atol=1e-14)


def test_backward_warp_is_not_the_adjoint_where_disparity_varies(oracle_mod):
    o = _oracle(oracle_mod)           # random disparity
    rng = np.random.default_rng(5)
    x = rng.standard_normal(o.hr)
    g = rng.standard_normal(o.hr)
    lhs = float(np.vdot(o.warp(0, x), g))
    assert abs(lhs - float(np.vdot(x, o.warp_bw(0, g)))) > 1e-3 * abs(lhs)


def test_backward_warp_admm_equals_exact_for_an_integer_disparity(oracle_mod):
    """With W_k^* = W_k^T (integer constant disparity) the two x-steps are the
    same operator, so the whole ADMM agrees."""
    rng = np.random.default_rng(6)
    a = _oracle(oracle_mod, disp=np.full((14, 16), 1.0), lambda1=2.0, lambda2=4.0, mu=3.0)
    b = _oracle(oracle_mod, disp=np.full((14, 16), 1.0), lambda1=2.0, lambda2=4.0, mu=3.0,
                adjoint="backward")
    y = rng.random((9, 7, 8))
    x0 = rng.random(a.hr)
    xa, wAa, _ = a.admm(y, x0, 3)
    xb, wAb, _ = b.admm(y, x0, 3)
    np.testing.assert_allclose(xb, xa, rtol=0, atol=1e-13)
    np.testing.assert_allclose(wAb, wAa, rtol=0, atol=1e-13)


def test_per_view_maps_reproduce_the_rendered_views(oracle_mod):
    """Integer disparities and angular offsets make every warp an exact
    shift.  Rendered without a PSF, view k at z shows the reference point
    u = z + theta_k omega_k(z); wherever the reference also sees that plane
    at u (no disocclusion), W_k gt(z) with the per-view maps equals the
    render exactly.  The reference map alone misses some of those pixels
    (where omega_0(z) is another plane's disparity)."""
    from paper_2206_05047_gb300.synth import _render
    wl = synth.custom(U=5, V=5, H=20, W=20, scale=2, kb=5, blur_sigma=1.0,
                      disparities=(-1.0, 0.0, 1.0), noise_sigma=0.0, impulse=0.0)
    pr = synth.make_problem(wl, seed=8, noise=False)
    maps = synth.view_disparity_maps(pr)
    assert np.array_equal(maps[wl.s_k // 2], pr.disparity)
    shared = oracle_mod.Oracle.from_problem(pr)
    per_view = oracle_mod.Oracle.from_problem(pr, disparity_views=maps)
    Hh, Wh = wl.HR
    Yg, Xg = np.meshgrid(np.arange(Hh, dtype=float), np.arange(Wh, dtype=float), indexing="ij")
    shared_misses = 0
    for k in range(wl.s_k):
        tu, tv = pr.theta[k]
        render = _render(pr.planes, Yg, Xg, tu, tv)[0]
        ui = (Yg + tv * maps[k]).astype(int)
        uj = (Xg + tu * maps[k]).astype(int)
        inside = (ui >= 0) & (ui < Hh) & (uj >= 0) & (uj < Wh)
        seen = np.zeros_like(inside)
        seen[inside] = pr.disparity[ui[inside], uj[inside]] == maps[k][inside]
        assert np.array_equal(per_view.warp(k, pr.gt)[seen], render[seen])
        shared_misses += int((shared.warp(k, pr.gt)[seen] != render[seen]).sum())
    assert shared_misses > 0

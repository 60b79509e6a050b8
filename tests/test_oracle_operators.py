"""Pins of the FP64 oracle's operators against mathematics, not against itself.

Adjoint identities, library routines (scipy.ndimage), exact special cases
(integer shifts, linear ramps, step edges) and closed forms.
"""
import math

import numpy as np
import pytest
import scipy.ndimage as ndi

from paper_2206_05047_gb300 import synth


def _oracle(oracle_mod, U=3, V=3, H=7, W=5, zeta=2, kb=3, blur=None, disp=None, seed=0, **kw):
    rng = np.random.default_rng(seed)
    hr = (zeta * H, zeta * W)
    if blur is None:
        blur = synth.gaussian_blur_kernel(kb, 0.9)
    if disp is None:
        disp = rng.uniform(-1.7, 1.3, size=hr)
    return oracle_mod.Oracle(U, V, H, W, zeta, blur, disp, **kw), rng


def _adj_err(Ax, y, x, ATy):
    lhs = float(np.vdot(Ax, y))
    rhs = float(np.vdot(x, ATy))
    return abs(lhs - rhs) / (np.linalg.norm(Ax) * np.linalg.norm(y) + 1e-300)


@pytest.mark.parametrize("zeta,H,W", [(2, 7, 5), (3, 4, 6), (1, 9, 9)])
def test_adjoint_identities(oracle_mod, zeta, H, W):
    """<Ax, y> = <x, A^T y> for W_k, B, D, A_k, S (Sec. 4.1 operator pairs)."""
    kb = 5
    rng0 = np.random.default_rng(7)
    blur_ns = rng0.random((kb, kb))            # non-symmetric kernel (motion-blur case)
    for blur in (synth.gaussian_blur_kernel(kb, 1.1), blur_ns):
        o, rng = _oracle(oracle_mod, U=3, V=5, H=H, W=W, zeta=zeta, blur=blur, window=5)
        x = rng.standard_normal(o.hr)
        g_hr = rng.standard_normal(o.hr)
        g_lr = rng.standard_normal((H, W))
        for k in range(o.s_k):
            assert _adj_err(o.warp(k, x), g_hr, x, o.warp_T(k, g_hr)) < 1e-12
            assert _adj_err(o.A(k, x), g_lr, x, o.A_T(k, g_lr)) < 1e-12
        assert _adj_err(o.blur_op(x), g_hr, x, o.blur_T(g_hr)) < 1e-12
        assert _adj_err(o.down(x), g_lr, x, o.up(g_lr)) < 1e-12
        w = rng.random((o.s_d,) + o.hr)
        gS = rng.standard_normal((o.s_d,) + o.hr)
        assert _adj_err(o.S(w, x), gS, x, o.S_T(w, gS)) < 1e-12


def test_blur_is_scipy_correlate(oracle_mod):
    """B equals scipy.ndimage.correlate with zero padding (textbook routine)."""
    rng = np.random.default_rng(1)
    K = rng.random((5, 5))
    o, _ = _oracle(oracle_mod, H=6, W=8, zeta=2, blur=K)
    x = rng.standard_normal(o.hr)
    ref = ndi.correlate(x, K, mode="constant", cval=0.0)
    np.testing.assert_allclose(o.blur_op(x), ref, rtol=0, atol=1e-13)
    # B^T is correlation with the flipped kernel
    ref_t = ndi.correlate(x, K[::-1, ::-1], mode="constant", cval=0.0)
    np.testing.assert_allclose(o.blur_T(x), ref_t, rtol=0, atol=1e-13)


def test_down_up_pick_top_left(oracle_mod):
    o, rng = _oracle(oracle_mod, H=5, W=4, zeta=3)
    x = rng.standard_normal(o.hr)
    assert np.array_equal(o.down(x), x[::3, ::3])
    g = rng.standard_normal((5, 4))
    up = o.up(g)
    assert np.array_equal(up[::3, ::3], g)
    up[::3, ::3] = 0
    assert not up.any()


def test_warp_integer_shift_is_exact(oracle_mod):
    """Integer disparity * theta gives an exact shift with zero fill."""
    H, W, zeta = 6, 7, 2
    disp = np.full((zeta * H, zeta * W), 1.0)
    o, rng = _oracle(oracle_mod, U=3, V=5, H=H, W=W, zeta=zeta, disp=disp)
    x = rng.standard_normal(o.hr)
    Hh, Wh = o.hr
    for k in range(o.s_k):
        u, v = k % 3, k // 3
        tu, tv = u - 1, v - 2
        ref = np.zeros_like(x)
        for i in range(Hh):
            for j in range(Wh):
                si, sj = i + tv, j + tu
                if 0 <= si < Hh and 0 <= sj < Wh:
                    ref[i, j] = x[si, sj]
        assert np.array_equal(o.warp(k, x), ref), k


def test_warp_reproduces_linear_ramp(oracle_mod):
    """Bilinear sampling is exact on an affine image (taps inside the image)."""
    H, W, zeta = 10, 10, 2
    rng = np.random.default_rng(3)
    disp = rng.uniform(-0.9, 0.9, (zeta * H, zeta * W))
    o, _ = _oracle(oracle_mod, U=3, V=3, H=H, W=W, zeta=zeta, disp=disp)
    ii, jj = np.meshgrid(np.arange(2 * H, dtype=float), np.arange(2 * W, dtype=float), indexing="ij")
    a, b, c = 0.37, -1.21, 0.5
    x = a * ii + b * jj + c
    for k in range(o.s_k):
        tu, tv = (k % 3) - 1, (k // 3) - 1
        ref = a * (ii + tv * disp) + b * (jj + tu * disp) + c
        out = o.warp(k, x)
        inner = (slice(2, -2), slice(2, -2))
        np.testing.assert_allclose(out[inner], ref[inner], rtol=0, atol=1e-12)


def test_blur_preserves_constant_interior(oracle_mod):
    o, _ = _oracle(oracle_mod, H=8, W=8, zeta=2, kb=5)
    x = np.full(o.hr, 0.625)
    out = o.blur_op(x)
    np.testing.assert_allclose(out[2:-2, 2:-2], 0.625, rtol=0, atol=1e-15)


def test_prox_closed_form(oracle_mod):
    """Soft threshold (Eq. sr_l1l2l1_prox) on hand-picked values, and the
    identity u - prox(u) = clamp(u, -t, t) up to one rounding."""
    o, rng = _oracle(oracle_mod)
    t = 0.5
    u = np.array([2.0, -2.0, 0.25, -0.25, 0.0, 0.5, -0.5, 0.75])
    np.testing.assert_array_equal(o.prox(u, t), [1.5, -1.5, 0, 0, 0, 0, 0, 0.25])
    u = rng.standard_normal(10000) * 3
    w = u - o.prox(u, t)
    np.testing.assert_allclose(w, np.clip(u, -t, t), rtol=0, atol=4 * np.finfo(float).eps * 10)


def test_weights_constant_image(oracle_mod):
    o, _ = _oracle(oracle_mod, H=6, W=5, zeta=2, window=5)
    w = o.weights(np.full(o.hr, 0.3))
    di, dj = o.dirs()
    Hh, Wh = o.hr
    for d in range(o.s_d):
        for i in range(Hh):
            for j in range(Wh):
                inside = 0 <= i + di[d] < Hh and 0 <= j + dj[d] < Wh
                assert w[d, i, j] == (1.0 if inside else 0.0)


def test_weights_symmetry_and_direction_order(oracle_mod):
    """w_d(u) = w_{-d}(u+d) exactly; directions: window minus centre, raster order."""
    o, rng = _oracle(oracle_mod, H=6, W=7, zeta=2, window=5)
    di, dj = o.dirs()
    assert o.s_d == 24
    assert list(zip(di[:3], dj[:3])) == [(-2, -2), (-2, -1), (-2, 0)]
    assert (0, 0) not in list(zip(di, dj))
    x = rng.random(o.hr)
    w = o.weights(x)
    Hh, Wh = o.hr
    for d in range(o.s_d):
        m = o.s_d - 1 - d
        assert di[m] == -di[d] and dj[m] == -dj[d]
        for i in range(Hh):
            for j in range(Wh):
                ni, nj = i + di[d], j + dj[d]
                if 0 <= ni < Hh and 0 <= nj < Wh:
                    assert w[d, i, j] == w[m, ni, nj]


def test_weights_match_library_patch_filter(oracle_mod):
    """Patch distance via edge padding + scipy uniform_filter (mean) matches."""
    o, rng = _oracle(oracle_mod, H=7, W=6, zeta=2, window=7, patch=3, h=0.2)
    x = rng.random(o.hr)
    w = o.weights(x)
    di, dj = o.dirs()
    Hh, Wh = o.hr
    R = 4  # window radius 3 + patch radius 1
    X = np.pad(x, R, mode="edge")
    for d in range(o.s_d):
        shifted = X[R + di[d] - 1:R + di[d] + Hh + 1, R + dj[d] - 1:R + dj[d] + Wh + 1]
        base = X[R - 1:R + Hh + 1, R - 1:R + Wh + 1]
        pd = ndi.uniform_filter((base - shifted) ** 2, size=3, mode="constant")[1:-1, 1:-1]
        ref = np.exp(-pd / 0.04)
        ii, jj = np.meshgrid(np.arange(Hh), np.arange(Wh), indexing="ij")
        inside = (ii + di[d] >= 0) & (ii + di[d] < Hh) & (jj + dj[d] >= 0) & (jj + dj[d] < Wh)
        ref = np.where(inside, ref, 0.0)
        np.testing.assert_allclose(w[d], ref, rtol=1e-13, atol=1e-15)


def test_weights_step_edge_closed_form(oracle_mod):
    """Across a vertical unit step, a 3x3 patch pair one column apart differs
    in exactly one column: pd = 3/9, w = exp(-1/(3 h^2))."""
    o, _ = _oracle(oracle_mod, H=5, W=6, zeta=2, window=3, patch=3, h=0.5)
    Hh, Wh = o.hr
    x = np.zeros(o.hr)
    c = 6
    x[:, c:] = 1.0
    w = o.weights(x)
    di, dj = o.dirs()
    d = [n for n in range(o.s_d) if di[n] == 0 and dj[n] == 1][0]
    assert math.isclose(w[d, 4, c - 1], math.exp(-(3 / 9) / 0.25), rel_tol=1e-15)
    # far from the edge the patches agree
    assert w[d, 4, 1] == 1.0


def test_normal_matrix_closed_form(oracle_mod):
    """M p equals G^T G p with G = [sqrt(l2) A; sqrt(mu/2) F], F = [l1 A; S],
    assembled as a dense matrix from operator columns (alpha_i = lambda_i)."""
    o, rng = _oracle(oracle_mod, U=3, V=3, H=3, W=4, zeta=2, lambda1=0.7, lambda2=2.5,
                     mu=1.9, window=3)
    p = o.p
    w = rng.random((o.s_d,) + o.hr)
    cols_A, cols_S = [], []
    for n in range(p):
        e = np.zeros(p); e[n] = 1.0
        e = e.reshape(o.hr)
        cols_A.append(np.concatenate([o.A(k, e).ravel() for k in range(o.s_k)]))
        cols_S.append(o.S(w, e).ravel())
    Ad = np.array(cols_A).T
    Sd = np.array(cols_S).T
    l1, l2, mu = 0.7, 2.5, 1.9
    G = np.vstack([math.sqrt(l2) * Ad, math.sqrt(mu / 2) * l1 * Ad, math.sqrt(mu / 2) * Sd])
    M = G.T @ G
    for _ in range(3):
        v = rng.standard_normal(o.hr)
        np.testing.assert_allclose(o.normal_apply(w, v).ravel(), M @ v.ravel(), rtol=1e-12,
                                   atol=1e-12 * np.abs(M).max())


def test_cg_full_steps_equals_dense_solve(oracle_mod):
    """Algorithm 2 with K = p steps solves M delta = -v exactly (dense solve)."""
    o, rng = _oracle(oracle_mod, U=3, V=3, H=4, W=4, zeta=2, window=3, lambda2=3.0)
    w = rng.random((o.s_d,) + o.hr) * 0.8 + 0.2
    p = o.p
    M = np.zeros((p, p))
    for n in range(p):
        e = np.zeros(p); e[n] = 1.0
        M[:, n] = o.normal_apply(w, e.reshape(o.hr)).ravel()
    np.testing.assert_allclose(M, M.T, rtol=0, atol=1e-12 * np.abs(M).max())
    assert np.linalg.eigvalsh(M).min() > 0
    v = rng.standard_normal(o.hr)
    x0 = rng.standard_normal(o.hr)
    x, steps, _ = o.cg(w, v, x0, K=4 * p, tau=1e-26)
    ref = x0.ravel() + np.linalg.solve(M, -v.ravel())
    assert np.linalg.norm(x.ravel() - ref) <= 1e-10 * np.linalg.norm(ref)


def test_cg_zero_rhs_takes_no_step(oracle_mod):
    o, rng = _oracle(oracle_mod)
    w = rng.random((o.s_d,) + o.hr)
    x0 = rng.standard_normal(o.hr)
    x, steps, pi = o.cg(w, np.zeros(o.hr), x0, K=5)
    assert steps == 0 and pi == 0.0 and np.array_equal(x, x0)


def test_star_subset_of_views():
    k = synth.star_views(5, 5)
    assert len(k) == 17 and 12 in k                       # centre view of 5 x 5
    assert set(24 - k) == set(k)                          # symmetric about the centre
    assert len(synth.star_views(9, 9)) == 33


def test_view_subset_operators_are_the_listed_views(oracle_mod):
    """A subset problem's view j is the full grid's view views[j]."""
    wl = synth.custom(U=5, V=5, H=8, W=9, scale=2, kb=3, disparities=(-1.3, 0.7))
    prob = synth.make_problem(wl, seed=3)
    full = oracle_mod.Oracle.from_problem(prob)
    ks = synth.star_views(5, 5)
    sub = oracle_mod.Oracle.from_problem(prob, views=ks)
    assert sub.s_k == 17
    x = np.random.default_rng(0).random(full.hr)
    g = np.random.default_rng(1).standard_normal((wl.H, wl.W))
    for j, k in enumerate(ks):
        assert np.array_equal(sub.A(j, x), full.A(int(k), x))
        assert np.array_equal(sub.A_T(j, g), full.A_T(int(k), g))


def test_single_view_subset_is_a_one_view_problem(oracle_mod):
    """The centre view alone (theta = 0) equals a 1 x 1 light field: the
    whole ADMM, not only the operators."""
    wl = synth.custom(U=3, V=3, H=10, W=10, scale=2, kb=3, disparities=(-1.0, 0.5))
    prob = synth.make_problem(wl, seed=5)
    sub = oracle_mod.Oracle.from_problem(prob, views=[4])
    one = oracle_mod.Oracle(1, 1, wl.H, wl.W, 2, prob.blur, prob.disparity, lambda1=wl.lambda1,
                            lambda2=wl.lambda2, mu=wl.mu, window=wl.window, patch=wl.patch,
                            h=wl.h, cg_iters=wl.cg_iters)
    y = prob.y[4:5]
    xs, _, _ = sub.admm(y, prob.x0, 4)
    xo, _, _ = one.admm(y, prob.x0, 4)
    assert np.array_equal(xs, xo)

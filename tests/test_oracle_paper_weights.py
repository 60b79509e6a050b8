"""Pins of the oracle's paper weights (Sec. 3.4 and Eq. weight_occ):
w_d(u) = w_s(d) e(u) o(u), spatial factor exp(-|d|^2/sigma_s), edge factor
exp(-|grad x|^2/sigma_e), occlusion factor from the disparity map's one-sided
divergence b and the projection error p.  Each factor is checked on inputs
where its value has a closed form: constant images, linear and quadratic
ramps (whose central differences are exact), disparity steps."""
import math

import numpy as np
import pytest

from paper_2206_05047_gb300 import synth


def _o(oracle_mod, H=6, W=7, zeta=1, disp=None, window=5, **kw):
    Hh, Wh = zeta * H, zeta * W
    d = np.zeros((Hh, Wh)) if disp is None else disp
    return oracle_mod.Oracle(3, 3, H, W, zeta, synth.gaussian_blur_kernel(3, 0.8), d,
                             window=window, weights="paper", **kw)


def _inside(o):
    """[d][u] = 1 where u + d lies in the image."""
    Hh, Wh = o.hr
    di, dj = o.dirs()
    m = np.zeros((o.s_d, Hh, Wh))
    for n in range(o.s_d):
        a, b = int(di[n]), int(dj[n])
        m[n, max(0, -a):min(Hh, Hh - a), max(0, -b):min(Wh, Wh - b)] = 1.0
    return m


def test_constant_image_flat_disparity_is_the_spatial_factor(oracle_mod):
    o = _o(oracle_mod, sigma_s=3.0, sigma_e=0.05, sigma_o1=0.5)
    w = o.weights(np.full(o.hr, 0.3))
    di, dj = o.dirs()
    for n in range(o.s_d):
        ws = math.exp(-(int(di[n]) ** 2 + int(dj[n]) ** 2) / 3.0)
        np.testing.assert_allclose(w[n], ws * _inside(o)[n], rtol=1e-15, atol=0)


def test_zero_sigmas_give_unit_factors(oracle_mod):
    rng = np.random.default_rng(1)
    o = _o(oracle_mod, disp=rng.uniform(-2, 2, (6, 7)), proj_err=rng.random((6, 7)))
    x = rng.random(o.hr)
    assert np.array_equal(o.weights(x), _inside(o))
    assert np.array_equal(o.edge_factor(x), np.ones(o.hr))
    assert np.array_equal(o.occlusion_factor(), np.ones(o.hr))


def test_edge_factor_of_a_linear_ramp(oracle_mod):
    """x = a i + b j: central differences give (a, b) inside, half of it
    where the clamped stencil folds (first / last row or column)."""
    a, b, se = 0.07, -0.03, 0.02
    o = _o(oracle_mod, sigma_e=se)
    Hh, Wh = o.hr
    I, J = np.mgrid[0:Hh, 0:Wh].astype(np.float64)
    e = o.edge_factor(a * I + b * J)
    gi = np.full(o.hr, a); gi[0, :] = gi[-1, :] = a / 2
    gj = np.full(o.hr, b); gj[:, 0] = gj[:, -1] = b / 2
    np.testing.assert_allclose(e, np.exp(-(gi ** 2 + gj ** 2) / se), rtol=1e-13)


def test_edge_factor_of_a_quadratic_is_the_derivative(oracle_mod):
    """x = c i^2: the central difference (x(i+1) - x(i-1)) / 2 = 2 c i
    exactly (a forward difference would give c (2 i + 1))."""
    c, se = 0.01, 0.03
    o = _o(oracle_mod, H=8, W=3, sigma_e=se)
    Hh, Wh = o.hr
    I = np.mgrid[0:Hh, 0:Wh][0].astype(np.float64)
    e = o.edge_factor(c * I ** 2)
    i = np.arange(1, Hh - 1)
    np.testing.assert_allclose(e[1:-1, 1], np.exp(-(2 * c * i) ** 2 / se), rtol=1e-13)


@pytest.mark.parametrize("axis", [0, 1])
def test_occlusion_factor_of_a_disparity_step(oracle_mod, axis):
    """A step from d_hi to d_lo along the axis: the forward difference is
    negative on the last pixel before the step only, so b = d_lo - d_hi there
    and o = exp(-b^2 / (2 sigma^2)); the opposite step (a disocclusion) has
    b = 0 and leaves o = 1 everywhere."""
    s1 = 0.7
    H, W, cut = 6, 7, 3
    for d_before, d_after, occluding in ((1.5, 0.25, True), (0.25, 1.5, False)):
        disp = np.full((H, W), d_before)
        if axis == 0:
            disp[cut:, :] = d_after
        else:
            disp[:, cut:] = d_after
        o = _o(oracle_mod, H=H, W=W, disp=disp, sigma_o1=s1)
        occ = o.occlusion_factor()
        ref = np.ones((H, W))
        if occluding:
            b = d_after - d_before
            if axis == 0:
                ref[cut - 1, :] = math.exp(-b * b / (2 * s1 * s1))
            else:
                ref[:, cut - 1] = math.exp(-b * b / (2 * s1 * s1))
        np.testing.assert_allclose(occ, ref, rtol=1e-15)


def test_occlusion_boundary_sums_both_components(oracle_mod):
    """A corner where omega drops by g_i down and by g_j right: b = g_i + g_j
    when the sum is negative, 0 when the components cancel."""
    s1 = 0.9
    disp = np.zeros((4, 4))
    disp[2, 1] = -0.6     # below (1, 1)
    disp[1, 2] = -0.5     # right of (1, 1)
    o = _o(oracle_mod, H=4, W=4, disp=disp, sigma_o1=s1)
    occ = o.occlusion_factor()
    assert occ[1, 1] == pytest.approx(math.exp(-1.1 ** 2 / (2 * s1 * s1)), rel=1e-14)
    disp[1, 2] = 0.6      # cancels
    o = _o(oracle_mod, H=4, W=4, disp=disp, sigma_o1=s1)
    assert o.occlusion_factor()[1, 1] == 1.0


def test_projection_error_factor(oracle_mod):
    rng = np.random.default_rng(3)
    pe = rng.standard_normal((6, 7))
    o = _o(oracle_mod, proj_err=pe, sigma_o2=0.8)
    np.testing.assert_allclose(o.occlusion_factor(), np.exp(-pe ** 2 / (2 * 0.64)), rtol=1e-14)


def test_weights_factorise_and_are_directed(oracle_mod):
    """w_d(u) / w_d'(u) = w_s(d) / w_s(d') at every pixel where both edges
    exist; w_d(u) and w_{-d}(u+d) differ by e(u) o(u) / (e(u+d) o(u+d))."""
    rng = np.random.default_rng(5)
    ss, se, so = 4.0, 0.05, 0.5
    o = _o(oracle_mod, H=9, W=8, disp=rng.uniform(-1, 1, (9, 8)), sigma_s=ss, sigma_e=se,
           sigma_o1=so)
    x = rng.random(o.hr)
    w = o.weights(x)
    di, dj = o.dirs()
    g = o.edge_factor(x) * o.occlusion_factor()
    Hh, Wh = o.hr
    for n in range(o.s_d):
        a, b = int(di[n]), int(dj[n])
        ws = math.exp(-(a * a + b * b) / ss)
        m = _inside(o)[n] > 0
        np.testing.assert_allclose(w[n][m], ws * g[m], rtol=1e-14)
        # the reverse edge: direction -d is index s_d - 1 - n in raster order
        r = o.s_d - 1 - n
        assert (int(di[r]), int(dj[r])) == (-a, -b)
        for i in range(max(0, -a), min(Hh, Hh - a)):
            for j in range(max(0, -b), min(Wh, Wh - b)):
                assert w[r][i + a, j + b] == pytest.approx(ws * g[i + a, j + b], rel=1e-14)
    assert not np.allclose(w[0][2:, 2:], w[o.s_d - 1][:-2, :-2])


def test_paper_weights_improve_quality_over_iterations(oracle_mod):
    """The quality trend of Sec. 6.1 with the paper's weights (sigma_s = 8,
    sigma_e = 0.1, sigma_o1 = 1)."""
    wl = synth.custom(U=5, V=5, H=24, W=24, scale=2, kb=5, blur_sigma=1.0,
                      disparities=(-1.0, 0.0, 0.8), noise_sigma=0.02, impulse=0.05,
                      window=5, iterations=10)
    prob = synth.make_problem(wl, seed=11)
    o = oracle_mod.Oracle.from_problem(prob, weights="paper", **synth.PAPER_SIGMAS)
    x20, wA, wS = o.admm(prob.y, prob.x0, 20)
    x40, _, _ = o.admm(prob.y, x20, 20, wA=wA, wS=wS)
    p0, p20, p40 = (synth.psnr(v, prob.gt) for v in (prob.x0, x20, x40))
    assert p20 > p0 + 2.0
    assert p40 > p20 + 1.0

"""Pins of the oracle's ADMM (Algorithm 1 + Algorithm 2) against mathematics:
exact fixed points, exact recovery, ADMM residual theory, and an
independent convex solver (scipy SLSQP) for the minimiser of J (Eq. sr_fin).
"""
import math

import numpy as np
import pytest
from scipy.optimize import minimize

from paper_2206_05047_gb300 import synth


def test_constant_image_is_exact_fixed_point(oracle_mod):
    """y_k = A_k c and x0 = c: residuals, S x and duals are all zero, so CG
    takes no step and x stays c bit for bit."""
    rng = np.random.default_rng(4)
    H, W, z = 6, 5, 2
    o = oracle_mod.Oracle(3, 3, H, W, z, synth.gaussian_blur_kernel(3, 0.9),
                          rng.uniform(-1.5, 1.5, (z * H, z * W)), window=5)
    c = np.full(o.hr, 0.4375)
    y = np.stack([o.A(k, c) for k in range(o.s_k)])
    x, wA, wS, diag = o.admm(y, c, 3, diagnostics=True)
    assert np.array_equal(x, c)
    assert not wA.any() and not wS.any()
    assert (diag[:, 4] == 0).all()


def test_exact_recovery_identity_operators():
    """zeta = 1, zero disparity, delta blur, no noise: A_k = I.  With
    lambda1 * s_k > 2 s_d the l1 data term dominates every TV subgradient
    (weights <= 1), so x = y is the unique minimiser and ADMM converges to
    it whatever the weights of each iteration."""
    from oracle import oracle as om
    rng = np.random.default_rng(0)
    H = W = 8
    gt = rng.random((H, W))
    o = om.Oracle(3, 3, H, W, 1, np.array([[1.0]]), np.zeros((H, W)), lambda1=2.0,
                  lambda2=1.0, mu=1.0, window=3, patch=3, h=0.3, cg_iters=5)
    assert 2.0 * 9 > 2 * 8
    y = np.repeat(gt[None], 9, axis=0)
    x0 = gt + 0.1 * rng.standard_normal((H, W))
    errs = []
    x, wA, wS = x0, None, None
    for _ in range(4):
        x, wA, wS = o.admm(y, x, 100, wA=wA, wS=wS)
        errs.append(np.linalg.norm(x - gt) / np.linalg.norm(gt))
    assert all(b < a for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 1e-5


def _tiny(oracle_mod, seed=0, mu=1.0, K=200):
    rng = np.random.default_rng(seed)
    o = oracle_mod.Oracle(3, 3, 2, 2, 2, synth.gaussian_blur_kernel(3, 0.8),
                          rng.uniform(-1, 1, (4, 4)), lambda1=0.5, lambda2=2.0, mu=mu,
                          window=3, patch=3, h=0.3, cg_iters=K, cg_tol=1e-28,
                          freeze_weights=True)
    y = rng.random((9, 2, 2))
    x0 = rng.random((4, 4))
    return o, y, x0


def test_he_yuan_residual_non_increasing(oracle_mod):
    """Frozen weights and an exact x-step: ||z_{n+1}-z_n||^2 + ||w_{n+1}-w_n||^2
    (scaled dual) never increases (He and Yuan's non-ergodic ADMM result)."""
    rng = np.random.default_rng(1)
    o = oracle_mod.Oracle(3, 3, 3, 3, 2, synth.gaussian_blur_kernel(3, 0.8),
                          rng.uniform(-1, 1, (6, 6)), lambda1=0.5, lambda2=2.0, mu=1.0,
                          window=3, patch=3, h=0.3, cg_iters=200, cg_tol=1e-28,
                          freeze_weights=True)
    y = rng.random((9, 3, 3))
    x0 = rng.random((6, 6))
    _, _, _, diag = o.admm(y, x0, 60, diagnostics=True)
    R = diag[1:, 0] + diag[1:, 1]
    assert np.all(np.diff(R) <= 1e-10 * R[:-1])
    assert R[-1] < 1e-2 * R[0]


def test_fixed_point_is_minimiser_of_J(oracle_mod):
    """With frozen weights, ADMM's limit minimises J: compare with an
    independent solver (SLSQP on the slack reformulation of the l1 terms)."""
    o, y, x0 = _tiny(oracle_mod, mu=3.0)
    w = o.weights(x0)
    p = o.p
    cols_A, cols_S = [], []
    for n in range(p):
        e = np.zeros(p); e[n] = 1.0
        e = e.reshape(o.hr)
        cols_A.append(np.concatenate([o.A(k, e).ravel() for k in range(o.s_k)]))
        cols_S.append(o.S(w, e).ravel())
    A = np.array(cols_A).T
    S = np.array(cols_S).T
    S = S[np.abs(S).sum(1) > 0]
    nA, nS = A.shape[0], S.shape[0]
    yy = y.ravel()
    l1, l2 = 0.5, 2.0

    def f(v):
        r = A @ v[:p] - yy
        return l1 * v[p:p + nA].sum() + l2 * r @ r + v[p + nA:].sum()

    def g(v):
        out = np.zeros_like(v)
        out[:p] = 2 * l2 * A.T @ (A @ v[:p] - yy)
        out[p:p + nA] = l1
        out[p + nA:] = 1.0
        return out

    Z = np.zeros
    I = np.eye
    Cm = np.vstack([np.hstack([A, -I(nA), Z((nA, nS))]), np.hstack([-A, -I(nA), Z((nA, nS))]),
                    np.hstack([S, Z((nS, nA)), -I(nS)]), np.hstack([-S, Z((nS, nA)), -I(nS)])])
    ub = np.concatenate([yy, -yy, Z(nS), Z(nS)])
    v0 = np.concatenate([x0.ravel(), np.abs(A @ x0.ravel() - yy) + 1, np.abs(S @ x0.ravel()) + 1])
    res = minimize(f, v0, jac=g, method="SLSQP", options={"maxiter": 2000, "ftol": 1e-14},
                   constraints=[{"type": "ineq", "fun": lambda v: ub - Cm @ v, "jac": lambda v: -Cm}])
    J_qp = o.cost(y, w, res.x[:p].reshape(o.hr))
    x, _, _ = o.admm(y, x0, 1000)
    J_admm = o.cost(y, w, x)
    # orc_cost against the SLSQP objective, which sums the slacks of the
    # dense operators' rows (tight at the solution): a wrong lambda, a missing
    # square or a dropped term of J moves one and not the other
    assert abs(J_qp - f(res.x)) <= 1e-7 * J_qp
    assert abs(J_admm - J_qp) <= 1e-7 * J_qp
    assert np.abs(x.ravel() - res.x[:p]).max() < 1e-4


def test_cost_closed_forms(oracle_mod):
    """J (Eq. sr_fin) on inputs where each term has a closed form.
    (a) A constant image has S x = 0; views y_k = A_k c except one LR pixel
        moved by delta: J = lambda1 |delta| + lambda2 delta^2.
    (b) Noise-free views of a vertical unit step with every weight 1: the
        data terms vanish and the regulariser counts the in-image pairs
        (u, u + d) across the step, (Hh - |d_i|) |d_j| of them for each
        direction d = (d_i, d_j) of the window (the step far from the
        borders)."""
    rng = np.random.default_rng(8)
    H, W, z = 6, 7, 2
    l1, l2 = 0.7, 3.0
    o = oracle_mod.Oracle(3, 3, H, W, z, synth.gaussian_blur_kernel(3, 0.9),
                          rng.uniform(-0.8, 0.8, (z * H, z * W)), lambda1=l1, lambda2=l2,
                          window=5)
    c = np.full(o.hr, 0.3)
    y = np.stack([o.A(k, c) for k in range(o.s_k)])
    delta = -0.125
    y[4, 2, 3] -= delta                     # residual A x - y = +delta there
    w = rng.random((o.s_d,) + o.hr)         # any weights: S c = 0
    assert abs(o.cost(y, w, c) - (l1 * abs(delta) + l2 * delta * delta)) <= 1e-12
    Hh, Wh = o.hr
    step = np.zeros(o.hr)
    step[:, Wh // 2:] = 1.0
    ys = np.stack([o.A(k, step) for k in range(o.s_k)])
    di, dj = o.dirs()
    count = sum((Hh - abs(int(a))) * abs(int(b)) for a, b in zip(di, dj))
    assert o.s_d == 24 and count > 0
    assert abs(o.cost(ys, np.ones((o.s_d,) + o.hr), step) - count) <= 1e-9 * count


def test_diagnostics_and_fixed_K(oracle_mod):
    prob = synth.make_problem(synth.custom(U=3, V=3, H=10, W=9, scale=2, kb=5,
                                           blur_sigma=1.0, window=5), seed=3)
    o = oracle_mod.Oracle.from_problem(prob)
    x, wA, wS, diag = o.admm(prob.y, prob.x0, 4, diagnostics=True)
    assert math.isnan(diag[0, 1]) and np.isfinite(diag[1:, 1]).all()
    assert (diag[:, 4] == 5).all()
    assert np.abs(wA).max() <= 1.0 / o.params["mu"] + 1e-15
    assert np.abs(wS).max() <= 1.0 / o.params["mu"] + 1e-15


def test_quality_improves_over_iterations(oracle_mod):
    """Synthetic analogue of the paper's PSNR-vs-iteration trend (Sec. 6.1)."""
    wl = synth.custom(U=5, V=5, H=24, W=24, scale=2, kb=5, blur_sigma=1.0,
                      disparities=(-1.0, 0.0, 0.8), noise_sigma=0.02, impulse=0.05,
                      window=5, iterations=10)
    prob = synth.make_problem(wl, seed=11)
    o = oracle_mod.Oracle.from_problem(prob)       # the configured h = 0.1
    x20, wA, wS = o.admm(prob.y, prob.x0, 20)
    x40, _, _ = o.admm(prob.y, x20, 20, wA=wA, wS=wS)
    p0, p20, p40 = (synth.psnr(v, prob.gt) for v in (prob.x0, x20, x40))
    assert p20 > p0 + 1.5
    assert p40 > p20 + 1.0


def test_pure_l2_data_term_keeps_the_data_duals_zero(oracle_mod):
    """lambda1 = 0 (the l2-only data term of Sec. 6.1's comparison): the data
    rows of F vanish, u_A = w_A = 0 stays inside the prox threshold, so the
    data duals stay exactly zero while the regulariser duals move."""
    wl = synth.custom(U=3, V=3, H=8, W=9, scale=2, kb=5, blur_sigma=1.0, window=3)
    prob = synth.make_problem(wl, seed=3)
    o = oracle_mod.Oracle.from_problem(prob, lambda1=0.0, lambda2=4.0, mu=300.0)
    x, wA, wS = o.admm(prob.y, prob.x0, 4)
    assert not wA.any() and wS.any()
    assert np.isfinite(x).all()


def test_pure_l1_data_term_solves_the_l1_problem(oracle_mod):
    """lambda2 = 0 (the l1-only data term, as in the paper's MISR runs): the
    compact form without the 1/sqrt(lambda2) scaling stays defined, and with
    identity operators x = y is recovered (exact-penalty argument as in
    test_exact_recovery_identity_operators)."""
    rng = np.random.default_rng(1)
    H = W = 6
    gt = rng.random((H, W))
    o = oracle_mod.Oracle(3, 3, H, W, 1, np.array([[1.0]]), np.zeros((H, W)), lambda1=2.0,
                          lambda2=0.0, mu=1.0, window=3, patch=3, h=0.3, cg_iters=5)
    y = np.repeat(gt[None], 9, axis=0)
    x, _, _ = o.admm(y, gt + 0.1 * rng.standard_normal((H, W)), 400)
    assert np.linalg.norm(x - gt) <= 1e-4 * np.linalg.norm(gt)


def test_rotated_order_equals_textbook_admm(oracle_mod):
    """Algorithm 1 runs ADMM in the order z, w, x and hands the x-step the
    over-relaxed dual f = 2w_n - w_{n-1}.  Written the textbook way instead
    -- x-update by a dense solve of the augmented Lagrangian's normal
    equations, soft threshold, dual ascent, with z = F x - b', F = [l1 A; S],
    b' = [l1 y; 0] -- and started from the (z, w) that x0 gives, the same
    problem produces the same iterates (frozen weights, exact x-step)."""
    rng = np.random.default_rng(7)
    l1, l2, mu = 0.7, 1.5, 2.0
    o = oracle_mod.Oracle(3, 3, 3, 3, 2, synth.gaussian_blur_kernel(3, 0.8),
                          rng.uniform(-1, 1, (6, 6)), lambda1=l1, lambda2=l2, mu=mu,
                          window=3, patch=3, h=0.3, cg_iters=400, cg_tol=1e-30,
                          freeze_weights=True)
    y = rng.random((9, 3, 3))
    x0 = rng.random((6, 6))
    p = 36
    w0 = o.weights(x0)
    eye = np.eye(p)
    A = np.array([np.concatenate([o.A(k, e.reshape(6, 6)).ravel() for k in range(9)])
                  for e in eye]).T
    S = np.array([o.S(w0, e.reshape(6, 6)).ravel() for e in eye]).T
    F = np.vstack([l1 * A, S])
    b = np.concatenate([l1 * y.ravel(), np.zeros(S.shape[0])])
    soft = lambda u: np.sign(u) * np.maximum(np.abs(u) - 1.0 / mu, 0.0)
    N = 6
    # textbook ADMM for  l2 |Ax - y|^2 + |z|_1  s.t.  z = F x - b'
    u = F @ x0.ravel() - b
    z = soft(u)
    w = u - z
    M = 2 * l2 * A.T @ A + mu * F.T @ F
    for k in range(N):
        x = np.linalg.solve(M, 2 * l2 * A.T @ y.ravel() + mu * F.T @ (b + z - w))
        if k < N - 1:
            u = F @ x - b + w
            z = soft(u)
            w = u - z
    xr, _, _ = o.admm(y, x0, N)
    np.testing.assert_allclose(xr.ravel(), x, rtol=0, atol=1e-9 * np.abs(x).max())

"""The paper's regulariser weights (Sec. 3.4: spatial * edge * occlusion,
directed) on the CUDA path against the FP64 oracle, through the C ABI.

The stored-weight kernels (windows 3, 5, 7) keep one root-mean-square weight
per edge for the x-step and update each dual of the edge with its own
directed weight; the generic kernel (window 9) stages the per-pixel factor
and recomputes the weights per direction.  Tolerances as for the patch
weights (the weights themselves are better conditioned: 1/sigma_e = 10
where the patch weights carry 1/h^2 = 100):
  weights                abs error <= 2e-6
  normal matrix          max-abs <= 5e-6 of the output's max, <p, M p> rel 2e-6
  one ADMM iteration     rel-L2 <= 2e-5 on x and on both dual blocks
  full solve, fixed N    rel-L2 <= 1e-4 and |dPSNR| <= 0.01 dB (float32 state);
                         rel-L2 <= 2e-3 and |dPSNR| <= 0.05 dB (half storage)
"""
import numpy as np
import pytest

from paper_2206_05047_gb300 import lfsr, synth
from tests.gpu_util import Case, f32, max_err, rel_err

pytestmark = pytest.mark.gpu

SIGMAS = dict(synth.PAPER_SIGMAS, sigma_o2=0.5)

CASES = [
    # (name, workload overrides, projection error given)
    ("w5_x2", dict(U=5, V=5, H=21, W=19, scale=2, kb=5, blur_sigma=1.0, window=5,
                   disparities=(-1.0, 0.0, 0.8)), True),
    ("w7_x3", dict(U=3, V=5, H=13, W=11, scale=3, kb=7, blur_sigma=1.3, window=7,
                   disparities=(-2.3, 0.4, 1.7)), False),
    ("w3_x2", dict(U=3, V=3, H=17, W=36, scale=2, kb=3, blur_sigma=0.8, window=3,
                   disparities=(-1.5, 1.1)), True),
    # 9x9 window: the generic NLTV kernel
    ("w9_generic", dict(U=3, V=3, H=12, W=13, scale=2, kb=3, blur_sigma=0.8, window=9,
                        disparities=(-0.7, 0.9)), True),
]


def _case(name, seed=0, precision="fp32", sigmas=None):
    ov, with_pe = {n: (o, p) for n, o, p in CASES}[name]
    wl = synth.custom(**ov)
    pe = None
    if with_pe:
        pe = np.random.default_rng(17).standard_normal(wl.HR) * 0.4
    return Case(wl, seed=seed, precision=precision, weights="paper",
                sigmas=SIGMAS if sigmas is None else sigmas, proj_err=pe)


@pytest.mark.parametrize("name", [c[0] for c in CASES])
def test_directed_weights(name):
    c = _case(name)
    o = c.oracle
    rng = np.random.default_rng(4)
    for x in (c.x0, f32(rng.random(o.hr))):
        w = c.empty(o.s_d, *o.hr)
        lfsr.weights(c.h, c.t(x), w)
        ref = o.weights(x.astype(np.float64))
        assert np.abs(c.np(w) - ref).max() <= 2e-6


def test_occlusion_factor_of_the_scene():
    """A constant x and no spatial factor leave w_d(u) = o(u): the
    occlusion factor of the scene's disparity map (plane boundaries) and
    of the projection error, computed once by lfsr_create."""
    c = _case("w5_x2", sigmas=dict(sigma_o1=0.5, sigma_o2=0.5))
    o = c.oracle
    w = c.empty(o.s_d, *o.hr)
    lfsr.weights(c.h, c.t(np.full(o.hr, 0.5, np.float32)), w)
    occ = o.occlusion_factor()
    assert (occ < 0.9).any()                      # the scene has occluding boundaries
    ref = o.weights(np.full(o.hr, 0.5))
    assert np.abs(c.np(w) - ref).max() <= 1e-6
    centre = o.s_d // 2                           # direction (0, 1): inside except the last column
    assert np.abs(c.np(w)[centre][:, :-1] - occ[:, :-1]).max() <= 1e-6


@pytest.mark.parametrize("name", [c[0] for c in CASES])
def test_normal_matrix(name):
    c = _case(name)
    o = c.oracle
    rng = np.random.default_rng(2)
    p = f32(rng.standard_normal(o.hr))
    q = c.empty(*o.hr)
    pMp = lfsr.apply_normal(c.h, c.t(c.x0), c.t(p), q)
    ref = o.normal_apply(o.weights(c.x0.astype(np.float64)), p.astype(np.float64))
    assert max_err(c.np(q), ref) <= 5e-6
    ref_pMp = float(np.vdot(p.astype(np.float64), ref))
    assert abs(pMp - ref_pMp) <= 2e-6 * abs(ref_pMp)


def _random_duals(c, rng):
    o, wl = c.oracle, c.wl
    t = 1.0 / c.params["mu"]
    wA = f32(np.clip(0.6 * t * rng.standard_normal((o.s_k, wl.H, wl.W)), -t, t))
    wS = np.clip(0.6 * t * rng.standard_normal((o.s_d,) + o.hr), -t, t)
    di, dj = o.dirs()
    Hh, Wh = o.hr
    ii, jj = np.meshgrid(np.arange(Hh), np.arange(Wh), indexing="ij")
    for d in range(o.s_d):
        inside = (ii + di[d] >= 0) & (ii + di[d] < Hh) & (jj + dj[d] >= 0) & (jj + dj[d] < Wh)
        wS[d][~inside] = 0.0
    return wA, f32(wS)


@pytest.mark.parametrize("name", [c[0] for c in CASES])
def test_one_iteration_from_state(name):
    """One ADMM iteration from an identical (x, wA, wS) state: the two duals
    of every edge move by their own directed weights."""
    c = _case(name)
    o = c.oracle
    wA, wS = _random_duals(c, np.random.default_rng(3))
    lfsr.load(c.h, c.t(c.y), c.t(c.x0))
    lfsr.set_state(c.h, c.t(c.x0), c.t(wA), c.t(wS))
    lfsr.iterate(c.h, 1)
    xs, wAs, wSs = c.empty(*o.hr), c.empty(*wA.shape), c.empty(*wS.shape)
    lfsr.get_state(c.h, xs, wAs, wSs)
    rx, rA, rS = o.admm(c.y.astype(np.float64), c.x0.astype(np.float64), 1,
                        wA=wA.astype(np.float64), wS=wS.astype(np.float64))
    assert rel_err(c.np(xs), rx) <= 2e-5
    assert rel_err(c.np(wAs), rA) <= 2e-5
    assert rel_err(c.np(wSs), rS) <= 2e-5


@pytest.mark.parametrize("name,n_iter", [("w5_x2", 15), ("w9_generic", 8)])
def test_full_solve(name, n_iter):
    c = _case(name)
    x = c.empty(*c.oracle.hr)
    lfsr.solve(c.h, c.t(c.y), n_iter, c.t(c.x0), x)
    ref, _, _ = c.oracle.admm(c.y.astype(np.float64), c.x0.astype(np.float64), n_iter)
    gx = c.np(x)
    assert rel_err(gx, ref) <= 1e-4
    assert abs(synth.psnr(gx, c.prob.gt) - synth.psnr(ref, c.prob.gt)) <= 0.01
    assert lfsr.stats(c.h)["status"] == 0


def test_lf5x5_solve_half_storage():
    """5x5 views, 64^2 -> 128^2, 30 iterations with half storage."""
    wl = synth.WORKLOADS["lf5x5_64_x2"]
    c = Case(wl, seed=0, precision="fp16", weights="paper", sigmas=synth.PAPER_SIGMAS)
    x = c.empty(*c.oracle.hr)
    lfsr.solve(c.h, c.t(c.y), 30, c.t(c.x0), x)
    ref, _, _ = c.oracle.admm(c.y.astype(np.float64), c.x0.astype(np.float64), 30)
    gx = c.np(x)
    assert rel_err(gx, ref) <= 2e-3
    assert abs(synth.psnr(gx, c.prob.gt) - synth.psnr(ref, c.prob.gt)) <= 0.05
    # the paper's weights improve on the initial estimate
    assert synth.psnr(ref, c.prob.gt) > synth.psnr(c.x0, c.prob.gt) + 1.0


def test_batch_equals_each_light_field_alone():
    import torch
    probs, kws = [], []
    for i, name in enumerate(("w5_x2", "w3_x2", "w7_x3")):
        ov = {n: o for n, o, _ in CASES}[name]
        wl = synth.custom(**dict(ov, window=5))
        pr = synth.make_problem(wl, seed=30 + i)
        probs.append(pr)
        kws.append(dict(U=wl.U, V=wl.V, H=wl.H, W=wl.W, scale=wl.scale, blur=f32(pr.blur),
                        disparity=f32(pr.disparity), lambda1=2.0, lambda2=4.0, mu=300.0,
                        nltv_window=5, cg_iters=5, weights="paper", **SIGMAS,
                        proj_err=f32(np.full(wl.HR, 0.2 * i))))
    b = lfsr.Batch(kws)
    dev = torch.device("cuda:0")
    for j, pr in enumerate(probs):
        b.load(j, torch.from_numpy(f32(pr.y)).to(dev), torch.from_numpy(f32(pr.x0)).to(dev))
    b.iterate(6)
    for j, (pr, kw) in enumerate(zip(probs, kws)):
        xb = torch.empty(pr.wl.HR, dtype=torch.float32, device=dev)
        b.get_x(j, xb)
        s = lfsr.Solver(**kw)
        xa = torch.empty(pr.wl.HR, dtype=torch.float32, device=dev)
        lfsr.solve(s.handle, torch.from_numpy(f32(pr.y)).to(dev), 6,
                   torch.from_numpy(f32(pr.x0)).to(dev), xa)
        s.close()
        assert rel_err(xb.cpu().numpy(), xa.cpu().numpy()) <= 1e-5, j
    b.close()


def test_state_bytes_and_no_alloc_entry_point():
    import torch
    a = _case("w5_x2")
    wl = a.wl
    patch = Case(wl, seed=0)
    p = wl.HR[0] * wl.HR[1]
    assert lfsr.stats(a.h)["state_bytes"] - lfsr.stats(patch.h)["state_bytes"] == 4 * p
    t = torch.zeros(wl.HR, dtype=torch.float32, device="cuda:0")
    with pytest.raises(lfsr.LfsrError) as e:
        lfsr.apply_normal_noalloc(wl.U, wl.V, wl.H, wl.W, wl.scale, a.blur, a.disp,
                                  torch.from_numpy(a.disp).to("cuda:0"), t, t, t.clone(),
                                  weights=lfsr.LFSR_WEIGHTS_PAPER)
    assert e.value.code == lfsr.LFSR_EUNSUPPORTED

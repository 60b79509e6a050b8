"""The continuous-batching server on the GPU: requests admitted while others
run (at either state parity) give the same result as each solved alone and
match the FP64 oracle, and the device memory returns to zero."""
import numpy as np
import pytest

from paper_2206_05047_gb300 import lfsr, synth
from tests.gpu_util import f32, rel_err
from tests.test_gpu_batch import GEOMS, SOLVER, _alone

pytestmark = pytest.mark.gpu


def _requests():
    out = []
    for i, gm in enumerate(GEOMS + GEOMS[:2]):
        wl = synth.custom(window=5, patch=3, **gm)
        pr = synth.make_problem(wl, seed=40 + i)
        kw = dict(U=wl.U, V=wl.V, H=wl.H, W=wl.W, scale=wl.scale, blur=f32(pr.blur),
                  disparity=f32(pr.disparity), **SOLVER)
        out.append((pr, kw))
    return out


def _oracle_x(pr, kw, n_iter):
    from oracle import oracle as om
    o = om.Oracle(kw["U"], kw["V"], kw["H"], kw["W"], kw["scale"],
                  f32(kw["blur"]).astype(np.float64), f32(kw["disparity"]).astype(np.float64),
                  lambda1=SOLVER["lambda1"], lambda2=SOLVER["lambda2"], mu=SOLVER["mu"],
                  window=SOLVER["nltv_window"], patch=SOLVER["nltv_patch"], h=SOLVER["nltv_h"],
                  cg_iters=SOLVER["cg_iters"], cg_tol=SOLVER["cg_tol"])
    ref, _, _ = o.admm(f32(pr.y).astype(np.float64), f32(pr.x0).astype(np.float64), n_iter)
    return ref


def test_results_are_the_same_alone_and_in_the_mix():
    reqs = _requests()
    n_iter = 9
    srv = lfsr.Server(8 << 30, max_active=3, iterations=n_iter, iterations_per_step=2)
    ids = [srv.submit(f32(pr.y), f32(pr.x0), **kw) for pr, kw in reqs[:2]]
    srv.step()                                   # 2 iterations
    srv.step()
    ids += [srv.submit(f32(pr.y), f32(pr.x0), **kw) for pr, kw in reqs[2:5]]
    srv.step()                                   # one joins (3 slots), 1 more iteration: odd parity
    ids += [srv.submit(f32(pr.y), f32(pr.x0), **kw) for pr, kw in reqs[5:]]
    for _ in range(200):
        if srv.stats()["done"] == len(reqs):
            break
        srv.step()
    st = srv.stats()
    assert st["done"] == len(reqs) and st["failed"] == 0 and st["active"] == 0
    assert st["bytes_in_use"] == 0 and st["batch_rebuilds"] >= 3
    for rid, (pr, kw) in zip(ids, reqs):
        state, iters, rc = srv.status(rid)
        assert state == lfsr.LFSR_REQ_DONE and iters == n_iter and rc == 0
        x = np.zeros(pr.wl.HR, np.float32)
        srv.fetch(rid, x)
        assert rel_err(x, _alone(kw, pr, n_iter)) <= 1e-5, rid
        # requests that joined mid-run (at odd and even state parity) against
        # the FP64 oracle, at the float32 path's parity tolerance
        ref = _oracle_x(pr, kw, n_iter)
        assert rel_err(x, ref) <= 1e-4, rid
        assert abs(synth.psnr(x, pr.gt) - synth.psnr(ref, pr.gt)) <= 0.01, rid
    srv.close()


def test_estimate_bounds_the_allocation():
    for pr, kw in _requests()[:3]:
        est = lfsr.estimate_state_bytes(**kw)
        s = lfsr.Solver(**kw)
        got = lfsr.stats(s.handle)["state_bytes"]
        assert got <= est <= got + (1 << 20), (got, est)
        s.close()


def test_paper_weight_requests_are_the_same_alone_and_in_the_mix():
    """Requests with the paper's weights and a projection error (copied at
    submission), one joining at odd parity."""
    reqs = []
    for i, (pr, kw) in enumerate(_requests()[:3]):
        pe = np.random.default_rng(60 + i).standard_normal(pr.wl.HR).astype(np.float32)
        reqs.append((pr, dict(kw, weights="paper", **synth.PAPER_SIGMAS, proj_err=pe)))
    for pr, kw in reqs:
        kw["sigma_o2"] = 0.5
    n_iter = 7
    srv = lfsr.Server(8 << 30, max_active=3, iterations=n_iter, iterations_per_step=3)
    ids = [srv.submit(f32(pr.y), f32(pr.x0), **kw) for pr, kw in reqs[:2]]
    srv.step()                                   # 3 iterations: the next joins at odd parity
    ids.append(srv.submit(f32(reqs[2][0].y), f32(reqs[2][0].x0), **reqs[2][1]))
    for _ in range(50):
        if srv.stats()["done"] == len(reqs):
            break
        srv.step()
    assert srv.stats()["done"] == len(reqs)
    for rid, (pr, kw) in zip(ids, reqs):
        x = np.zeros(pr.wl.HR, np.float32)
        srv.fetch(rid, x)
        assert rel_err(x, _alone(kw, pr, n_iter)) <= 1e-5, rid
    srv.close()
    est = lfsr.estimate_state_bytes(**reqs[0][1])
    s = lfsr.Solver(**reqs[0][1])
    got = lfsr.stats(s.handle)["state_bytes"]
    assert got <= est <= got + (1 << 20), (got, est)
    s.close()


def test_a_request_failing_at_admission_leaves_the_others_running():
    """A request the served kernels cannot take (a non-separable blur needs
    the generic operator kernel) fails when admitted, with its error code;
    the requests around it complete as if it had not been there."""
    reqs = _requests()[:3]
    pr_bad, kw_bad = reqs[1]
    K = np.random.default_rng(9).random((5, 5)) ** 3
    kw_bad = dict(kw_bad, blur=f32(K / K.sum()))
    n_iter = 5
    srv = lfsr.Server(8 << 30, max_active=3, iterations=n_iter, iterations_per_step=2)
    ids = [srv.submit(f32(reqs[0][0].y), f32(reqs[0][0].x0), **reqs[0][1]),
           srv.submit(f32(pr_bad.y), f32(pr_bad.x0), **kw_bad),
           srv.submit(f32(reqs[2][0].y), f32(reqs[2][0].x0), **reqs[2][1])]
    for _ in range(20):
        st = srv.stats()
        if st["done"] + st["failed"] == 3:
            break
        srv.step()
    st = srv.stats()
    assert st["done"] == 2 and st["failed"] == 1 and st["bytes_in_use"] == 0
    state, _, rc = srv.status(ids[1])
    assert state == lfsr.LFSR_REQ_FAILED and rc == lfsr.LFSR_EUNSUPPORTED
    for rid, (pr, kw) in ((ids[0], reqs[0]), (ids[2], reqs[2])):
        x = np.zeros(pr.wl.HR, np.float32)
        srv.fetch(rid, x)
        assert rel_err(x, _alone(kw, pr, n_iter)) <= 1e-5, rid
    srv.close()

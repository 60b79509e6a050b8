"""Batches of uneven light fields (one launch per phase over a work list that
spans all of them): every light field's result in the batch equals its
result solved alone (same arithmetic; only the order of float atomic
additions differs) and matches the FP64 oracle."""
import numpy as np
import pytest

from paper_2206_05047_gb300 import lfsr, synth
from tests.gpu_util import f32, rel_err

pytestmark = pytest.mark.gpu

# uneven geometries: two operator groups (x2 with a 5x5 blur, x3 with 7x7),
# a single-view light field and ragged tiles everywhere
GEOMS = [
    dict(U=3, V=3, H=20, W=20, scale=2, kb=5, blur_sigma=1.0, disparities=(-1.0, 0.6)),
    dict(U=5, V=3, H=17, W=23, scale=2, kb=5, blur_sigma=1.0, disparities=(-0.8, 0.3, 1.1)),
    dict(U=3, V=3, H=14, W=13, scale=3, kb=7, blur_sigma=1.3, disparities=(-1.2, 0.9)),
    dict(U=1, V=1, H=25, W=22, scale=2, kb=5, blur_sigma=1.0, disparities=(0.0, 0.4)),
    dict(U=3, V=5, H=11, W=30, scale=3, kb=7, blur_sigma=1.3, disparities=(-0.5, 1.5)),
]
SOLVER = dict(lambda1=2.0, lambda2=4.0, mu=300.0, nltv_window=5, nltv_patch=3, nltv_h=0.1,
              cg_iters=5, cg_tol=0.0)


def _jobs(precision="fp32"):
    probs, kws = [], []
    for i, gm in enumerate(GEOMS):
        wl = synth.custom(window=5, patch=3, **gm)
        pr = synth.make_problem(wl, seed=20 + i)
        probs.append(pr)
        kws.append(dict(U=wl.U, V=wl.V, H=wl.H, W=wl.W, scale=wl.scale, blur=f32(pr.blur),
                        disparity=f32(pr.disparity), precision=precision, **SOLVER))
    return probs, kws


def _t(a):
    import torch
    return torch.from_numpy(f32(a)).to("cuda:0")


def _alone(kw, pr, n_iter):
    import torch
    s = lfsr.Solver(**kw)
    x = torch.empty(pr.wl.HR, dtype=torch.float32, device="cuda:0")
    lfsr.solve(s.handle, _t(pr.y), n_iter, _t(pr.x0), x)
    out = x.cpu().numpy().astype(np.float64)
    s.close()
    return out


def _batch_x(b, j, hr):
    import torch
    x = torch.empty(hr, dtype=torch.float32, device="cuda:0")
    b.get_x(j, x)
    return x.cpu().numpy().astype(np.float64)


def test_batch_equals_each_light_field_alone_and_the_oracle():
    from oracle import oracle as om
    probs, kws = _jobs()
    n_iter = 8
    b = lfsr.Batch(kws)
    assert b.launches_per_iteration() == 2 + 2 + 5 * (2 + 2)   # two operator groups
    for j, pr in enumerate(probs):
        b.load(j, _t(pr.y), _t(pr.x0))
    b.iterate(n_iter)
    for j, (pr, kw) in enumerate(zip(probs, kws)):
        xb = _batch_x(b, j, pr.wl.HR)
        xa = _alone(kw, pr, n_iter)
        assert rel_err(xb, xa) <= 1e-5, j
        o = om.Oracle(kw["U"], kw["V"], kw["H"], kw["W"], kw["scale"], f32(pr.blur).astype(np.float64),
                      f32(pr.disparity).astype(np.float64), lambda1=2.0, lambda2=4.0, mu=300.0,
                      window=5, patch=3, h=0.1, cg_iters=5, cg_tol=0.0)
        ref, _, _ = o.admm(f32(pr.y).astype(np.float64), f32(pr.x0).astype(np.float64), n_iter)
        assert rel_err(xb, ref) <= 1e-4, j
        st = b.stats(j)
        assert st["iterations"] == n_iter and st["status"] == 0 and st["cg_steps"] == 5
    b.close()


def test_batch_reload_at_odd_parity():
    """A light field loaded after an odd number of iterations (state parity
    1) runs exactly as a fresh solve."""
    probs, kws = _jobs()
    b = lfsr.Batch(kws)
    for j, pr in enumerate(probs):
        b.load(j, _t(pr.y), _t(pr.x0))
    b.iterate(3)
    j = 2
    b.load(j, _t(probs[j].y), _t(probs[j].x0))
    b.iterate(4)
    assert rel_err(_batch_x(b, j, probs[j].wl.HR), _alone(kws[j], probs[j], 4)) <= 1e-5
    assert rel_err(_batch_x(b, 0, probs[0].wl.HR), _alone(kws[0], probs[0], 7)) <= 1e-5
    b.close()


def test_batch_half_storage_equals_alone():
    probs, kws = _jobs("fp16")
    b = lfsr.Batch(kws)
    for j, pr in enumerate(probs):
        b.load(j, _t(pr.y), _t(pr.x0))
    b.iterate(6)
    for j in (0, 2, 3):
        assert rel_err(_batch_x(b, j, probs[j].wl.HR), _alone(kws[j], probs[j], 6)) <= 1e-5
    b.close()


def test_batch_host_memory_and_single_light_field():
    probs, kws = _jobs()
    b = lfsr.Batch(kws[:1])
    assert b.launches_per_iteration() == 3 + 3 * 5
    b.load(0, f32(probs[0].y), f32(probs[0].x0))
    b.iterate(5)
    xh = np.zeros(probs[0].wl.HR, np.float32)
    b.get_x(0, xh)
    assert rel_err(xh, _alone(kws[0], probs[0], 5)) <= 1e-5
    b.close()


def test_batch_rejects_unsupported_light_fields():
    probs, kws = _jobs()
    bad = dict(kws[0])
    K = np.random.default_rng(9).random((5, 5)) ** 3
    bad["blur"] = f32(K / K.sum())                 # not separable: generic kernel only
    with pytest.raises(lfsr.LfsrError) as e:
        lfsr.Batch([kws[1], bad])
    assert e.value.code == lfsr.LFSR_EUNSUPPORTED
    assert "light field 1" in lfsr.batch_last_error(None)


@pytest.mark.parametrize("tiles,chunk", [((32, 32), 3), ((64, 32), 6), ((32, 64), 6)])
def test_batch_tunings_give_the_same_results(tiles, chunk):
    """Every tile side / stencil blocking the autotuner may choose computes
    the same iteration (up to the order of float atomic additions)."""
    probs, kws = _jobs()
    b = lfsr.Batch(kws)
    b.set_tuning(tiles, chunk)
    assert b.tuning() == {"operator_tile": list(tiles), "nltv_apply_chunk": chunk,
                          "form": "phases"}
    for j, pr in enumerate(probs):
        b.load(j, _t(pr.y), _t(pr.x0))
    b.iterate(5)
    for j in range(len(probs)):
        assert rel_err(_batch_x(b, j, probs[j].wl.HR), _alone(kws[j], probs[j], 5)) <= 1e-5, j
    b.close()


def test_batch_autotune_then_reload():
    probs, kws = _jobs()
    b = lfsr.Batch(kws)
    for j, pr in enumerate(probs):
        b.load(j, _t(pr.y), _t(pr.x0))
    choice = b.autotune()
    assert all(t in (32, 64) for t in choice["operator_tile"]) and len(choice["operator_tile"]) == 2
    assert choice["nltv_apply_chunk"] in (3, 6)
    for j, pr in enumerate(probs):
        b.load(j, _t(pr.y), _t(pr.x0))
    b.iterate(4)
    for j in range(len(probs)):
        assert rel_err(_batch_x(b, j, probs[j].wl.HR), _alone(kws[j], probs[j], 4)) <= 1e-5, j
    with pytest.raises(lfsr.LfsrError):
        b.set_tuning((64,), 6)                     # one tile side per group
    b.close()


"""The persistent form of a batch iteration (one cooperative launch runs every
phase of Algorithm 1 with the CG steps of Algorithm 2 for every light field,
grid barriers between the phases): each light field's result equals the
per-phase launches' (same arithmetic; only the order of float atomic
additions differs) and the FP64 oracle; a barrier wait that runs out comes
back as LFSR_ETIMEOUT and leaves the batch usable after a reload."""
import numpy as np
import pytest

from paper_2206_05047_gb300 import lfsr, synth
from tests.gpu_util import f32, rel_err

pytestmark = pytest.mark.gpu

# one group, x2 with a 5x5 blur, NLTV window 5: uneven sizes, ragged tiles,
# a single-view light field
GEOMS_W5 = [
    dict(U=3, V=3, H=20, W=20, scale=2, kb=5, blur_sigma=1.0, disparities=(-1.0, 0.6)),
    dict(U=5, V=3, H=17, W=23, scale=2, kb=5, blur_sigma=1.0, disparities=(-0.8, 0.3, 1.1)),
    dict(U=1, V=1, H=25, W=22, scale=2, kb=5, blur_sigma=1.0, disparities=(0.0, 0.4)),
    dict(U=5, V=5, H=40, W=36, scale=2, kb=5, blur_sigma=1.0, disparities=(-1.0, 0.0, 0.8)),
]
# two groups, NLTV window 7: the x3 (9x9 blur) light field first, so the
# kernel's group slots (x2 first) differ from the batch's group order
GEOMS_W7 = [
    dict(U=3, V=3, H=14, W=13, scale=3, kb=9, blur_sigma=1.5, disparities=(-1.2, 0.9)),
    dict(U=3, V=5, H=22, W=30, scale=2, kb=7, blur_sigma=1.2, disparities=(-0.5, 1.5)),
    dict(U=5, V=5, H=19, W=21, scale=3, kb=9, blur_sigma=1.5, disparities=(-1.0, 0.0, 1.0)),
    dict(U=1, V=1, H=33, W=17, scale=2, kb=7, blur_sigma=1.2, disparities=(0.0, 0.7)),
]


def _jobs(geoms, window, precision="fp32", seed0=40):
    probs, kws = [], []
    for i, gm in enumerate(geoms):
        wl = synth.custom(window=window, patch=3, **gm)
        pr = synth.make_problem(wl, seed=seed0 + i)
        probs.append(pr)
        kws.append(dict(U=wl.U, V=wl.V, H=wl.H, W=wl.W, scale=wl.scale, blur=f32(pr.blur),
                        disparity=f32(pr.disparity), precision=precision, lambda1=2.0,
                        lambda2=4.0, mu=300.0, nltv_window=window, nltv_patch=3, nltv_h=0.1,
                        cg_iters=5, cg_tol=0.0))
    return probs, kws


def _t(a):
    import torch
    return torch.from_numpy(f32(a)).to("cuda:0")


def _run(b, probs, n_iter):
    import torch
    for j, pr in enumerate(probs):
        b.load(j, _t(pr.y), _t(pr.x0))
    b.iterate(n_iter)
    xs = []
    for j, pr in enumerate(probs):
        x = torch.empty(pr.wl.HR, dtype=torch.float32, device="cuda:0")
        b.get_x(j, x)
        xs.append(x.cpu().numpy().astype(np.float64))
    return xs


def _oracle(kw, pr, window, n_iter):
    from oracle import oracle as om
    o = om.Oracle(kw["U"], kw["V"], kw["H"], kw["W"], kw["scale"],
                  f32(pr.blur).astype(np.float64), f32(pr.disparity).astype(np.float64),
                  lambda1=2.0, lambda2=4.0, mu=300.0, window=window, patch=3, h=0.1,
                  cg_iters=5, cg_tol=0.0)
    ref, _, _ = o.admm(f32(pr.y).astype(np.float64), f32(pr.x0).astype(np.float64), n_iter)
    return ref


@pytest.mark.parametrize("geoms,window,groups", [(GEOMS_W5, 5, 1), (GEOMS_W7, 7, 2)])
def test_persistent_equals_per_phase_and_oracle(geoms, window, groups):
    probs, kws = _jobs(geoms, window)
    n_iter = 7   # odd: the last iteration runs from the single-iteration graph
    b = lfsr.Batch(kws)
    assert b.persistent_available()
    assert b.form() == "phases"
    assert b.launches_per_iteration() == 2 + groups + 5 * (2 + groups)
    x_phase = _run(b, probs, n_iter)
    b.set_form("persistent")
    assert b.form() == "persistent" and b.launches_per_iteration() == 1
    x_pers = _run(b, probs, n_iter)
    for j, (pr, kw) in enumerate(zip(probs, kws)):
        assert rel_err(x_pers[j], x_phase[j]) <= 1e-5, j
        assert rel_err(x_pers[j], _oracle(kw, pr, window, n_iter)) <= 1e-4, j
        st = b.stats(j)
        assert st["status"] == 0 and st["cg_steps"] == 5
    b.close()


def test_persistent_half_storage_matches_per_phase():
    probs, kws = _jobs(GEOMS_W7, 7, precision="fp16", seed0=60)
    b = lfsr.Batch(kws)
    assert b.persistent_available()
    x_phase = _run(b, probs, 6)
    b.set_form("persistent")
    x_pers = _run(b, probs, 6)
    for j in range(len(probs)):
        # 16-bit storage rounds each stored value: the atomic order moves
        # single roundings, so the bound is the storage type's
        assert rel_err(x_pers[j], x_phase[j]) <= 1e-3, j
    b.close()


def test_barrier_timeout_reports_and_reload_recovers():
    probs, kws = _jobs(GEOMS_W5, 5, seed0=80)
    b = lfsr.Batch(kws)
    b.set_form("persistent")
    x_ok = _run(b, probs, 3)
    # every wait runs out after 2 ms: the iteration is abandoned and the
    # status reports it for every light field
    b.set_device_wait(2_000_000, test_unreachable=True)
    for j, pr in enumerate(probs):
        b.load(j, _t(pr.y), _t(pr.x0))
    b.iterate(2)
    import torch
    for j, pr in enumerate(probs):
        x = torch.empty(pr.wl.HR, dtype=torch.float32, device="cuda:0")
        with pytest.raises(lfsr.LfsrError) as ei:
            b.get_x(j, x)
        assert ei.value.code == lfsr.LFSR_ETIMEOUT
    # the default limit again: a reload starts clean and the solve is the same
    b.set_device_wait(lfsr.LFSR_DEFAULT_WAIT_NS)
    for _ in range(2):
        x_again = _run(b, probs, 3)
        for j in range(len(probs)):
            assert rel_err(x_again[j], x_ok[j]) <= 1e-5, j
    b.close()


def test_form_choice_and_unsupported_batches():
    probs, kws = _jobs(GEOMS_W5, 5, seed0=100)
    b = lfsr.Batch(kws)
    for j, pr in enumerate(probs):
        b.load(j, _t(pr.y), _t(pr.x0))
    tuning = b.autotune()
    assert tuning["form"] == b.form()
    if not b.persistent_available():
        # the tuned operator tile has no persistent instance: the per-phase
        # form stays; the 64 x 64 tiles bring the persistent form back
        assert b.form() == "phases"
        b.set_tuning([64] * len(tuning["operator_tile"]), tuning["nltv_apply_chunk"])
        assert b.persistent_available()
    x_tuned = _run(b, probs, 4)
    other = "phases" if b.form() == "persistent" else "persistent"
    b.set_form(other)
    x_other = _run(b, probs, 4)
    for j in range(len(probs)):
        assert rel_err(x_tuned[j], x_other[j]) <= 1e-5, j
    b.close()
    # (2, 5) and (3, 7) groups with a 5 x 5 window: no compiled instance
    geoms = [GEOMS_W5[0], dict(U=3, V=3, H=14, W=13, scale=3, kb=7, blur_sigma=1.3,
                               disparities=(-1.2, 0.9))]
    probs, kws = _jobs(geoms, 5, seed0=120)
    b = lfsr.Batch(kws)
    assert not b.persistent_available()
    with pytest.raises(lfsr.LfsrError) as ei:
        b.set_form("persistent")
    assert ei.value.code == lfsr.LFSR_EUNSUPPORTED
    assert b.form() == "phases"
    b.close()


def test_persistent_cg_early_exit_matches_per_phase():
    """With a CG threshold tau the x-step of each light field stops on its own
    step; the persistent launch skips the finished light fields' work in
    every later phase exactly as the per-phase launches do."""
    probs, kws = _jobs(GEOMS_W5, 5, seed0=140)
    # a threshold above every light field's final |r|^2 of a run without one:
    # the light fields whose residual falls faster stop before step 5
    b = lfsr.Batch(kws)
    _run(b, probs, 5)
    pis = [b.stats(j)["cg_pi"] for j in range(len(probs))]
    b.close()
    for kw in kws:
        kw["cg_tol"] = float(1.5 * max(pis))
    b = lfsr.Batch(kws)
    x_phase = _run(b, probs, 5)
    steps_phase = [b.stats(j)["cg_steps"] for j in range(len(probs))]
    b.set_form("persistent")
    x_pers = _run(b, probs, 5)
    steps_pers = [b.stats(j)["cg_steps"] for j in range(len(probs))]
    assert steps_pers == steps_phase
    assert min(steps_pers) < 5            # the threshold ends some x-steps early
    for j in range(len(probs)):
        assert rel_err(x_pers[j], x_phase[j]) <= 1e-5, j
    b.close()

"""The continuous-batching server's scheduling, checked without a device
(dry-run mode runs the same admission, stepping and retirement logic):
arrival-order admission with no overtaking, active slots, the device-memory
budget, retirement exactly at N iterations, and the size estimate."""
import numpy as np
import pytest

from paper_2206_05047_gb300 import lfsr


def _req(U=3, V=3, H=16, W=16, scale=2, **kw):
    blur = np.ones((5, 5), np.float32) / 25
    disp = np.zeros((scale * H, scale * W), np.float32)
    y = np.zeros((U * V, H, W), np.float32)
    x0 = np.full((scale * H, scale * W), 0.5, np.float32)
    args = dict(U=U, V=V, H=H, W=W, scale=scale, blur=blur, disparity=disp, **kw)
    return y, x0, args


def _submit(srv, **kw):
    y, x0, args = _req(**kw)
    return srv.submit(y, x0, **args)


def test_estimate_grows_with_size_and_halves_with_16bit_storage():
    small = lfsr.estimate_state_bytes(**_req(H=16, W=16)[2])
    big = lfsr.estimate_state_bytes(**_req(H=64, W=64)[2])
    assert big > 10 * small
    h32 = lfsr.estimate_state_bytes(**_req(U=9, V=9, H=128, W=128)[2])
    h16 = lfsr.estimate_state_bytes(**_req(U=9, V=9, H=128, W=128, precision="fp16")[2])
    assert 0.45 * h32 < h16 < 0.75 * h32


def test_slots_arrival_order_and_retirement_at_N():
    srv = lfsr.Server(1 << 40, max_active=2, iterations=7, iterations_per_step=3, dry_run=True)
    ids = [_submit(srv) for _ in range(3)]
    assert ids == [0, 1, 2]
    assert srv.step() == 2                       # admits 0 and 1, runs 3 iterations
    assert [srv.status(i)[:2] for i in ids] == [(1, 3), (1, 3), (0, 0)]
    assert srv.step() == 2                       # 6 iterations
    assert srv.step() == 0                       # 1 more (not 3): both due at 7, retired
    assert [srv.status(i)[:2] for i in ids[:2]] == [(2, 7), (2, 7)]
    assert srv.status(2)[0] == lfsr.LFSR_REQ_QUEUED
    assert srv.step() == 1                       # the third, counted from its admission
    assert srv.status(2)[:2] == (1, 3)
    st = srv.stats()
    assert st["admitted"] == 3 and st["retired"] == 2 and st["iterations"] == 10
    x = np.zeros((32, 32), np.float32)
    srv.fetch(0, x)
    assert srv.status(0)[0] == lfsr.LFSR_REQ_FETCHED
    with pytest.raises(lfsr.LfsrError):
        srv.fetch(2, x)                          # not done yet
    srv.close()


def test_budget_blocks_without_overtaking_and_frees_on_retirement():
    big = lfsr.estimate_state_bytes(**_req(U=5, V=5, H=48, W=48)[2])
    small = lfsr.estimate_state_bytes(**_req(H=16, W=16)[2])
    srv = lfsr.Server(big + small // 2, max_active=8, iterations=2, iterations_per_step=2,
                      dry_run=True)
    a = _submit(srv, U=5, V=5, H=48, W=48)       # fits alone
    b = _submit(srv, U=5, V=5, H=48, W=48)       # must wait for a
    c = _submit(srv)                             # would fit beside a, but arrived after b
    assert srv.step() == 0                       # a admitted, 2 iterations, retired
    assert srv.status(a)[0] == lfsr.LFSR_REQ_DONE
    assert srv.status(b)[0] == lfsr.LFSR_REQ_QUEUED and srv.status(c)[0] == lfsr.LFSR_REQ_QUEUED
    st = srv.stats()
    assert st["bytes_in_use"] == 0 and st["bytes_peak"] == big
    srv.step()                                   # b admitted and done; c still behind it
    assert srv.status(b)[0] == lfsr.LFSR_REQ_DONE and srv.status(c)[0] == lfsr.LFSR_REQ_QUEUED
    srv.step()
    assert srv.status(c)[0] == lfsr.LFSR_REQ_DONE
    srv.close()


def test_request_larger_than_the_budget_fails_and_later_ones_proceed():
    srv = lfsr.Server(1 << 20, max_active=4, iterations=1, dry_run=True)
    big = _submit(srv, U=9, V=9, H=64, W=64)
    small = _submit(srv, H=8, W=8)
    srv.step()
    state, _, rc = srv.status(big)
    assert state == lfsr.LFSR_REQ_FAILED and rc == lfsr.LFSR_ENOMEM
    assert srv.status(small)[0] == lfsr.LFSR_REQ_DONE
    srv.close()


def test_requests_share_the_solver_constants():
    srv = lfsr.Server(1 << 40, dry_run=True)
    _submit(srv)
    with pytest.raises(lfsr.LfsrError) as e:
        _submit(srv, mu=7.0)
    assert e.value.code == lfsr.LFSR_EINVAL
    with pytest.raises(lfsr.LfsrError):
        lfsr.Server(0, dry_run=True)             # no budget
    srv.close()


def test_served_requests_take_one_map_and_the_exact_adjoint():
    srv = lfsr.Server(1 << 40, dry_run=True)
    for extra in (dict(adjoint="backward"),
                  dict(disparity_views=np.zeros((9, 32, 32), np.float32))):
        with pytest.raises(lfsr.LfsrError) as e:
            _submit(srv, **extra)
        assert e.value.code == lfsr.LFSR_EUNSUPPORTED
    # the paper's weights (with a projection error, copied at submission) are served
    pe = np.zeros((32, 32), np.float32)
    rid = _submit(srv, weights="paper", sigma_s=8.0, sigma_e=0.1, sigma_o1=1.0, sigma_o2=0.5,
                  proj_err=pe)
    del pe
    assert rid == 0
    srv.close()

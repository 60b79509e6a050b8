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


# --------------------------------------------------------------------------
# failure paths on the host: cancelled requests, injected allocation faults
# --------------------------------------------------------------------------
def test_cancel_queued_active_and_done_requests():
    srv = lfsr.Server(1 << 40, max_active=2, iterations=6, iterations_per_step=2, dry_run=True)
    ids = [_submit(srv) for _ in range(5)]
    assert srv.step() == 2                       # 0 and 1 active
    srv.cancel(3)                                # queued
    srv.cancel(0)                                # active: its slot frees at once
    assert srv.status(0)[0] == lfsr.LFSR_REQ_CANCELLED
    assert srv.status(3)[0] == lfsr.LFSR_REQ_CANCELLED
    st = srv.stats()
    assert st["active"] == 1 and st["queued"] == 2 and st["cancelled"] == 2
    assert srv.step() == 2                       # 2 takes the freed slot; 4 waits
    assert srv.status(2)[:2] == (lfsr.LFSR_REQ_ACTIVE, 2)
    for _ in range(20):
        if srv.stats()["done"] == 3:
            break
        srv.step()
    st = srv.stats()
    assert st["done"] == 3 and st["failed"] == 0 and st["cancelled"] == 2
    assert st["active"] == 0 and st["bytes_in_use"] == 0
    srv.cancel(4)                                # done, not fetched: drops its result
    assert srv.status(4)[0] == lfsr.LFSR_REQ_CANCELLED
    with pytest.raises(lfsr.LfsrError):
        srv.fetch(4, np.zeros((32, 32), np.float32))
    for bad in (0, 4, 99):                       # already cancelled, unknown
        with pytest.raises(lfsr.LfsrError) as e:
            srv.cancel(bad)
        assert e.value.code == lfsr.LFSR_EINVAL
    x = np.zeros((32, 32), np.float32)
    srv.fetch(1, x)
    with pytest.raises(lfsr.LfsrError):          # fetched: nothing left to cancel
        srv.cancel(1)
    assert srv.stats()["cancelled"] == 3
    srv.close()


def test_injected_allocation_fault_fails_one_admission(monkeypatch):
    """LFSR_FAULT=alloc:2 fails the second admission as an allocation error:
    that request fails with LFSR_ENOMEM and holds no slot or budget, the
    others run to the end."""
    y, x0, args = _req()
    est = lfsr.estimate_state_bytes(**args)
    srv = lfsr.Server(4 * est, max_active=3, iterations=4, iterations_per_step=2, dry_run=True)
    ids = [srv.submit(y, x0, **args) for _ in range(4)]
    monkeypatch.setenv("LFSR_FAULT", "alloc:2")
    assert srv.step() == 3                       # 0, 2, 3 admitted; 1 failed
    monkeypatch.delenv("LFSR_FAULT")
    state, _, rc = srv.status(ids[1])
    assert state == lfsr.LFSR_REQ_FAILED and rc == lfsr.LFSR_ENOMEM
    assert srv.stats()["bytes_in_use"] == 3 * est
    while srv.step() > 0:
        pass
    st = srv.stats()
    assert st["done"] == 3 and st["failed"] == 1 and st["bytes_in_use"] == 0
    srv.close()


def test_every_allocation_failing_fails_every_admission(monkeypatch):
    srv = lfsr.Server(1 << 40, max_active=4, iterations=4, iterations_per_step=2, dry_run=True)
    ids = [_submit(srv) for _ in range(3)]
    monkeypatch.setenv("LFSR_FAULT", "alloc")
    assert srv.step() == 0
    assert all(srv.status(i)[2] == lfsr.LFSR_ENOMEM for i in ids)
    monkeypatch.setenv("LFSR_FAULT", "none")     # any other value: no fault
    i = _submit(srv)
    assert srv.step() == 1 and srv.status(i)[0] == lfsr.LFSR_REQ_ACTIVE
    srv.close()


def test_cancel_from_another_thread_while_stepping():
    """The server's entry points may be called from several host threads: a
    cancel issued while another thread steps takes effect between steps."""
    import threading
    srv = lfsr.Server(1 << 40, max_active=4, iterations=40, iterations_per_step=1, dry_run=True)
    ids = [_submit(srv) for _ in range(6)]
    stop = threading.Event()

    def loop():
        while not stop.is_set():
            srv.step()
            st = srv.stats()
            if st["active"] == 0 and st["queued"] == 0:
                break

    t = threading.Thread(target=loop)
    t.start()
    for i in (1, 4, 5):
        try:
            srv.cancel(i)
        except lfsr.LfsrError:
            pass                                 # finished before the cancel
    t.join(timeout=60)
    stop.set()
    assert not t.is_alive()
    st = srv.stats()
    assert st["done"] + st["cancelled"] == 6 and st["failed"] == 0
    assert st["active"] == 0 and st["bytes_in_use"] == 0
    for i in ids:
        assert srv.status(i)[0] in (lfsr.LFSR_REQ_DONE, lfsr.LFSR_REQ_CANCELLED)
    srv.close()

"""Failure paths on the GPU, injected on the host (no device fault):

* an allocation failure (LFSR_FAULT=alloc:K) inside lfsr_create and
  lfsr_batch_create returns LFSR_ENOMEM, and the next create succeeds;
* in the server, a request whose admission fails to allocate and a request
  cancelled while active both free their slot and budget, and the requests
  around them finish with the same results as alone and as the FP64 oracle.
"""
import numpy as np
import pytest

from paper_2206_05047_gb300 import lfsr, synth
from tests.gpu_util import f32, rel_err
from tests.test_gpu_batch import SOLVER, _alone, _jobs
from tests.test_gpu_server import _oracle_x, _requests

load_lib = lfsr.load_library

pytestmark = pytest.mark.gpu


def test_create_returns_enomem_under_an_injected_allocation_fault(monkeypatch):
    wl = synth.custom(U=3, V=3, H=12, W=10, scale=2, kb=5, blur_sigma=1.0, window=3)
    pr = synth.make_problem(wl, seed=1)
    kw = dict(U=wl.U, V=wl.V, H=wl.H, W=wl.W, scale=wl.scale, blur=f32(pr.blur),
              disparity=f32(pr.disparity), **SOLVER)
    for k in (1, 3, 9):
        monkeypatch.setenv("LFSR_FAULT", f"alloc:{k}")
        with pytest.raises(lfsr.LfsrError) as e:
            lfsr.Solver(**kw)
        assert e.value.code == lfsr.LFSR_ENOMEM
    monkeypatch.delenv("LFSR_FAULT")
    x = _alone(kw, pr, 3)                        # creates and solves normally again
    assert rel_err(x, _oracle_x(pr, kw, 3)) <= 1e-4


def test_batch_create_returns_enomem_under_an_injected_allocation_fault(monkeypatch):
    probs, kws = _jobs()
    monkeypatch.setenv("LFSR_FAULT", "alloc")
    with pytest.raises(lfsr.LfsrError) as e:
        lfsr.Batch(kws[:2])
    assert e.value.code == lfsr.LFSR_ENOMEM
    monkeypatch.delenv("LFSR_FAULT")
    b = lfsr.Batch(kws[:2])
    assert load_lib().lfsr_batch_size(b.handle) == 2
    b.close()


def test_served_requests_survive_a_failed_admission_and_a_cancel(monkeypatch):
    reqs = _requests()[:5]
    n_iter = 7
    srv = lfsr.Server(8 << 30, max_active=4, iterations=n_iter, iterations_per_step=2)
    ids = [srv.submit(f32(pr.y), f32(pr.x0), **kw) for pr, kw in reqs[:3]]
    srv.step()                                   # 0, 1, 2 active, 2 iterations
    srv.cancel(ids[1])                           # active: state freed at once
    assert srv.status(ids[1])[0] == lfsr.LFSR_REQ_CANCELLED
    # the next admission fails to allocate: its first device allocation
    monkeypatch.setenv("LFSR_FAULT", "alloc:1")
    ids.append(srv.submit(f32(reqs[3][0].y), f32(reqs[3][0].x0), **reqs[3][1]))
    srv.step()
    monkeypatch.delenv("LFSR_FAULT")
    state, _, rc = srv.status(ids[3])
    assert state == lfsr.LFSR_REQ_FAILED and rc == lfsr.LFSR_ENOMEM
    ids.append(srv.submit(f32(reqs[4][0].y), f32(reqs[4][0].x0), **reqs[4][1]))
    for _ in range(50):
        st = srv.stats()
        if st["active"] == 0 and st["queued"] == 0:
            break
        srv.step()
    st = srv.stats()
    assert st["done"] == 3 and st["failed"] == 1 and st["cancelled"] == 1
    assert st["bytes_in_use"] == 0
    for k in (0, 2, 4):
        pr, kw = reqs[k]
        x = np.zeros(pr.wl.HR, np.float32)
        srv.fetch(ids[k], x)
        assert rel_err(x, _alone(kw, pr, n_iter)) <= 1e-5, k
        assert rel_err(x, _oracle_x(pr, kw, n_iter)) <= 1e-4, k
    srv.close()

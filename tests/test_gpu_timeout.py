"""The fused CG step (normal-matrix product, grid barrier, step length and
vector update, grid barrier, beta: one cooperative launch per CG step) and
its bounded waits.

* The launch count per ADMM iteration is 2 + 2K with the specialised
  operator kernel (the x-step initialisation lives in the data-block launch,
  the CG update in the normal-matrix launch) and 3 + 3K on the generic
  path.
* A wait that cannot complete (every barrier waits for one arrival more
  than the launch has) gives up after its limit: the solve reports
  LFSR_ETIMEOUT, the context stays usable, and the next solve with the
  default limit matches the FP64 oracle.
"""
import numpy as np
import pytest

from paper_2206_05047_gb300 import lfsr, synth
from tests.gpu_util import Case, rel_err

pytestmark = pytest.mark.gpu


def _solve(c, n):
    x = c.empty(*c.oracle.hr)
    lfsr.solve(c.h, c.t(c.y), n, c.t(c.x0), x)
    return c.np(x)


def test_fused_cg_step_launch_count_and_parity():
    wl = synth.custom(U=5, V=5, H=19, W=21, scale=2, kb=5, blur_sigma=1.0, window=5,
                      iterations=6)
    c = Case(wl, seed=12)
    n = wl.iterations
    got = _solve(c, n)
    st = lfsr.stats(c.h)
    assert st["launches"] == n * (2 + 2 * wl.cg_iters)
    assert st["status"] == 0 and st["cg_steps"] == wl.cg_iters
    ref, _, _ = c.oracle.admm(c.y.astype(np.float64), c.x0.astype(np.float64), n)
    assert rel_err(got, ref) <= 1e-4
    c.solver.close()


def test_generic_path_keeps_the_update_launch():
    wl = synth.custom(U=3, V=3, H=12, W=14, scale=2, kb=5, blur_sigma=1.0, window=3,
                      iterations=3)
    k = np.random.default_rng(4).random((5, 5)) + 0.1
    c = Case(wl, seed=3, blur=k / k.sum())          # non-separable: generic kernel
    _solve(c, wl.iterations)
    assert lfsr.stats(c.h)["launches"] == wl.iterations * (3 + 3 * wl.cg_iters)
    c.solver.close()


def test_a_wait_that_cannot_complete_times_out_and_the_handle_recovers():
    wl = synth.custom(U=5, V=5, H=22, W=20, scale=2, kb=5, blur_sigma=1.0, window=5,
                      iterations=4)
    c = Case(wl, seed=5)
    lfsr.set_device_wait(c.h, 2_000_000, test_unreachable=True)     # 2 ms, never released
    with pytest.raises(lfsr.LfsrError) as e:
        _solve(c, 2)
    assert e.value.code == lfsr.LFSR_ETIMEOUT
    assert "gave up" in lfsr.last_error(c.h)
    assert lfsr.stats(c.h)["status"] == lfsr.LFSR_ETIMEOUT
    # the default limit again: a fresh solve is exact, twice in a row
    lfsr.set_device_wait(c.h)
    ref, _, _ = c.oracle.admm(c.y.astype(np.float64), c.x0.astype(np.float64), wl.iterations)
    for _ in range(2):
        got = _solve(c, wl.iterations)
        assert lfsr.stats(c.h)["status"] == 0
        assert rel_err(got, ref) <= 1e-4
    c.solver.close()

"""Cost-balanced ranges of the operator launches.

lfsr_create (and a batch that owns its light fields, for each operator
group) times every (64 x 64 tile, view pair) unit of one normal-matrix
launch and splits the units over the CTAs in contiguous ranges of equal
measured cost.  The split changes only which CTA runs a unit (and so the
order of the float atomic additions):

* a light field with enough units reports both load-balance figures, the
  balanced one no worse than the even split's, alone and in a batch;
* its solve matches the FP64 oracle, the batch, and the server (whose
  batch keeps the even split);
* a light field with fewer than two units per CTA keeps the even split and
  reports no measurement.
"""
import numpy as np
import pytest

from paper_2206_05047_gb300 import lfsr, synth
from tests.gpu_util import Case, f32, rel_err

pytestmark = pytest.mark.gpu


def _solve(c, n):
    x = c.empty(*c.oracle.hr)
    lfsr.solve(c.h, c.t(c.y), n, c.t(c.x0), x)
    return c.np(x)


def test_balanced_ranges_match_the_oracle_and_the_even_split():
    # 9 x 9 views, 128^2 -> 256^2: 16 tiles x 41 view pairs = 656 units
    wl = synth.custom(U=9, V=9, H=128, W=128, scale=2, kb=7, blur_sigma=1.2, window=7,
                      disparities=tuple(np.linspace(-2.0, 2.0, 5)), iterations=2)
    c = Case(wl, seed=31)
    st = lfsr.stats(c.h)
    assert st["op_split_even"] >= 1.0
    assert 1.0 <= st["op_split_balanced"] <= st["op_split_even"]
    n = wl.iterations
    got = _solve(c, n)
    assert lfsr.stats(c.h)["status"] == 0
    ref, _, _ = c.oracle.admm(c.y.astype(np.float64), c.x0.astype(np.float64), n)
    assert rel_err(got, ref) <= 1e-4
    kw = dict(U=wl.U, V=wl.V, H=wl.H, W=wl.W, scale=wl.scale, blur=c.blur, disparity=c.disp,
              lambda1=wl.lambda1, lambda2=wl.lambda2, mu=wl.mu, nltv_window=wl.window,
              nltv_patch=wl.patch, nltv_h=wl.h, cg_iters=wl.cg_iters, cg_tol=0.0)
    # the same light field in a batch table, its group balanced
    b = lfsr.Batch([kw])
    bs = b.stats(0)
    assert 1.0 <= bs["op_split_balanced"] <= bs["op_split_even"]
    b.load(0, c.t(c.y), c.t(c.x0))
    b.iterate(n)
    xb = c.empty(*c.oracle.hr)
    b.get_x(0, xb)
    assert rel_err(c.np(xb), got) <= 1e-5
    b.close()
    # ... and served: the server's batch keeps the even split
    srv = lfsr.Server(8 << 30, max_active=2, iterations=n, iterations_per_step=1)
    rid = srv.submit(c.y, c.x0, **kw)
    for _ in range(4 * n):
        if srv.status(rid)[0] == lfsr.LFSR_REQ_DONE:
            break
        srv.step()
    xs = np.zeros(c.oracle.hr, np.float32)
    srv.fetch(rid, xs)
    assert rel_err(xs, got) <= 1e-5
    srv.close()
    c.solver.close()


def test_few_units_keep_the_even_split():
    wl = synth.custom(U=3, V=3, H=12, W=10, scale=2, kb=5, blur_sigma=1.0, window=3)
    pr = synth.make_problem(wl, seed=2)
    s = lfsr.Solver(U=wl.U, V=wl.V, H=wl.H, W=wl.W, scale=wl.scale, blur=f32(pr.blur),
                    disparity=f32(pr.disparity), lambda1=2.0, lambda2=4.0, mu=300.0,
                    nltv_window=3, nltv_patch=3, nltv_h=0.1, cg_iters=5, cg_tol=0.0)
    st = lfsr.stats(s.handle)
    assert st["op_split_even"] == 0.0 and st["op_split_balanced"] == 0.0
    s.close()

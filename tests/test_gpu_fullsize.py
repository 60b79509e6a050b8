"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times (graph-captured lfsr_load + lfsr_iterate on the same plan).

* every operator of one ADMM iteration at full size against the oracle;
* the first iterations of the 9x9-view x2 and x3 light fields against the
  oracle (x, both dual blocks), the whole 100-iteration solve of the
  9x9-view x2 light field at its configured h = 0.1 against the oracle run
  here, and of the x3 light field against the oracle's stored iterate
  (tests/golden/, written by make_golden.py: minutes of oracle);
* properties that hold at any N: a constant image stays fixed, duals stay in
  [-1/mu, 1/mu].
"""
import numpy as np
import pytest

from paper_2206_05047_gb300 import lfsr, synth
from tests.gpu_util import Case, check_golden_inputs, f32, golden, max_err, rel_err

pytestmark = pytest.mark.gpu

FULL = ["lf9x9_256_x2", "lf9x9_200_x3"]


@pytest.fixture(scope="module", params=FULL)
def full_case(request):
    c = Case(synth.WORKLOADS[request.param], seed=2000)
    yield c
    c.solver.close()


def test_full_size_operators(full_case):
    c = full_case
    o, wl = c.oracle, c.wl
    x = c.x0
    out = c.empty(o.s_k, wl.H, wl.W)
    lfsr.apply_A(c.h, -1, c.t(x), out)
    got = c.np(out)
    for k in (0, o.s_k // 2, o.s_k - 1, 17):
        assert max_err(got[k], o.A(k, x.astype(np.float64))) <= 2e-6, k
    g = f32(np.random.default_rng(0).standard_normal((wl.H, wl.W)))
    outT = c.empty(*o.hr)
    for k in (0, 40, o.s_k - 1):
        lfsr.apply_AT(c.h, k, c.t(g), outT)
        assert max_err(c.np(outT), o.A_T(k, g.astype(np.float64))) <= 2e-6, k
    w = c.empty(o.s_d, *o.hr)
    lfsr.weights(c.h, c.t(x), w)
    wref = o.weights(x.astype(np.float64))
    assert np.abs(c.np(w) - wref).max() <= 3e-5
    p = f32(np.random.default_rng(1).standard_normal(o.hr))
    q = c.empty(*o.hr)
    pMp = lfsr.apply_normal(c.h, c.t(x), c.t(p), q)
    qref = o.normal_apply(wref, p.astype(np.float64))
    assert max_err(c.np(q), qref) <= 5e-6
    assert abs(pMp - float(np.vdot(p, qref))) <= 2e-6 * abs(float(np.vdot(p, qref)))


def test_full_size_first_iterations(full_case):
    c = full_case
    n = 2 if c.wl.scale == 2 else 1
    lfsr.load(c.h, c.t(c.y), c.t(c.x0))
    lfsr.iterate(c.h, n)
    x = c.empty(*c.oracle.hr)
    wA = c.empty(c.oracle.s_k, c.wl.H, c.wl.W)
    wS = c.empty(c.oracle.s_d, *c.oracle.hr)
    lfsr.get_state(c.h, x, wA, wS)
    rx, rA, rS = c.oracle.admm(c.y.astype(np.float64), c.x0.astype(np.float64), n)
    assert rel_err(c.np(x), rx) <= 1e-4
    assert rel_err(c.np(wA), rA) <= 1e-4
    assert rel_err(c.np(wS), rS) <= 1e-4


def test_full_size_constant_image_and_dual_bounds():
    """x0 = c with noise-free views y_k = A_k c (oracle): the GPU iterate stays
    at c through a full 100-iteration solve; every dual stays in [-1/mu, 1/mu]."""
    wl = synth.WORKLOADS["lf9x9_256_x2"]
    c = Case(wl, seed=2000)
    o = c.oracle
    cst = np.full(o.hr, 0.4375)
    y = f32(np.stack([o.A(k, cst) for k in range(o.s_k)]))
    x = c.empty(*o.hr)
    lfsr.solve(c.h, c.t(y), wl.iterations, c.t(cst), x)
    assert np.abs(c.np(x) - cst).max() <= 1e-5
    # dual bounds on the real data
    lfsr.load(c.h, c.t(c.y), c.t(c.x0))
    lfsr.iterate(c.h, 7)
    wA = c.empty(o.s_k, wl.H, wl.W)
    wS = c.empty(o.s_d, *o.hr)
    lfsr.get_state(c.h, None, wA, wS)
    t = float(np.float32(1.0 / wl.mu))          # the kernels' float threshold
    assert c.np(wA).max() <= t and c.np(wA).min() >= -t
    assert c.np(wS).max() <= t and c.np(wS).min() >= -t
    assert lfsr.stats(c.h)["status"] == 0
    c.solver.close()


def _full_n(name, seed):
    wl = synth.WORKLOADS[name]
    c = Case(wl, seed=seed)
    x = c.empty(*c.oracle.hr)
    lfsr.solve(c.h, c.t(c.y), wl.iterations, c.t(c.x0), x)
    ref, _, _ = c.oracle.admm(c.y.astype(np.float64), c.x0.astype(np.float64), wl.iterations)
    gx = c.np(x)
    assert rel_err(gx, ref) <= 1e-4
    assert abs(synth.psnr(gx, c.prob.gt) - synth.psnr(ref, c.prob.gt)) <= 0.01
    assert synth.psnr(ref, c.prob.gt) > synth.psnr(c.x0, c.prob.gt) + 3.0
    c.solver.close()


def test_full_size_full_N_lf9x9_256_x2():
    """The benchmark workload, all 100 iterations at its configured h = 0.1."""
    _full_n("lf9x9_256_x2", 2000)


def test_full_size_full_N_lf9x9_200_x3():
    """The x3 task (Sec. 6): 9x9 views, 200^2 -> 600^2, 9x9 blur, all 100
    iterations, against the oracle's stored float64 iterate."""
    name, seed = "lf9x9_200_x3", 3000
    wl = synth.WORKLOADS[name]
    g = golden(name, seed, wl.iterations)
    c = Case(wl, seed=seed)
    check_golden_inputs(c, g)
    x = c.empty(*c.oracle.hr)
    lfsr.solve(c.h, c.t(c.y), wl.iterations, c.t(c.x0), x)
    gx, ref = c.np(x), g["x"]
    assert rel_err(gx, ref) <= 1e-4
    assert abs(synth.psnr(gx, c.prob.gt) - float(g["psnr_x"])) <= 0.01
    assert float(g["psnr_x"]) > float(g["psnr_x0"]) + 3.0
    c.solver.close()

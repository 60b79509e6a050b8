"""The data-term variants the paper compares (Sec. 6.1): l1 only
(lambda2 = 0, as in its MISR runs), l2 only (lambda1 = 0) and the joint
l1-l2 term, on the specialised and the generic operator kernels, against
the FP64 oracle (tolerances of test_gpu_parity.py)."""
import numpy as np
import pytest

from paper_2206_05047_gb300 import lfsr, synth
from tests.gpu_util import Case, f32, rel_err

pytestmark = pytest.mark.gpu

TERMS = {"l1_only": dict(lambda1=2.0, lambda2=0.0), "l2_only": dict(lambda1=0.0, lambda2=4.0)}
GEOMS = {
    "x2_5x5": (dict(U=5, V=5, H=21, W=19, scale=2, kb=5, blur_sigma=1.0, window=5,
                    disparities=(-1.0, 0.0, 0.8)), False),
    "x4_nonsep": (dict(U=3, V=3, H=9, W=10, scale=4, kb=5, blur_sigma=1.0, window=7,
                       disparities=(-0.6, 1.2)), True),
}


def _case(geom, term):
    ov, nonsep = GEOMS[geom]
    kw = {}
    if nonsep:
        K = np.random.default_rng(9).random((5, 5)) ** 3
        kw["blur"] = K / K.sum()
    return Case(synth.custom(**ov), seed=0, **kw, **TERMS[term])


@pytest.mark.parametrize("geom", list(GEOMS))
@pytest.mark.parametrize("term", list(TERMS))
def test_solve(geom, term):
    c = _case(geom, term)
    o = c.oracle
    n_iter = 12
    x = c.empty(*o.hr)
    lfsr.solve(c.h, c.t(c.y), n_iter, c.t(c.x0), x)
    ref, rA, _ = o.admm(c.y.astype(np.float64), c.x0.astype(np.float64), n_iter)
    assert rel_err(c.np(x), ref) <= 1e-4
    assert abs(synth.psnr(c.np(x), c.prob.gt) - synth.psnr(ref, c.prob.gt)) <= 0.01
    wA = c.empty(*rA.shape)
    lfsr.get_state(c.h, None, wA, None)
    if term == "l2_only":
        assert not c.np(wA).any()               # the data duals never move
    else:
        assert rel_err(c.np(wA), rA) <= 1e-4

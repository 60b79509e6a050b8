"""The stored FP64 oracle iterates of tests/golden/ belong to the inputs the
generator makes today: regenerating the workload at the stored seed gives
the stored checksums, and the stored solver parameters are the workload's.
(The iterates themselves come from tests/golden/make_golden.py, which runs
the oracle alone.)"""
import os

import numpy as np
import pytest

from paper_2206_05047_gb300 import synth
from tests.gpu_util import golden

GOLDEN = [("lf9x9_200_x3", 3000)]


@pytest.mark.parametrize("name,seed", GOLDEN)
def test_golden_matches_regenerated_inputs(name, seed):
    from tests.golden.make_golden import checksums, inputs
    wl = synth.WORKLOADS[name]
    g = golden(name, seed, wl.iterations)
    assert str(g["workload"]) == name and int(g["seed"]) == seed
    assert int(g["iterations"]) == wl.iterations
    for k in ("lambda1", "lambda2", "mu", "h"):
        assert float(g[k]) == float(getattr(wl, k)), k
    for k in ("window", "patch", "cg_iters"):
        assert int(g[k]) == int(getattr(wl, k)), k
    _, prob, a = inputs(name, seed)
    for key, val in checksums(a).items():
        ref = float(g[key])
        assert abs(val - ref) <= 1e-6 * max(abs(ref), 1.0), key
    x = g["x"]
    assert x.shape == wl.HR and x.dtype == np.float64 and np.isfinite(x).all()
    # the stored iterate is the reconstruction its PSNR says, and beats bicubic
    assert abs(synth.psnr(x, prob.gt) - float(g["psnr_x"])) <= 1e-9
    assert float(g["psnr_x"]) > float(g["psnr_x0"]) + 3.0


def test_golden_directory_holds_only_listed_files():
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    names = {f for f in os.listdir(here) if f.endswith(".npz")}
    want = {f"{n}_seed{s}_n{synth.WORKLOADS[n].iterations}.npz" for n, s in GOLDEN}
    assert names == want

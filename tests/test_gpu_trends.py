"""Synthetic analogues of the paper's experimental trends (Sec. 6.1) on the
CUDA path -- the paper's datasets are not available, so these check the
direction of each effect on seeded synthetic light fields, not its numbers:
the joint l1-l2 data term beats either term alone under mixed noise, PSNR
rises with the number of input views, and the NLTV weights computed from
the iterate approach those of the ground truth as the iterations proceed."""
import numpy as np
import pytest

from paper_2206_05047_gb300 import lfsr, synth

pytestmark = pytest.mark.gpu


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to("cuda:0")


def _solve(pr, n, views=None, **kw):
    import torch
    s = lfsr.Solver(pr, views=views, **kw)
    x = torch.empty(pr.wl.HR, dtype=torch.float32, device="cuda:0")
    y = pr.y if views is None else pr.y[np.asarray(views)]
    lfsr.solve(s.handle, _t(y), n, _t(pr.x0), x)
    s.close()
    return x.cpu().numpy().astype(np.float64)


def test_joint_data_term_beats_either_term_alone():
    """Sec. 6.1's l1 / l2 / l1+l2 comparison under Gaussian + impulse noise
    (5x5 views, 64^2 -> 128^2, 50 iterations); each single term also at a
    stronger weight."""
    wl = synth.WORKLOADS["lf5x5_64_x2"]
    pr = synth.make_problem(wl, seed=0)
    joint = synth.psnr(_solve(pr, wl.iterations), pr.gt)
    singles = [synth.psnr(_solve(pr, wl.iterations, lambda1=l1, lambda2=l2), pr.gt)
               for l1, l2 in ((2.0, 0.0), (4.0, 0.0), (0.0, 4.0), (0.0, 16.0))]
    assert joint > max(singles) + 1.0, (joint, singles)


def test_psnr_rises_with_the_number_of_views():
    """Sec. 6.1's PSNR against the number of input views: centred square
    subsets of a 7 x 7 grid (1, 9, 25 and 49 views) of one scene."""
    wl = synth.custom(U=7, V=7, H=64, W=64, scale=2, kb=5, blur_sigma=1.0,
                      disparities=(-1.0, 0.0, 0.8), noise_sigma=0.02, impulse=0.05, window=5)
    pr = synth.make_problem(wl, seed=1)
    p = {}
    for r in (0, 1, 2, 3):
        views = [v * 7 + u for v in range(3 - r, 4 + r) for u in range(3 - r, 4 + r)]
        p[len(views)] = synth.psnr(_solve(pr, 50, views=views), pr.gt)
    assert p[1] + 3.0 < p[9] < p[25], p
    assert p[49] > p[25] - 0.5, p


def test_weights_approach_those_of_the_ground_truth():
    """The weight maps sharpen over the iterations (Sec. 6.1's weight-map
    figure): the distance between the weights of the iterate and those of
    the ground truth falls."""
    import torch
    wl = synth.WORKLOADS["lf5x5_64_x2"]
    pr = synth.make_problem(wl, seed=0)
    s = lfsr.Solver(pr)
    w_gt = torch.empty((wl.s_d,) + wl.HR, dtype=torch.float32, device="cuda:0")
    lfsr.weights(s.handle, _t(pr.gt), w_gt)
    errs = []
    for n in (0, 5, 20, 50):
        x = pr.x0 if n == 0 else _solve(pr, n)
        w = torch.empty_like(w_gt)
        lfsr.weights(s.handle, _t(x), w)
        errs.append(float(torch.linalg.norm(w - w_gt) / torch.linalg.norm(w_gt)))
    s.close()
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 0.75 * errs[0], errs

"""Writes the stored FP64 reference iterates of tests/golden/ with the
oracle alone (no CUDA code is imported or run).

    python tests/golden/make_golden.py lf9x9_200_x3 3000

For a named workload and seed: the seeded synthetic inputs (float32, as the
GPU tests pass them; the oracle reads their float64 images), then N ADMM
iterations of the FP64 oracle (Algorithm 1 with the K-step CG x-step of
Algorithm 2), then an .npz holding x_N in float64, the PSNR of x_N and of
the bicubic start against the ground truth, and float64 checksums of the
inputs (sum and sum of squares of y, x0, the disparity map and the blur),
by which a test confirms that it regenerated the same inputs.

The x3 workload (9 x 9 views, 200^2 -> 600^2, 9 x 9 blur, 100 iterations)
takes minutes of oracle on a host's cores; its iterate is stored so that
the GPU parity test at the full iteration count runs in seconds.
"""
import hashlib
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def checksums(arrays):
    out = {}
    for name, a in arrays.items():
        a64 = np.asarray(a, np.float64)
        out[f"sum_{name}"] = float(a64.sum())
        out[f"sumsq_{name}"] = float((a64 * a64).sum())
    return out


def inputs(name, seed):
    from paper_2206_05047_gb300 import synth
    wl = synth.WORKLOADS[name]
    prob = synth.make_problem(wl, seed=seed)
    f = lambda a: np.ascontiguousarray(np.asarray(a, np.float32))
    return wl, prob, dict(y=f(prob.y), x0=f(prob.x0), disp=f(prob.disparity), blur=f(prob.blur))


def path_for(name, seed, n):
    return os.path.join(HERE, f"{name}_seed{seed}_n{n}.npz")


def main(name, seed, n=None):
    from oracle import oracle as om
    from paper_2206_05047_gb300 import synth
    wl, prob, a = inputs(name, seed)
    n = wl.iterations if n is None else n
    o = om.Oracle(wl.U, wl.V, wl.H, wl.W, wl.scale, a["blur"].astype(np.float64),
                  a["disp"].astype(np.float64), lambda1=wl.lambda1, lambda2=wl.lambda2,
                  mu=wl.mu, window=wl.window, patch=wl.patch, h=wl.h, cg_iters=wl.cg_iters)
    t0 = time.time()
    x, _, _ = o.admm(a["y"].astype(np.float64), a["x0"].astype(np.float64), n)
    dt = time.time() - t0
    meta = checksums(a)
    sha = hashlib.sha256(b"".join(a[k].tobytes() for k in ("y", "x0", "disp", "blur")))
    np.savez_compressed(
        path_for(name, seed, n), x=x, workload=name, seed=seed, iterations=n,
        lambda1=wl.lambda1, lambda2=wl.lambda2, mu=wl.mu, window=wl.window, patch=wl.patch,
        h=wl.h, cg_iters=wl.cg_iters, psnr_x=synth.psnr(x, prob.gt),
        psnr_x0=synth.psnr(a["x0"], prob.gt), inputs_sha256=sha.hexdigest(),
        oracle_threads=om.num_threads(), oracle_seconds=dt,
        **{k: np.float64(v) for k, v in meta.items()})
    print(f"{name} seed {seed}: {n} iterations in {dt:.1f} s, PSNR {synth.psnr(x, prob.gt):.3f} "
          f"dB (bicubic {synth.psnr(a['x0'], prob.gt):.3f}) -> {path_for(name, seed, n)}")


if __name__ == "__main__":
    main(sys.argv[1], int(sys.argv[2]), int(sys.argv[3]) if len(sys.argv) > 3 else None)

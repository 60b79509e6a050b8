"""Helpers shared by the GPU parity tests: build the same float32 inputs for
the CUDA path and (as float64) for the oracle."""
import numpy as np

from paper_2206_05047_gb300 import synth


def f32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def rel_err(a, ref):
    a = np.asarray(a, np.float64)
    ref = np.asarray(ref, np.float64)
    return float(np.linalg.norm(a - ref) / max(np.linalg.norm(ref), 1e-30))


def round_f16(a):
    """Round-to-nearest-even float32 -> IEEE half -> float32 (numpy's cast)."""
    return np.asarray(a, np.float32).astype(np.float16).astype(np.float32)


def round_bf16(a):
    """Round-to-nearest-even float32 -> bfloat16 -> float32, on the bits
    (finite inputs)."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


ROUND = {"fp32": lambda a: np.asarray(a, np.float32), "fp16": round_f16, "bf16": round_bf16}


def max_err(a, ref):
    a = np.asarray(a, np.float64)
    ref = np.asarray(ref, np.float64)
    return float(np.abs(a - ref).max() / max(np.abs(ref).max(), 1e-30))


class Case:
    """One problem: float32 arrays, an oracle on their float64 images and a
    GPU solver on the same float32 values."""

    def __init__(self, wl, seed=0, blur=None, disparity=None, precision="fp32", views=None,
                 weights="patch", sigmas=None, proj_err=None, disparity_views=None,
                 adjoint="exact", **overrides):
        import torch
        from oracle import oracle as om
        from paper_2206_05047_gb300 import lfsr
        self.wl = wl
        self.prob = synth.make_problem(wl, seed=seed)
        self.blur = f32(self.prob.blur if blur is None else blur)
        self.disp = f32(self.prob.disparity if disparity is None else disparity)
        self.views = None if views is None else np.asarray(views, np.int32)
        self.y = f32(self.prob.y if views is None else self.prob.y[self.views])
        self.x0 = f32(self.prob.x0)
        self.params = dict(lambda1=wl.lambda1, lambda2=wl.lambda2, mu=wl.mu, window=wl.window,
                           patch=wl.patch, h=wl.h, cg_iters=wl.cg_iters, cg_tol=0.0)
        self.params.update(overrides)
        p = self.params
        # the paper's weights: sigmas as float32 (the C ABI's type) on both sides
        sg = {k: float(np.float32(v)) for k, v in (sigmas or {}).items()}
        self.proj_err = None if proj_err is None else f32(proj_err)
        self.disp_views = None if disparity_views is None else f32(disparity_views)
        wkw = dict(weights=weights, adjoint=adjoint, **sg)
        self.oracle = om.Oracle(wl.U, wl.V, wl.H, wl.W, wl.scale, self.blur.astype(np.float64),
                                self.disp.astype(np.float64), views=self.views,
                                proj_err=None if proj_err is None
                                else self.proj_err.astype(np.float64),
                                disparity_views=None if disparity_views is None
                                else self.disp_views.astype(np.float64), **wkw, **p)
        self.solver = lfsr.Solver(U=wl.U, V=wl.V, H=wl.H, W=wl.W, scale=wl.scale, blur=self.blur,
                                  disparity=self.disp, lambda1=p["lambda1"], lambda2=p["lambda2"],
                                  mu=p["mu"], nltv_window=p["window"], nltv_patch=p["patch"],
                                  nltv_h=p["h"], cg_iters=p["cg_iters"], cg_tol=p["cg_tol"],
                                  precision=precision, views=self.views,
                                  proj_err=self.proj_err, disparity_views=self.disp_views,
                                  **wkw)
        self.h = self.solver.handle
        self.torch = torch
        self.dev = torch.device("cuda:0")

    def t(self, a):
        return self.torch.from_numpy(f32(a)).to(self.dev)

    def empty(self, *shape):
        return self.torch.empty(*shape, dtype=self.torch.float32, device=self.dev)

    @staticmethod
    def np(t):
        return t.detach().cpu().numpy().astype(np.float64)


def golden(name, seed, n):
    """The stored FP64 oracle iterate of tests/golden/ for (workload, seed,
    N), written by tests/golden/make_golden.py, as a dict."""
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                        f"{name}_seed{seed}_n{n}.npz")
    with np.load(path) as z:
        return {k: z[k] for k in z.files}


def check_golden_inputs(c, g):
    """The case regenerated the inputs the golden iterate was computed from
    (float64 checksums; tolerant of last-bit differences of the host's libm,
    which move the iterate far below the parity tolerances)."""
    for name, a in (("y", c.y), ("x0", c.x0), ("disp", c.disp), ("blur", c.blur)):
        a64 = np.asarray(a, np.float64)
        for key, val in ((f"sum_{name}", a64.sum()), (f"sumsq_{name}", (a64 * a64).sum())):
            ref = float(g[key])
            assert abs(val - ref) <= 1e-6 * max(abs(ref), 1.0), (key, val, ref)

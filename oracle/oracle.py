"""ctypes binding of the FP64 CPU oracle (``oracle/lfsr_oracle.c``).

TEST INFRASTRUCTURE ONLY.  The oracle is the plain, slow reference that the
CUDA path is checked against; only the tests, the smoke check and the
benchmark's CPU-baseline leg may use it.  It shares no code with the CUDA
library.  All arrays are float64, row-major; HR images are
(zeta*H) x (zeta*W), LR stacks s_k x H x W, weights / duals s_d x HR.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lfsr_oracle.c")
_LIB = os.path.join(_HERE, "liblfsr_oracle.so")

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP) into oracle/liblfsr_oracle.so."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "lfsr_oracle.h"))):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-Wall", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Problem(C.Structure):
    _fields_ = [("U", C.c_int), ("V", C.c_int), ("H", C.c_int), ("W", C.c_int),
                ("zeta", C.c_int), ("kb", C.c_int),
                ("blur", C.POINTER(C.c_double)), ("disp", C.POINTER(C.c_double)),
                ("lambda1", C.c_double), ("lambda2", C.c_double), ("mu", C.c_double),
                ("window", C.c_int), ("patch", C.c_int), ("h", C.c_double),
                ("cg_iters", C.c_int), ("cg_tol", C.c_double),
                ("freeze_weights", C.c_int), ("n_views", C.c_int),
                ("views", C.POINTER(C.c_int)),
                ("weight_scheme", C.c_int), ("sigma_s", C.c_double), ("sigma_e", C.c_double),
                ("sigma_o1", C.c_double), ("sigma_o2", C.c_double),
                ("proj_err", C.POINTER(C.c_double)),
                ("disp_views", C.POINTER(C.c_double)), ("adjoint", C.c_int)]


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        P = C.POINTER(_Problem)
        sig = {
            "orc_num_threads": (C.c_int, []),
            "orc_set_threads": (None, [C.c_int]),
            "orc_num_dirs": (C.c_int, [P]),
            "orc_dirs": (None, [P, np.ctypeslib.ndpointer(np.int32), np.ctypeslib.ndpointer(np.int32)]),
            "orc_warp": (None, [P, C.c_int, _dp, _dp]),
            "orc_warp_T": (None, [P, C.c_int, _dp, _dp]),
            "orc_warp_bw": (None, [P, C.c_int, _dp, _dp]),
            "orc_blur": (None, [P, _dp, _dp]),
            "orc_blur_T": (None, [P, _dp, _dp]),
            "orc_down": (None, [P, _dp, _dp]),
            "orc_up": (None, [P, _dp, _dp]),
            "orc_A": (None, [P, C.c_int, _dp, _dp]),
            "orc_A_T": (None, [P, C.c_int, _dp, _dp]),
            "orc_weights": (None, [P, _dp, _dp]),
            "orc_edge_factor": (None, [P, _dp, _dp]),
            "orc_occlusion_factor": (None, [P, _dp]),
            "orc_S": (None, [P, _dp, _dp, _dp]),
            "orc_S_T": (None, [P, _dp, _dp, _dp]),
            "orc_prox": (None, [C.c_long, _dp, C.c_double, _dp]),
            "orc_normal_apply": (None, [P, _dp, _dp, _dp]),
            "orc_cost": (C.c_double, [P, _dp, _dp, _dp]),
            "orc_cg": (C.c_int, [P, _dp, _dp, _dp, C.c_int, C.c_double, C.POINTER(C.c_double)]),
            "orc_admm": (C.c_int, [P, _dp, _dp, C.c_int, _dp, _dp, _dp, C.c_void_p]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def num_threads() -> int:
    return _load().orc_num_threads()


def set_threads(n: int) -> None:
    _load().orc_set_threads(int(n))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


class Oracle:
    """One light-field problem (geometry, blur, disparity, solver weights)."""

    def __init__(self, U, V, H, W, zeta, blur, disparity, lambda1=1.0, lambda2=4.0,
                 mu=1.0, window=5, patch=3, h=0.1, cg_iters=5, cg_tol=0.0,
                 freeze_weights=False, views=None, weights="patch", sigma_s=0.0, sigma_e=0.0,
                 sigma_o1=0.0, sigma_o2=0.0, proj_err=None, disparity_views=None,
                 adjoint="exact"):
        self._lib = _load()
        self.blur = _f64(blur)
        kb = self.blur.shape[0]
        assert self.blur.shape == (kb, kb) and kb % 2 == 1
        self.disp = _f64(disparity)
        assert self.disp.shape == (zeta * H, zeta * W)
        self.U, self.V, self.H, self.W, self.zeta = U, V, H, W, zeta
        # views: grid indices k = v*U + u of the views used (Sec. 6.1 uses a
        # star of 17 of 5 x 5), ascending; None: the full grid
        self.views = None if views is None else np.ascontiguousarray(views, dtype=np.int32)
        if self.views is not None:
            assert self.views.ndim == 1 and len(self.views) >= 1
            assert (np.diff(self.views) > 0).all() and self.views[0] >= 0
            assert self.views[-1] < U * V
        self.s_k = U * V if self.views is None else len(self.views)
        # weights: "patch" (exp(-pd/h^2)) or "paper" (Sec. 3.4: spatial *
        # edge * occlusion, each factor with sigma 0 is 1); proj_err: the
        # HR projection error p of the occlusion factor (None: 0)
        assert weights in ("patch", "paper")
        self.proj_err = None if proj_err is None else _f64(proj_err)
        if self.proj_err is not None:
            assert self.proj_err.shape == (zeta * H, zeta * W)
        # warps (Sec. 4.1): disparity_views = per-view maps omega_k (s_k x HR,
        # data order; None: the shared map); adjoint "exact" (scatter) or
        # "backward" (the paper's backward warp by the reference map)
        assert adjoint in ("exact", "backward")
        self.disp_views = None if disparity_views is None else _f64(disparity_views)
        if self.disp_views is not None:
            assert self.disp_views.shape == (self.s_k, zeta * H, zeta * W)
        self.hr = (zeta * H, zeta * W)
        self.p = zeta * H * zeta * W
        self.q = H * W
        self._P = _Problem(U, V, H, W, zeta, kb,
                           self.blur.ctypes.data_as(C.POINTER(C.c_double)),
                           self.disp.ctypes.data_as(C.POINTER(C.c_double)),
                           lambda1, lambda2, mu, window, patch, h, cg_iters, cg_tol,
                           int(bool(freeze_weights)),
                           0 if self.views is None else len(self.views),
                           None if self.views is None
                           else self.views.ctypes.data_as(C.POINTER(C.c_int)),
                           int(weights == "paper"), sigma_s, sigma_e, sigma_o1, sigma_o2,
                           None if self.proj_err is None
                           else self.proj_err.ctypes.data_as(C.POINTER(C.c_double)),
                           None if self.disp_views is None
                           else self.disp_views.ctypes.data_as(C.POINTER(C.c_double)),
                           int(adjoint == "backward"))
        self.s_d = self._lib.orc_num_dirs(C.byref(self._P))

    @classmethod
    def from_problem(cls, prob, **overrides):
        wl = prob.wl
        kw = dict(lambda1=wl.lambda1, lambda2=wl.lambda2, mu=wl.mu, window=wl.window,
                  patch=wl.patch, h=wl.h, cg_iters=wl.cg_iters)
        kw.update(overrides)
        return cls(wl.U, wl.V, wl.H, wl.W, wl.scale, prob.blur, prob.disparity, **kw)

    # ---- parameters -------------------------------------------------
    @property
    def params(self):
        P = self._P
        return dict(lambda1=P.lambda1, lambda2=P.lambda2, mu=P.mu, window=P.window,
                    patch=P.patch, h=P.h, cg_iters=P.cg_iters, cg_tol=P.cg_tol,
                    freeze_weights=P.freeze_weights)

    def set(self, **kw):
        for k, v in kw.items():
            setattr(self._P, k, v)

    @property
    def _p(self):
        return C.byref(self._P)

    def dirs(self):
        di = np.zeros(self.s_d, np.int32)
        dj = np.zeros(self.s_d, np.int32)
        self._lib.orc_dirs(self._p, di, dj)
        return di, dj

    # ---- operators ----------------------------------------------------
    def _hr(self):
        return np.zeros(self.hr)

    def _lr(self):
        return np.zeros((self.H, self.W))

    def warp(self, k, x):
        out = self._hr(); self._lib.orc_warp(self._p, k, _f64(x), out); return out

    def warp_T(self, k, g):
        out = self._hr(); self._lib.orc_warp_T(self._p, k, _f64(g), out); return out

    def warp_bw(self, k, g):
        out = self._hr(); self._lib.orc_warp_bw(self._p, k, _f64(g), out); return out

    def blur_op(self, x):
        out = self._hr(); self._lib.orc_blur(self._p, _f64(x), out); return out

    def blur_T(self, g):
        out = self._hr(); self._lib.orc_blur_T(self._p, _f64(g), out); return out

    def down(self, x):
        out = self._lr(); self._lib.orc_down(self._p, _f64(x), out); return out

    def up(self, g):
        out = self._hr(); self._lib.orc_up(self._p, _f64(g), out); return out

    def A(self, k, x):
        out = self._lr(); self._lib.orc_A(self._p, k, _f64(x), out); return out

    def A_T(self, k, g):
        out = self._hr(); self._lib.orc_A_T(self._p, k, _f64(g), out); return out

    def weights(self, x):
        out = np.zeros((self.s_d,) + self.hr)
        self._lib.orc_weights(self._p, _f64(x), out)
        return out

    def edge_factor(self, x):
        out = self._hr(); self._lib.orc_edge_factor(self._p, _f64(x), out); return out

    def occlusion_factor(self):
        out = self._hr(); self._lib.orc_occlusion_factor(self._p, out); return out

    def S(self, w, x):
        out = np.zeros((self.s_d,) + self.hr)
        self._lib.orc_S(self._p, _f64(w), _f64(x), out)
        return out

    def S_T(self, w, g):
        out = self._hr(); self._lib.orc_S_T(self._p, _f64(w), _f64(g), out); return out

    def prox(self, u, t):
        u = _f64(u)
        out = np.zeros_like(u)
        self._lib.orc_prox(u.size, u, float(t), out)
        return out

    def normal_apply(self, w, p):
        out = self._hr(); self._lib.orc_normal_apply(self._p, _f64(w), _f64(p), out); return out

    def cost(self, y, w, x):
        return self._lib.orc_cost(self._p, _f64(y), _f64(w), _f64(x))

    def cg(self, w, v, x, K, tau=0.0):
        x = _f64(x).copy()
        pi = C.c_double(0.0)
        steps = self._lib.orc_cg(self._p, _f64(w), _f64(v), x, int(K), float(tau), C.byref(pi))
        return x, steps, pi.value

    def admm(self, y, x0, N, wA: Optional[np.ndarray] = None, wS: Optional[np.ndarray] = None,
             diagnostics: bool = False):
        """Run N iterations of Algorithm 1 from (x0, wA, wS); duals default to 0.

        Returns (x, wA, wS[, diag]) with diag an N x 5 array:
        ||dw||^2, ||dz||^2, J(x_n), final CG pi, CG steps."""
        y = _f64(y)
        assert y.shape == (self.s_k, self.H, self.W)
        x = _f64(x0).copy()
        wA = np.zeros((self.s_k, self.H, self.W)) if wA is None else _f64(wA).copy()
        wS = np.zeros((self.s_d,) + self.hr) if wS is None else _f64(wS).copy()
        diag = np.zeros((max(N, 1), 5)) if diagnostics else None
        self._lib.orc_admm(self._p, y, x, int(N), x, wA, wS,
                           diag.ctypes.data if diagnostics else None)
        return (x, wA, wS, diag) if diagnostics else (x, wA, wS)

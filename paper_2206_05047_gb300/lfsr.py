"""Python binding of liblfsr (include/lfsr.h): argument marshalling only.

Every function has the name of the C entry point it calls.  Arrays are
either CUDA torch tensors (passed as device pointers, LFSR_MEM_DEVICE) or
numpy arrays (host memory, LFSR_MEM_HOST); float32, C-contiguous.  All work
runs in the CUDA library; if the library is missing or fails to load the
import raises -- there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

LFSR_OK = 0
LFSR_EINVAL = -1
LFSR_ENOMEM = -2
LFSR_ECUDA = -3
LFSR_ENUMERIC = -4
LFSR_ETIMEOUT = -5
LFSR_EUNSUPPORTED = -6
LFSR_MEM_HOST = 0
LFSR_MEM_DEVICE = 1
LFSR_FP32 = 0
LFSR_FP16_STORAGE = 1
LFSR_BF16_STORAGE = 2
LFSR_KEEP_VIEWS_FP32 = 256
LFSR_FP16_MAX_INV_MU = 8192.0
LFSR_SERVER_DRY_RUN = 1
LFSR_WEIGHTS_PATCH = 0
LFSR_WEIGHTS_PAPER = 1
WEIGHT_SCHEMES = {"patch": LFSR_WEIGHTS_PATCH, "paper": LFSR_WEIGHTS_PAPER}
LFSR_ADJOINT_EXACT = 0
LFSR_ADJOINT_BACKWARD_WARP = 1
ADJOINTS = {"exact": LFSR_ADJOINT_EXACT, "backward": LFSR_ADJOINT_BACKWARD_WARP}
LFSR_REQ_QUEUED, LFSR_REQ_ACTIVE, LFSR_REQ_DONE, LFSR_REQ_FETCHED, LFSR_REQ_FAILED = 0, 1, 2, 3, 4
LFSR_REQ_CANCELLED = 5
LFSR_BATCH_PHASES, LFSR_BATCH_PERSISTENT = 0, 1
BATCH_FORMS = {"phases": LFSR_BATCH_PHASES, "persistent": LFSR_BATCH_PERSISTENT}
# precision names accepted by Solver(precision=...) and the benchmark
PRECISIONS = {"fp32": LFSR_FP32, "fp16": LFSR_FP16_STORAGE, "bf16": LFSR_BF16_STORAGE,
              "fp16-views32": LFSR_FP16_STORAGE | LFSR_KEEP_VIEWS_FP32,
              "bf16-views32": LFSR_BF16_STORAGE | LFSR_KEEP_VIEWS_FP32}

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "liblfsr.so")

# Entry points declared in include/lfsr.h (checked by the test-suite).
EXPORTS = ("lfsr_create", "lfsr_solve", "lfsr_destroy", "lfsr_last_error", "lfsr_stats",
           "lfsr_load", "lfsr_iterate", "lfsr_get_x", "lfsr_set_state", "lfsr_get_state",
           "lfsr_apply_A", "lfsr_apply_AT", "lfsr_weights", "lfsr_apply_normal",
           "lfsr_set_profiling", "lfsr_set_device_wait", "lfsr_apply_normal_noalloc",
           "lfsr_batch_create",
           "lfsr_batch_destroy", "lfsr_batch_last_error", "lfsr_batch_size", "lfsr_batch_load",
           "lfsr_batch_iterate", "lfsr_batch_get_x", "lfsr_batch_stats",
           "lfsr_batch_launches_per_iteration", "lfsr_batch_set_profiling",
           "lfsr_batch_kernel_times", "lfsr_batch_autotune", "lfsr_batch_tuning",
           "lfsr_batch_set_tuning", "lfsr_batch_persistent_available", "lfsr_batch_form",
           "lfsr_batch_set_form", "lfsr_batch_set_device_wait", "lfsr_estimate_state_bytes", "lfsr_server_create",
           "lfsr_server_destroy", "lfsr_server_last_error", "lfsr_server_submit",
           "lfsr_server_step", "lfsr_server_status", "lfsr_server_fetch", "lfsr_server_stats",
           "lfsr_server_cancel")


class lfsr_params(C.Structure):
    _fields_ = [("struct_size", C.c_uint32), ("U", C.c_int32), ("V", C.c_int32),
                ("H", C.c_int32), ("W", C.c_int32), ("scale", C.c_int32), ("kb", C.c_int32),
                ("blur", C.POINTER(C.c_float)), ("disparity", C.POINTER(C.c_float)),
                ("lambda1", C.c_double), ("lambda2", C.c_double), ("mu", C.c_double),
                ("nltv_window", C.c_int32), ("nltv_patch", C.c_int32), ("nltv_h", C.c_double),
                ("cg_iters", C.c_int32), ("cg_tol", C.c_double), ("precision", C.c_int32),
                ("views", C.POINTER(C.c_int32)), ("n_views", C.c_int32),
                ("weights", C.c_int32), ("sigma_s", C.c_float), ("sigma_e", C.c_float),
                ("sigma_o1", C.c_float), ("sigma_o2", C.c_float),
                ("proj_err", C.POINTER(C.c_float)),
                ("disparity_views", C.POINTER(C.c_float)), ("adjoint", C.c_int32)]


class lfsr_stats_t(C.Structure):
    _fields_ = [("struct_size", C.c_uint32), ("iterations", C.c_int32), ("cg_steps", C.c_int32),
                ("status", C.c_int32), ("dual_change_sq", C.c_double), ("cg_pi", C.c_double),
                ("state_bytes", C.c_int64), ("launches", C.c_int64),
                ("kernel_ms", C.c_double * 8), ("kernel_launches", C.c_int64 * 8),
                ("op_split_even", C.c_double), ("op_split_balanced", C.c_double)]


class lfsr_server_config(C.Structure):
    _fields_ = [("struct_size", C.c_uint32), ("hbm_budget_bytes", C.c_int64),
                ("max_active", C.c_int32), ("iterations", C.c_int32),
                ("iterations_per_step", C.c_int32), ("flags", C.c_int32)]


class lfsr_server_stats_t(C.Structure):
    _fields_ = [("struct_size", C.c_uint32), ("queued", C.c_int32), ("active", C.c_int32),
                ("done", C.c_int32), ("failed", C.c_int32), ("bytes_in_use", C.c_int64),
                ("bytes_peak", C.c_int64), ("iterations", C.c_int64),
                ("batch_rebuilds", C.c_int64), ("admitted", C.c_int64), ("retired", C.c_int64),
                ("launches", C.c_int64), ("cancelled", C.c_int64)]


class LfsrError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"lfsr error {code}: {msg}")
        self.code = code


_lib = None


def load_library(path: str = _LIB_PATH):
    """Loads liblfsr.so (raises if it is missing: there is no CPU path)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing; build it with __graft_entry__.build()")
    lib = C.CDLL(path)
    H = C.c_void_p
    fp = C.c_void_p
    sig = {
        "lfsr_create": (C.c_int, [C.POINTER(lfsr_params), C.c_void_p, C.POINTER(C.c_void_p)]),
        "lfsr_solve": (C.c_int, [H, fp, C.c_int, fp, fp, C.c_int]),
        "lfsr_destroy": (None, [H]),
        "lfsr_last_error": (C.c_char_p, [H]),
        "lfsr_stats": (C.c_int, [H, C.POINTER(lfsr_stats_t)]),
        "lfsr_load": (C.c_int, [H, fp, fp, C.c_int]),
        "lfsr_iterate": (C.c_int, [H, C.c_int]),
        "lfsr_get_x": (C.c_int, [H, fp, C.c_int]),
        "lfsr_set_state": (C.c_int, [H, fp, fp, fp, C.c_int]),
        "lfsr_get_state": (C.c_int, [H, fp, fp, fp, C.c_int]),
        "lfsr_apply_A": (C.c_int, [H, C.c_int, fp, fp, C.c_int]),
        "lfsr_apply_AT": (C.c_int, [H, C.c_int, fp, fp, C.c_int]),
        "lfsr_weights": (C.c_int, [H, fp, fp, C.c_int]),
        "lfsr_apply_normal": (C.c_int, [H, fp, fp, fp, C.POINTER(C.c_double), C.c_int]),
        "lfsr_set_profiling": (C.c_int, [H, C.c_int]),
        "lfsr_set_device_wait": (C.c_int, [H, C.c_int64, C.c_int]),
        "lfsr_apply_normal_noalloc": (C.c_int, [C.POINTER(lfsr_params), fp, fp, fp, fp,
                                                C.POINTER(C.c_double), C.c_void_p]),
        "lfsr_batch_create": (C.c_int, [C.POINTER(lfsr_params), C.c_int, C.c_void_p,
                                        C.POINTER(C.c_void_p)]),
        "lfsr_batch_destroy": (None, [H]),
        "lfsr_batch_last_error": (C.c_char_p, [H]),
        "lfsr_batch_size": (C.c_int, [H]),
        "lfsr_batch_load": (C.c_int, [H, C.c_int, fp, fp, C.c_int]),
        "lfsr_batch_iterate": (C.c_int, [H, C.c_int]),
        "lfsr_batch_get_x": (C.c_int, [H, C.c_int, fp, C.c_int]),
        "lfsr_batch_stats": (C.c_int, [H, C.c_int, C.POINTER(lfsr_stats_t)]),
        "lfsr_batch_launches_per_iteration": (C.c_int, [H]),
        "lfsr_batch_set_profiling": (C.c_int, [H, C.c_int]),
        "lfsr_batch_autotune": (C.c_int, [H]),
        "lfsr_estimate_state_bytes": (C.c_int64, [C.POINTER(lfsr_params)]),
        "lfsr_server_create": (C.c_int, [C.POINTER(lfsr_server_config), C.c_void_p,
                                         C.POINTER(C.c_void_p)]),
        "lfsr_server_destroy": (None, [H]),
        "lfsr_server_last_error": (C.c_char_p, [H]),
        "lfsr_server_submit": (C.c_int, [H, C.POINTER(lfsr_params), fp, fp,
                                         C.POINTER(C.c_int64)]),
        "lfsr_server_step": (C.c_int, [H]),
        "lfsr_server_status": (C.c_int, [H, C.c_int64, C.POINTER(C.c_int),
                                         C.POINTER(C.c_int)]),
        "lfsr_server_fetch": (C.c_int, [H, C.c_int64, fp, C.c_int]),
        "lfsr_server_stats": (C.c_int, [H, C.POINTER(lfsr_server_stats_t)]),
        "lfsr_server_cancel": (C.c_int, [H, C.c_int64]),
        "lfsr_batch_set_tuning": (C.c_int, [H, C.POINTER(C.c_int), C.c_int, C.c_int]),
        "lfsr_batch_persistent_available": (C.c_int, [H]),
        "lfsr_batch_form": (C.c_int, [H]),
        "lfsr_batch_set_form": (C.c_int, [H, C.c_int]),
        "lfsr_batch_set_device_wait": (C.c_int, [H, C.c_int64, C.c_int]),
        "lfsr_batch_tuning": (C.c_int, [H, C.POINTER(C.c_int), C.c_int, C.POINTER(C.c_int)]),
        "lfsr_batch_kernel_times": (C.c_int, [H, C.POINTER(C.c_double),
                                              C.POINTER(C.c_int64)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _ptr(a, count: Optional[int] = None):
    """(pointer, mem_kind) of a float32 contiguous array / CUDA tensor."""
    if a is None:
        return None, None
    if isinstance(a, np.ndarray):
        if a.dtype != np.float32 or not a.flags.c_contiguous:
            raise TypeError("numpy arrays must be float32 and C-contiguous")
        if count is not None and a.size != count:
            raise ValueError(f"expected {count} elements, got {a.size}")
        return a.ctypes.data, LFSR_MEM_HOST
    import torch
    if not isinstance(a, torch.Tensor):
        raise TypeError("expected a numpy array or a torch tensor")
    if a.dtype != torch.float32 or not a.is_contiguous():
        raise TypeError("tensors must be float32 and contiguous")
    if count is not None and a.numel() != count:
        raise ValueError(f"expected {count} elements, got {a.numel()}")
    if a.is_cuda:
        return a.data_ptr(), LFSR_MEM_DEVICE
    return a.data_ptr(), LFSR_MEM_HOST


def _kind(*kinds):
    ks = {k for k in kinds if k is not None}
    if len(ks) != 1:
        raise ValueError("all arrays of one call must live in the same memory (host or device)")
    return ks.pop()


def last_error(handle) -> str:
    return load_library().lfsr_last_error(handle).decode()


def _check(rc: int, handle=None):
    if rc != LFSR_OK:
        raise LfsrError(rc, last_error(handle))


def _params(U, V, H, W, scale, blur, disparity, lambda1=2.0, lambda2=4.0, mu=300.0,
            nltv_window=5, nltv_patch=3, nltv_h=0.1, cg_iters=5, cg_tol=0.0,
            precision=LFSR_FP32, views=None, weights=LFSR_WEIGHTS_PATCH, sigma_s=0.0,
            sigma_e=0.0, sigma_o1=0.0, sigma_o2=0.0, proj_err=None, disparity_views=None,
            adjoint=LFSR_ADJOINT_EXACT):
    """(lfsr_params, arrays it points to: keep them alive while it is used).
    views: optional grid indices k = v*U + u of the views used (ascending).
    weights: "patch" / "paper" (or the LFSR_WEIGHTS_* value); the sigmas and
    the optional HR projection error proj_err belong to the paper's
    weights.  disparity_views: optional per-view maps (s_k x HR); adjoint:
    "exact" / "backward" (or the LFSR_ADJOINT_* value)."""
    blur = np.ascontiguousarray(blur, dtype=np.float32)
    disp = np.ascontiguousarray(disparity, dtype=np.float32)
    if isinstance(precision, str):
        precision = PRECISIONS[precision]
    if isinstance(weights, str):
        weights = WEIGHT_SCHEMES[weights]
    if isinstance(adjoint, str):
        adjoint = ADJOINTS[adjoint]
    s_k = U * V if views is None else len(views)
    dv = None if disparity_views is None else np.ascontiguousarray(disparity_views,
                                                                   dtype=np.float32)
    if dv is not None and dv.size != s_k * scale * H * scale * W:
        raise ValueError("disparity_views must hold s_k x (scale*H) x (scale*W) values")
    vw = None if views is None else np.ascontiguousarray(views, dtype=np.int32)
    pe = None if proj_err is None else np.ascontiguousarray(proj_err, dtype=np.float32)
    if pe is not None and pe.size != scale * H * scale * W:
        raise ValueError("proj_err must hold (scale*H) x (scale*W) values")
    prm = lfsr_params(C.sizeof(lfsr_params), U, V, H, W, scale, blur.shape[0],
                      blur.ctypes.data_as(C.POINTER(C.c_float)),
                      disp.ctypes.data_as(C.POINTER(C.c_float)),
                      lambda1, lambda2, mu, nltv_window, nltv_patch, nltv_h, cg_iters, cg_tol,
                      precision, None if vw is None else vw.ctypes.data_as(C.POINTER(C.c_int32)),
                      0 if vw is None else len(vw), weights, sigma_s, sigma_e, sigma_o1,
                      sigma_o2, None if pe is None else pe.ctypes.data_as(C.POINTER(C.c_float)),
                      None if dv is None else dv.ctypes.data_as(C.POINTER(C.c_float)), adjoint)
    return prm, (blur, disp, vw, pe, dv)


def _stream(stream):
    if stream is None:
        try:
            import torch
            return torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else 0
        except ImportError:
            return 0
    return stream if isinstance(stream, int) else stream.cuda_stream


def create(U, V, H, W, scale, blur, disparity, lambda1=2.0, lambda2=4.0, mu=300.0,
           nltv_window=5, nltv_patch=3, nltv_h=0.1, cg_iters=5, cg_tol=0.0,
           precision=LFSR_FP32, stream=None, views=None, weights=LFSR_WEIGHTS_PATCH,
           sigma_s=0.0, sigma_e=0.0, sigma_o1=0.0, sigma_o2=0.0, proj_err=None,
           disparity_views=None, adjoint=LFSR_ADJOINT_EXACT):
    """lfsr_create; returns an opaque handle.  stream: torch.cuda.Stream,
    an integer cudaStream_t, or None (the current torch stream if torch has
    CUDA, else the legacy default stream)."""
    lib = load_library()
    prm, keep = _params(U, V, H, W, scale, blur, disparity, lambda1, lambda2, mu, nltv_window,
                        nltv_patch, nltv_h, cg_iters, cg_tol, precision, views, weights,
                        sigma_s, sigma_e, sigma_o1, sigma_o2, proj_err, disparity_views, adjoint)
    h = C.c_void_p()
    _check(lib.lfsr_create(C.byref(prm), C.c_void_p(_stream(stream)), C.byref(h)))
    del keep
    return h


def destroy(handle) -> None:
    load_library().lfsr_destroy(handle)


def solve(handle, lr_views, iterations: int, x0, x_out) -> None:
    py, ky = _ptr(lr_views)
    px, kx = _ptr(x0)
    po, ko = _ptr(x_out)
    _check(load_library().lfsr_solve(handle, py, int(iterations), px, po, _kind(ky, kx, ko)), handle)


def load(handle, lr_views, x0) -> None:
    py, ky = _ptr(lr_views)
    px, kx = _ptr(x0)
    _check(load_library().lfsr_load(handle, py, px, _kind(ky, kx)), handle)


def iterate(handle, iterations: int) -> None:
    _check(load_library().lfsr_iterate(handle, int(iterations)), handle)


def get_x(handle, x_out) -> None:
    po, ko = _ptr(x_out)
    _check(load_library().lfsr_get_x(handle, po, ko), handle)


def set_state(handle, x=None, wA=None, wS=None) -> None:
    (a, ka), (b, kb), (c, kc) = _ptr(x), _ptr(wA), _ptr(wS)
    _check(load_library().lfsr_set_state(handle, a, b, c, _kind(ka, kb, kc)), handle)


def get_state(handle, x=None, wA=None, wS=None) -> None:
    (a, ka), (b, kb), (c, kc) = _ptr(x), _ptr(wA), _ptr(wS)
    _check(load_library().lfsr_get_state(handle, a, b, c, _kind(ka, kb, kc)), handle)


def apply_A(handle, view: int, x, out) -> None:
    (a, ka), (b, kb) = _ptr(x), _ptr(out)
    _check(load_library().lfsr_apply_A(handle, int(view), a, b, _kind(ka, kb)), handle)


def apply_AT(handle, view: int, g, out) -> None:
    (a, ka), (b, kb) = _ptr(g), _ptr(out)
    _check(load_library().lfsr_apply_AT(handle, int(view), a, b, _kind(ka, kb)), handle)


def weights(handle, x, w) -> None:
    (a, ka), (b, kb) = _ptr(x), _ptr(w)
    _check(load_library().lfsr_weights(handle, a, b, _kind(ka, kb)), handle)


def apply_normal(handle, xw, p, q) -> float:
    (a, ka), (b, kb), (c, kc) = _ptr(xw), _ptr(p), _ptr(q)
    out = C.c_double(0.0)
    _check(load_library().lfsr_apply_normal(handle, a, b, c, C.byref(out), _kind(ka, kb, kc)),
           handle)
    return out.value


def set_profiling(handle, on: bool) -> None:
    _check(load_library().lfsr_set_profiling(handle, int(bool(on))), handle)


LFSR_DEFAULT_WAIT_NS = 1_000_000_000


def set_device_wait(handle, limit_ns: int = LFSR_DEFAULT_WAIT_NS,
                    test_unreachable: bool = False) -> None:
    """lfsr_set_device_wait: bound of the fused CG step's grid-barrier waits
    (ns); test_unreachable makes every wait run out (LFSR_ETIMEOUT)."""
    _check(load_library().lfsr_set_device_wait(handle, int(limit_ns), int(bool(test_unreachable))),
           handle)


def stats(handle) -> dict:
    st = lfsr_stats_t()
    st.struct_size = C.sizeof(lfsr_stats_t)
    _check(load_library().lfsr_stats(handle, C.byref(st)), handle)
    return dict(iterations=st.iterations, cg_steps=st.cg_steps, status=st.status,
                dual_change_sq=st.dual_change_sq, cg_pi=st.cg_pi, state_bytes=st.state_bytes,
                launches=st.launches, kernel_ms=list(st.kernel_ms),
                kernel_launches=list(st.kernel_launches), op_split_even=st.op_split_even,
                op_split_balanced=st.op_split_balanced)


def apply_normal_noalloc(U, V, H, W, scale, blur, disparity, d_disparity, xw, p, q,
                         lambda1=1.0, lambda2=4.0, mu=1.0, nltv_window=5, nltv_patch=3,
                         nltv_h=0.1, stream=None, weights=LFSR_WEIGHTS_PATCH, views=None,
                         precision=LFSR_FP32) -> float:
    """lfsr_apply_normal_noalloc: q = M p and <p, M p> without a handle and
    without device allocation.  For callers that cannot allocate device
    memory (a host framework owns the device heap, a hard memory cap, or no
    tolerance for the synchronisation cudaMalloc implies).  disparity is
    the host map (the same map as d_disparity); d_disparity, xw, p, q are
    contiguous float32 CUDA tensors of the current device with at least
    (scale*H) * (scale*W) elements; views: optional grid indices of the
    views used."""
    import torch
    lib = load_library()
    Hh, Wh = scale * H, scale * W
    b = np.asarray(blur)
    if b.ndim != 2 or b.shape[0] != b.shape[1]:
        raise ValueError("blur must be a square kb x kb array")
    if np.asarray(disparity).shape != (Hh, Wh):
        raise ValueError(f"disparity must have shape {(Hh, Wh)}, got "
                         f"{np.asarray(disparity).shape}")
    for name, t in (("d_disparity", d_disparity), ("xw", xw), ("p", p), ("q", q)):
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise TypeError(f"{name} must be a CUDA tensor")
        if t.dtype != torch.float32 or not t.is_contiguous() or t.numel() < Hh * Wh:
            raise ValueError(f"{name} must be a contiguous float32 tensor of at least "
                             f"{Hh * Wh} elements")
    prm, keep = _params(U, V, H, W, scale, blur, disparity, lambda1, lambda2, mu, nltv_window,
                        nltv_patch, nltv_h, 0, 0.0, precision, views, weights)
    ptrs = [_ptr(t) for t in (d_disparity, xw, p, q)]
    out = C.c_double(0.0)
    _check(lib.lfsr_apply_normal_noalloc(C.byref(prm), *[a for a, _ in ptrs], C.byref(out),
                                         C.c_void_p(_stream(stream))))
    del keep
    return out.value


class Solver:
    """Owns one handle; a convenience wrapper over the functions above."""

    def __init__(self, problem=None, **kw):
        if problem is not None:
            wl = problem.wl
            base = dict(U=wl.U, V=wl.V, H=wl.H, W=wl.W, scale=wl.scale, blur=problem.blur,
                        disparity=problem.disparity, lambda1=wl.lambda1, lambda2=wl.lambda2,
                        mu=wl.mu, nltv_window=wl.window, nltv_patch=wl.patch, nltv_h=wl.h,
                        cg_iters=wl.cg_iters)
            base.update(kw)
            kw = base
        if isinstance(kw.get("precision"), str):
            kw = dict(kw, precision=PRECISIONS[kw["precision"]])
        self.kw = kw
        self.handle = create(**kw)
        self.s_k = kw["U"] * kw["V"] if kw.get("views") is None else len(kw["views"])
        self.hr = (kw["scale"] * kw["H"], kw["scale"] * kw["W"])
        self.s_d = kw.get("nltv_window", 5) ** 2 - 1

    def close(self):
        if self.handle is not None:
            destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


# ---- batches ---------------------------------------------------------------
def batch_last_error(batch) -> str:
    return load_library().lfsr_batch_last_error(batch).decode()


def _bcheck(rc: int, batch=None):
    if rc != LFSR_OK:
        raise LfsrError(rc, batch_last_error(batch))


class Batch:
    """lfsr_batch: many light fields stepped together, one launch per phase or
    one persistent launch per iteration (set_form).

    jobs: a list of dicts of create()'s keyword arguments (U, V, H, W, scale,
    blur, disparity, and the solver constants, which must be equal)."""

    def __init__(self, jobs, stream=None):
        lib = load_library()
        arr = (lfsr_params * len(jobs))()
        keep = []
        for j, kw in enumerate(jobs):
            kw = dict(kw)
            kw.pop("stream", None)
            prm, k = _params(**kw)
            arr[j] = prm
            keep.append(k)
        b = C.c_void_p()
        _bcheck(lib.lfsr_batch_create(arr, len(jobs), C.c_void_p(_stream(stream)), C.byref(b)))
        del keep
        self.handle = b
        self.n = len(jobs)

    def load(self, job, lr_views, x0):
        py, ky = _ptr(lr_views)
        px, kx = _ptr(x0)
        _bcheck(load_library().lfsr_batch_load(self.handle, int(job), py, px, _kind(ky, kx)),
                self.handle)

    def iterate(self, iterations):
        _bcheck(load_library().lfsr_batch_iterate(self.handle, int(iterations)), self.handle)

    def get_x(self, job, x_out):
        po, ko = _ptr(x_out)
        _bcheck(load_library().lfsr_batch_get_x(self.handle, int(job), po, ko), self.handle)

    def stats(self, job) -> dict:
        st = lfsr_stats_t()
        st.struct_size = C.sizeof(lfsr_stats_t)
        _bcheck(load_library().lfsr_batch_stats(self.handle, int(job), C.byref(st)), self.handle)
        return dict(iterations=st.iterations, cg_steps=st.cg_steps, status=st.status,
                    dual_change_sq=st.dual_change_sq, cg_pi=st.cg_pi,
                    state_bytes=st.state_bytes, op_split_even=st.op_split_even,
                    op_split_balanced=st.op_split_balanced)

    def launches_per_iteration(self) -> int:
        return load_library().lfsr_batch_launches_per_iteration(self.handle)

    def autotune(self) -> dict:
        """lfsr_batch_autotune (iterates the loaded state: load again
        afterwards); returns the choices."""
        _bcheck(load_library().lfsr_batch_autotune(self.handle), self.handle)
        return self.tuning()

    def tuning(self) -> dict:
        tiles = (C.c_int * 64)()
        chunk = C.c_int(0)
        g = load_library().lfsr_batch_tuning(self.handle, tiles, 64, C.byref(chunk))
        return {"operator_tile": list(tiles[:g]), "nltv_apply_chunk": chunk.value,
                "form": self.form()}

    def set_tuning(self, operator_tile, nltv_apply_chunk):
        tiles = (C.c_int * len(operator_tile))(*operator_tile)
        _bcheck(load_library().lfsr_batch_set_tuning(self.handle, tiles, len(operator_tile),
                                                     int(nltv_apply_chunk)), self.handle)

    def persistent_available(self) -> bool:
        return bool(load_library().lfsr_batch_persistent_available(self.handle))

    def form(self) -> str:
        f = load_library().lfsr_batch_form(self.handle)
        return {v: k for k, v in BATCH_FORMS.items()}[f]

    def set_form(self, form: str):
        """'phases' (one launch per phase) or 'persistent' (one launch per
        iteration)."""
        _bcheck(load_library().lfsr_batch_set_form(self.handle, BATCH_FORMS[form]), self.handle)

    def set_device_wait(self, limit_ns: int, test_unreachable: bool = False):
        _bcheck(load_library().lfsr_batch_set_device_wait(self.handle, int(limit_ns),
                                                          int(bool(test_unreachable))),
                self.handle)

    def set_profiling(self, on: bool):
        _bcheck(load_library().lfsr_batch_set_profiling(self.handle, int(bool(on))), self.handle)

    def kernel_times(self):
        """(ms[8], launches[8]) by launch class since profiling was switched on."""
        ms = (C.c_double * 8)()
        n = (C.c_int64 * 8)()
        _bcheck(load_library().lfsr_batch_kernel_times(self.handle, ms, n), self.handle)
        return list(ms), list(n)

    def close(self):
        if self.handle is not None:
            load_library().lfsr_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


# ---- size estimate and the continuous-batching server ----------------------
def estimate_state_bytes(**kw) -> int:
    """lfsr_estimate_state_bytes for create()'s keyword arguments."""
    prm, keep = _params(**kw)
    n = load_library().lfsr_estimate_state_bytes(C.byref(prm))
    del keep
    if n < 0:
        raise LfsrError(LFSR_EINVAL, last_error(None))
    return int(n)


def server_last_error(server) -> str:
    return load_library().lfsr_server_last_error(server).decode()


class Server:
    """lfsr_server: requests admitted as slots and the budget allow, all
    active light fields stepped together, each retired at its N-th
    iteration."""

    def __init__(self, hbm_budget_bytes, max_active=64, iterations=100, iterations_per_step=4,
                 dry_run=False, stream=None):
        cfg = lfsr_server_config(C.sizeof(lfsr_server_config), int(hbm_budget_bytes),
                                 int(max_active), int(iterations), int(iterations_per_step),
                                 LFSR_SERVER_DRY_RUN if dry_run else 0)
        h = C.c_void_p()
        rc = load_library().lfsr_server_create(C.byref(cfg), C.c_void_p(_stream(stream)),
                                               C.byref(h))
        if rc != LFSR_OK:
            raise LfsrError(rc, server_last_error(None))
        self.handle = h

    def _check(self, rc):
        if rc < 0:
            raise LfsrError(rc, server_last_error(self.handle))
        return rc

    def submit(self, lr_views, x0, **kw) -> int:
        """Queues one request (host numpy arrays); kw as for create()."""
        prm, keep = _params(**kw)
        y = np.ascontiguousarray(lr_views, dtype=np.float32)
        x = np.ascontiguousarray(x0, dtype=np.float32)
        rid = C.c_int64(-1)
        self._check(load_library().lfsr_server_submit(
            self.handle, C.byref(prm), y.ctypes.data_as(C.c_void_p), x.ctypes.data_as(C.c_void_p),
            C.byref(rid)))
        del keep
        return rid.value

    def step(self) -> int:
        return self._check(load_library().lfsr_server_step(self.handle))

    def status(self, rid):
        st, it = C.c_int(0), C.c_int(0)
        rc = load_library().lfsr_server_status(self.handle, int(rid), C.byref(st), C.byref(it))
        return st.value, it.value, rc

    def fetch(self, rid, x_out):
        po, ko = _ptr(x_out)
        self._check(load_library().lfsr_server_fetch(self.handle, int(rid), po, ko))

    def stats(self) -> dict:
        st = lfsr_server_stats_t()
        st.struct_size = C.sizeof(lfsr_server_stats_t)
        self._check(load_library().lfsr_server_stats(self.handle, C.byref(st)))
        return {k: getattr(st, k) for k, _ in lfsr_server_stats_t._fields_ if k != "struct_size"}

    def cancel(self, rid) -> None:
        """lfsr_server_cancel: a queued, active or done request leaves the
        server (state LFSR_REQ_CANCELLED; slot and budget freed)."""
        self._check(load_library().lfsr_server_cancel(self.handle, int(rid)))

    def close(self):
        if self.handle is not None:
            load_library().lfsr_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


"""Seeded synthetic light fields shaped like the paper's workloads.

This module only *makes inputs*.  It holds none of the solver's arithmetic:
it never applies the discrete warp / blur / decimation operators of the
degradation model (Sec. 3.1, Eq. sr_model_op).  Instead it renders a
continuous scene of fronto-parallel textured planes with occlusion, through a
Gaussian point-spread function integrated by Gauss-Hermite quadrature, at the
low-resolution sensor positions of every view.  The same arrays feed the FP64
oracle and the CUDA path.

Scene recipe (stand-in for the HCI / Inria light fields the paper uses,
Sec. 6.1, which are not available here):

* P planes, each with a value-noise texture: 3 octaves with lattice
  spacing 16, 8, 4 HR px and amplitude 1, 1/2, 1/4, smoothstep
  interpolation, normalised to [0, 1].  (A 2 px octave sits at the HR
  Nyquist limit, where no bilinear warp can model the views.)
* Plane 0 (smallest disparity) covers the frame; the others are seeded
  rectangles or discs covering 15-35 % of the frame, composited so that a
  larger disparity is in front.
* View k = (u, v) on a U x V grid has angular offset
  theta_k = (u - (U-1)/2, v - (V-1)/2); its pixel z sees the reference-view
  point z + theta_k * d (u shifts columns, v shifts rows).
* LR pixel (i', j') integrates the scene around HR position (zeta i', zeta j')
  with a Gaussian PSF of the configured sigma (3x3 Gauss-Hermite nodes).
* Noise: additive Gaussian sigma, then a fraction nu of pixels replaced by 0
  or 1 with probability 1/2 each (salt and pepper); no clipping.
* Ground truth: the reference (centre) view point-sampled on the HR grid;
  disparity map: the disparity of the front plane at each HR pixel.
* x0: Keys bicubic (a = -0.5) up-sampling of the noisy centre LR view, with LR
  pixel (i', j') placed at HR (zeta i', zeta j') and clamped edges (the
  initial guess of Algorithm 1 is a bicubic up-sampling).

Random streams: numpy PCG64 seeded with ``seed`` and split by SeedSequence;
identical on every platform.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional, Tuple

import numpy as np


# --------------------------------------------------------------------------
# Workload descriptions (sizes, noise and solver settings of the benchmarked
# light fields).  Solver weights lambda1, lambda2, mu are fixed here and used
# for every workload; the paper tunes them per case (Sec. 6.1) and gives no
# values.  lambda1 = 2, lambda2 = 4, mu = 300: from a sweep over lambda1 in
# {1, 2, 4}, lambda2 in {0.25, 1, 4}, mu in {30, 100, 300, 1000} on six
# workloads (the three named ones and three of the batched configuration) at
# their h = 0.1, the best mean PSNR gain over bicubic after 100 iterations
# (+5.2 dB or more on each), with a perturbation of x0 growing at most 1.2x
# over the 100 iterations.  A small mu (e.g. 1) lets the reweighted iteration
# diverge at h = 0.1.
# --------------------------------------------------------------------------
@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    U: int
    V: int
    H: int            # LR rows
    W: int            # LR cols
    scale: int        # zeta
    kb: int           # blur size (odd)
    blur_sigma: float
    disparities: Tuple[float, ...]
    noise_sigma: float
    impulse: float
    window: int       # NLTV search window (odd)
    patch: int        # NLTV patch (odd)
    h: float          # NLTV filtering parameter
    iterations: int   # ADMM iterations N
    cg_iters: int = 5  # K
    lambda1: float = 2.0
    lambda2: float = 4.0
    mu: float = 300.0

    @property
    def s_k(self) -> int:
        return self.U * self.V

    @property
    def HR(self) -> Tuple[int, int]:
        return (self.scale * self.H, self.scale * self.W)

    @property
    def s_d(self) -> int:
        return self.window * self.window - 1


# Scales of the paper's own weights (Sec. 3.4: spatial, edge, occlusion
# boundary, projection error; 0 turns a factor off).  The paper prints no
# values; these were chosen by an oracle sweep on the 5x5, 24^2 -> 48^2 scene
# of the quality tests (sigma_s in {2, 8, 16}, sigma_e in {0.002 .. 0.3},
# sigma_o1 in {0.25, 0.5, 1}): 40 iterations reach 25.1 dB there against
# 23.8 dB with the patch weights at h = 0.1.
PAPER_SIGMAS: Dict[str, float] = dict(sigma_s=8.0, sigma_e=0.1, sigma_o1=1.0, sigma_o2=0.0)


WORKLOADS: Dict[str, Workload] = {
    # 5x5 views, 64^2 -> 128^2 (x2), 3 planes
    "lf5x5_64_x2": Workload("lf5x5_64_x2", 5, 5, 64, 64, 2, 5, 1.0,
                            (-1.0, 0.0, 0.8), 0.02, 0.05, 5, 3, 0.1, 50),
    # 9x9 views, 256^2 -> 512^2 (x2), 5 planes (the HCI light-field shape)
    "lf9x9_256_x2": Workload("lf9x9_256_x2", 9, 9, 256, 256, 2, 7, 1.2,
                             (-2.0, -1.0, 0.0, 1.0, 2.0), 0.03, 0.10, 7, 3,
                             0.1, 100),
    # 9x9 views, 200^2 -> 600^2 (x3), 5 planes
    "lf9x9_200_x3": Workload("lf9x9_200_x3", 9, 9, 200, 200, 3, 9, 1.5,
                             (-2.0, -1.0, 0.0, 1.0, 2.0), 0.02, 0.15, 7, 3,
                             0.1, 100),
}


def batch_workloads(n: int = 64, seed: int = 4000) -> List[Workload]:
    """The uneven light fields of the batched configuration: square angular
    grid from {5, 7, 9}, square LR side uniform in [96, 384], scale from
    {2, 3} (blur 7 / sigma 1.2 for x2 and 9 / sigma 1.5 for x3), 2-6 planes at
    sorted disparities uniform in [-2, 2], impulse fraction uniform in
    [0, 0.2], Gaussian sigma uniform in [0.01, 0.03]; 7x7 NLTV window, 3x3
    patch, h = 0.1, 100 iterations.  Light field i is generated with
    make_problem(wl, seed + 1 + i)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        ang = int(rng.choice([5, 7, 9]))
        side = int(rng.integers(96, 385))
        zeta = int(rng.choice([2, 3]))
        planes = int(rng.integers(2, 7))
        disp = tuple(float(d) for d in np.sort(rng.uniform(-2.0, 2.0, planes)))
        impulse = float(rng.uniform(0.0, 0.2))
        sigma = float(rng.uniform(0.01, 0.03))
        kb, bs = (7, 1.2) if zeta == 2 else (9, 1.5)
        out.append(Workload(f"batch{seed}_{i:03d}", ang, ang, side, side, zeta, kb, bs, disp,
                            sigma, impulse, 7, 3, 0.1, 100))
    return out


def custom(name: str = "custom", **kw) -> Workload:
    """A Workload with explicit sizes (used for small and edge-case tests)."""
    base = dict(U=3, V=3, H=8, W=8, scale=2, kb=3, blur_sigma=0.8,
                disparities=(-1.0, 0.5), noise_sigma=0.02, impulse=0.05,
                window=3, patch=3, h=0.1, iterations=5)
    base.update(kw)
    return Workload(name=name, **base)


# --------------------------------------------------------------------------
# Scene
# --------------------------------------------------------------------------
_OCTAVES = ((16.0, 1.0), (8.0, 0.5), (4.0, 0.25))


class _ValueNoise:
    """Smoothstep-interpolated value noise on a lattice, summed over octaves."""

    def __init__(self, rng: np.random.Generator, lo: float, hi: float):
        # domain [lo, hi] in both axes (HR px, reference-view coordinates)
        self.lo = lo
        self.layers = []
        for spacing, amp in _OCTAVES:
            n = int(math.ceil((hi - lo) / spacing)) + 3
            self.layers.append((spacing, amp, rng.random((n, n))))
        self.norm = sum(a for _, a in _OCTAVES)

    def __call__(self, Y: np.ndarray, X: np.ndarray) -> np.ndarray:
        out = np.zeros(np.broadcast(Y, X).shape)
        for spacing, amp, lat in self.layers:
            gy = (Y - self.lo) / spacing
            gx = (X - self.lo) / spacing
            iy = np.floor(gy)
            ix = np.floor(gx)
            ty = gy - iy
            tx = gx - ix
            iy = np.clip(iy.astype(np.int64), 0, lat.shape[0] - 2)
            ix = np.clip(ix.astype(np.int64), 0, lat.shape[1] - 2)
            sy = ty * ty * (3.0 - 2.0 * ty)
            sx = tx * tx * (3.0 - 2.0 * tx)
            a = lat[iy, ix]
            b = lat[iy, ix + 1]
            c = lat[iy + 1, ix]
            d = lat[iy + 1, ix + 1]
            top = a + (b - a) * sx
            bot = c + (d - c) * sx
            out += amp * (top + (bot - top) * sy)
        return out / self.norm


@dataclasses.dataclass
class _Plane:
    disparity: float
    kind: str                 # "full", "rect", "disc"
    geom: Tuple[float, ...]   # rect: y0, x0, y1, x1; disc: cy, cx, r
    tex: _ValueNoise

    def covers(self, Y: np.ndarray, X: np.ndarray) -> np.ndarray:
        if self.kind == "full":
            return np.ones(np.broadcast(Y, X).shape, dtype=bool)
        if self.kind == "rect":
            y0, x0, y1, x1 = self.geom
            return (Y >= y0) & (Y < y1) & (X >= x0) & (X < x1)
        cy, cx, r = self.geom
        return (Y - cy) ** 2 + (X - cx) ** 2 < r * r


def _make_scene(wl: Workload, rng: np.random.Generator) -> List[_Plane]:
    HH, WW = wl.HR
    amax = max((wl.U - 1) / 2.0, (wl.V - 1) / 2.0)
    dmax = max(abs(d) for d in wl.disparities)
    margin = amax * dmax + 4.0 * wl.blur_sigma + 8.0
    lo, hi = -margin, max(HH, WW) + margin
    planes = []
    disp = sorted(wl.disparities)
    for idx, d in enumerate(disp):
        tex = _ValueNoise(rng, lo, hi)
        if idx == 0:
            planes.append(_Plane(d, "full", (), tex))
            continue
        area = rng.uniform(0.15, 0.35) * HH * WW
        if rng.random() < 0.5:
            aspect = rng.uniform(0.6, 1.6)
            h = min(math.sqrt(area * aspect), 0.9 * HH)
            w = min(area / h, 0.9 * WW)
            y0 = rng.uniform(0.05 * HH, HH - h - 0.05 * HH) if HH - h > 0.1 * HH else 0.0
            x0 = rng.uniform(0.05 * WW, WW - w - 0.05 * WW) if WW - w > 0.1 * WW else 0.0
            planes.append(_Plane(d, "rect", (y0, x0, y0 + h, x0 + w), tex))
        else:
            r = math.sqrt(area / math.pi)
            # (images thinner than the disc: centred on that axis)
            cy = rng.uniform(r * 0.5, HH - r * 0.5) if HH > r else 0.5 * HH
            cx = rng.uniform(r * 0.5, WW - r * 0.5) if WW > r else 0.5 * WW
            planes.append(_Plane(d, "disc", (cy, cx, r), tex))
    return planes


def _render(planes: List[_Plane], Y: np.ndarray, X: np.ndarray,
            tu: float, tv: float) -> Tuple[np.ndarray, np.ndarray]:
    """Scene value and front-plane disparity seen at view-(tu, tv) points."""
    val = np.empty(Y.shape)
    dsp = np.empty(Y.shape)
    todo = np.ones(Y.shape, dtype=bool)
    for pl in reversed(planes):          # front (largest disparity) first
        Yr = Y + tv * pl.disparity
        Xr = X + tu * pl.disparity
        m = todo & pl.covers(Yr, Xr)
        if m.any():
            val[m] = pl.tex(Yr[m], Xr[m])
            dsp[m] = pl.disparity
            todo &= ~m
    assert not todo.any()
    return val, dsp


# Gauss-Hermite nodes/weights for the standard normal (3 points)
_GH_NODES = (-math.sqrt(3.0), 0.0, math.sqrt(3.0))
_GH_WEIGHTS = (1.0 / 6.0, 2.0 / 3.0, 1.0 / 6.0)


def view_offsets(U: int, V: int) -> np.ndarray:
    """theta_k = (tu, tv) for k = v*U + u (centre view at (0, 0))."""
    out = np.zeros((U * V, 2))
    for v in range(V):
        for u in range(U):
            out[v * U + u] = (u - (U - 1) / 2.0, v - (V - 1) / 2.0)
    return out


def star_views(U: int, V: int) -> np.ndarray:
    """Grid indices k = v*U + u of the views on the centre row, the centre
    column and the two diagonals through the centre (square grid): 17 of
    5 x 5, the star-shaped subset of Sec. 6.1's x4 experiment."""
    assert U == V and U % 2 == 1
    c = (U - 1) // 2
    ks = set()
    for t in range(U):
        for (u, v) in ((t, c), (c, t), (t, t), (t, U - 1 - t)):
            ks.add(v * U + u)
    return np.array(sorted(ks), dtype=np.int32)


def gaussian_blur_kernel(kb: int, sigma: float) -> np.ndarray:
    """kb x kb Gaussian taps normalised to sum 1 (the blur PSF of Sec. 4.1)."""
    r = (kb - 1) // 2
    a = np.arange(-r, r + 1, dtype=np.float64)
    g = np.exp(-(a[:, None] ** 2 + a[None, :] ** 2) / (2.0 * sigma * sigma))
    return g / g.sum()


def _keys(t: np.ndarray, a: float = -0.5) -> np.ndarray:
    t = np.abs(t)
    out = np.zeros_like(t)
    m1 = t <= 1
    m2 = (t > 1) & (t < 2)
    out[m1] = (a + 2) * t[m1] ** 3 - (a + 3) * t[m1] ** 2 + 1
    out[m2] = a * t[m2] ** 3 - 5 * a * t[m2] ** 2 + 8 * a * t[m2] - 4 * a
    return out


def _bicubic_axis(n_lr: int, zeta: int) -> np.ndarray:
    """(zeta*n_lr) x n_lr interpolation matrix along one axis."""
    n_hr = zeta * n_lr
    M = np.zeros((n_hr, n_lr))
    for i in range(n_hr):
        c = i / zeta
        i0 = int(math.floor(c))
        for t in range(i0 - 1, i0 + 3):
            w = _keys(np.array([c - t]))[0]
            M[i, min(max(t, 0), n_lr - 1)] += w
    return M


def bicubic_upsample(lr: np.ndarray, zeta: int) -> np.ndarray:
    My = _bicubic_axis(lr.shape[0], zeta)
    Mx = _bicubic_axis(lr.shape[1], zeta)
    return My @ lr @ Mx.T


@dataclasses.dataclass
class Problem:
    wl: Workload
    seed: int
    blur: np.ndarray        # kb x kb float64
    disparity: np.ndarray   # HR float64
    y: np.ndarray           # s_k x H x W float64
    x0: np.ndarray          # HR float64
    gt: np.ndarray          # HR float64
    theta: np.ndarray       # s_k x 2 (tu, tv)
    planes: Optional[List[_Plane]] = None   # the scene (for per-view disparity maps)


def make_problem(wl: Workload, seed: int = 0,
                 noise: Optional[bool] = True) -> Problem:
    ss = np.random.SeedSequence(seed)
    s_scene, s_noise, s_imp = ss.spawn(3)
    rng = np.random.Generator(np.random.PCG64(s_scene))
    planes = _make_scene(wl, rng)
    HH, WW = wl.HR
    z = wl.scale
    # ground truth and disparity on the HR reference grid
    Yg, Xg = np.meshgrid(np.arange(HH, dtype=np.float64),
                         np.arange(WW, dtype=np.float64), indexing="ij")
    gt, disp = _render(planes, Yg, Xg, 0.0, 0.0)
    # views: PSF-integrated renders at LR sensor positions
    theta = view_offsets(wl.U, wl.V)
    Yl, Xl = np.meshgrid(z * np.arange(wl.H, dtype=np.float64),
                         z * np.arange(wl.W, dtype=np.float64), indexing="ij")
    y = np.zeros((wl.s_k, wl.H, wl.W))
    for k in range(wl.s_k):
        tu, tv = theta[k]
        acc = np.zeros((wl.H, wl.W))
        for ny, wy in zip(_GH_NODES, _GH_WEIGHTS):
            for nx, wx in zip(_GH_NODES, _GH_WEIGHTS):
                v, _ = _render(planes, Yl + ny * wl.blur_sigma,
                               Xl + nx * wl.blur_sigma, tu, tv)
                acc += wy * wx * v
        y[k] = acc
    if noise:
        rn = np.random.Generator(np.random.PCG64(s_noise))
        y = y + rn.normal(0.0, wl.noise_sigma, size=y.shape)
        ri = np.random.Generator(np.random.PCG64(s_imp))
        hit = ri.random(y.shape) < wl.impulse
        salt = ri.random(y.shape) < 0.5
        y = np.where(hit, np.where(salt, 1.0, 0.0), y)
    c = wl.s_k // 2 if (wl.U % 2 == 1 and wl.V % 2 == 1) else 0
    x0 = bicubic_upsample(y[c], z)
    return Problem(wl=wl, seed=seed, blur=gaussian_blur_kernel(wl.kb, wl.blur_sigma),
                   disparity=disp, y=y, x0=x0, gt=gt, theta=theta, planes=planes)


def view_disparity_maps(prob: Problem, views=None) -> np.ndarray:
    """Per-view disparity maps omega_k (Sec. 4.1): the disparity of the front
    plane seen at each HR grid point of view k, for the views listed (grid
    indices, ascending; None: all), s_k x HR float64.  At occlusion
    boundaries they differ from the reference map shifted: a view sees
    around the front planes."""
    wl = prob.wl
    HH, WW = wl.HR
    Yg, Xg = np.meshgrid(np.arange(HH, dtype=np.float64), np.arange(WW, dtype=np.float64),
                         indexing="ij")
    ks = range(wl.s_k) if views is None else [int(k) for k in views]
    out = np.empty((len(ks), HH, WW))
    for j, k in enumerate(ks):
        tu, tv = prob.theta[k]
        out[j] = _render(prob.planes, Yg, Xg, tu, tv)[1]
    return out


def psnr(x: np.ndarray, ref: np.ndarray) -> float:
    """10 log10(1 / MSE) over the full image, peak 1.0."""
    mse = float(np.mean((np.asarray(x, np.float64) - np.asarray(ref, np.float64)) ** 2))
    return float("inf") if mse == 0.0 else 10.0 * math.log10(1.0 / mse)


def rel_l2(a: np.ndarray, b: np.ndarray) -> float:
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def random_state(rng: np.random.Generator, shape, scale: float = 1.0) -> np.ndarray:
    """Seeded random array (used for operator tests and dual states)."""
    return scale * rng.standard_normal(shape)

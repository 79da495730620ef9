"""Seeded synthetic stereo pairs shaped like the paper's workloads.

This module only draws inputs. It holds none of the matching method's
arithmetic (no grey conversion, census, arms, costs or aggregation), so it can
feed both the CUDA path and the CPU oracle without coupling them.

Scene model (a stand-in for the Middlebury v3 half-size images of Sec. V,
which are not available here):

* K planes own the pixels of a seeded Voronoi partition of the left image.
* Plane k has disparity d(x, y) = a_k + b_k x + c_k y with a_k ~ U[0, Dmax-1]
  and |b_k|, |c_k| <= 0.05, clipped to [0, Dmax-1] and rounded per pixel
  (the integer ground truth).
* Texture: per-pixel uniform noise of standard deviation 20 grey levels
  (U(-20*sqrt(3), 20*sqrt(3))) attached to the surface, plus a smooth
  per-plane, per-channel colour gradient.
* The right image is the left image forward-warped along the epipolar line
  (Sec. II: a left pixel (x, y) appears at (x - d, y) in the right image),
  z-buffered so that the larger disparity (closer surface) wins; pixels that
  receive no left pixel (occlusions) get fresh noise.
* Gaussian sensor noise (sigma 2) on both images, then rounding and clipping to
  uint8 RGB.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

__all__ = ["StereoScene", "make_scene", "shift_pair", "paper_shapes", "scene_pool"]


@dataclass
class StereoScene:
    left: np.ndarray      # (H, W, 3) uint8, HWC interleaved
    right: np.ndarray     # (H, W, 3) uint8
    disp: np.ndarray      # (H, W) int32 ground-truth disparity of the left image
    visible: np.ndarray   # (H, W) bool, left pixel visible in the right image
    dmax: int             # number of disparities (d in [0, dmax-1])
    seed: int


# The paper's measured shapes (Table II) and the mixed-resolution set used by
# the batched and served forms: (width, height, Dmax).
paper_shapes = {
    "adirondack_h": (1436, 992, 145),
    "pipes_h": (1482, 994, 128),
    "vintage_h": (1444, 960, 380),
    "vga": (640, 480, 64),
    "xga": (1024, 768, 96),
    "fhd": (1920, 1080, 192),
}


def _voronoi_labels(rng: np.random.Generator, W: int, H: int, K: int) -> np.ndarray:
    sx = rng.uniform(0, W, size=K)
    sy = rng.uniform(0, H, size=K)
    xs = np.arange(W, dtype=np.float32)
    best = np.full((H, W), np.inf, dtype=np.float32)
    lab = np.zeros((H, W), dtype=np.int32)
    for k in range(K):
        dx2 = (xs - np.float32(sx[k])) ** 2
        for y0 in range(0, H, 256):
            y1 = min(H, y0 + 256)
            dy2 = (np.arange(y0, y1, dtype=np.float32)[:, None] - np.float32(sy[k])) ** 2
            dist = dy2 + dx2[None, :]
            sel = dist < best[y0:y1]
            best[y0:y1][sel] = dist[sel]
            lab[y0:y1][sel] = k
    return lab


def _scene_base(W: int, H: int, dmax: int, planes: int, seed: int):
    """Noise-free left image (float), disparity and the warped right image."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lab = _voronoi_labels(rng, W, H, planes)
    a = rng.uniform(0, dmax - 1, size=planes)
    b = rng.uniform(-0.05, 0.05, size=planes)
    c = rng.uniform(-0.05, 0.05, size=planes)
    base = rng.uniform(40, 215, size=(planes, 3))
    gx = rng.uniform(-60, 60, size=(planes, 3)) / max(W, 1)
    gy = rng.uniform(-60, 60, size=(planes, 3)) / max(H, 1)

    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    dcont = a[lab] + b[lab] * xx + c[lab] * yy
    disp = np.rint(np.clip(dcont, 0, dmax - 1)).astype(np.int32)

    amp = 20.0 * np.sqrt(3.0)
    tex = rng.uniform(-amp, amp, size=(H, W))
    left = np.empty((H, W, 3), dtype=np.float64)
    for ch in range(3):
        left[..., ch] = base[lab, ch] + gx[lab, ch] * xx + gy[lab, ch] * yy + tex

    # Forward warp with a z-buffer: target column x - d, larger d wins; among
    # equal d the key keeps the larger source column, which is deterministic.
    xt = xx.astype(np.int64) - disp
    ok = xt >= 0
    rows = yy.astype(np.int64)
    tgt = rows * W + np.where(ok, xt, 0)
    src = (rows * W + xx.astype(np.int64))
    key = disp.astype(np.int64) * (W * H + 1) + src
    zbuf = np.full(W * H, -1, dtype=np.int64)
    np.maximum.at(zbuf, tgt[ok], key[ok])
    filled = zbuf >= 0
    win = np.where(filled, zbuf % (W * H + 1), 0)

    right = np.empty((H * W, 3), dtype=np.float64)
    lflat = left.reshape(-1, 3)
    right[filled] = lflat[win[filled]]
    n_holes = int((~filled).sum())
    right[~filled] = rng.uniform(40, 215, size=(n_holes, 1)) + rng.uniform(-amp, amp, size=(n_holes, 3))
    right = right.reshape(H, W, 3)

    visible = np.zeros(W * H, dtype=bool)
    visible[win[filled]] = True
    visible = visible.reshape(H, W) & ok
    return rng, left, right, disp, visible


def _finish(rng: np.random.Generator, img: np.ndarray, sigma: float) -> np.ndarray:
    noisy = img + rng.normal(0.0, sigma, size=img.shape)
    return np.clip(np.rint(noisy), 0, 255).astype(np.uint8)


def make_scene(W: int, H: int, dmax: int, planes: int = 12, seed: int = 0,
               sensor_sigma: float = 2.0) -> StereoScene:
    """One seeded piecewise-planar stereo pair of size W x H with dmax disparities."""
    if W < 1 or H < 1 or dmax < 1:
        raise ValueError("W, H and dmax must be positive")
    rng, left, right, disp, visible = _scene_base(W, H, dmax, planes, seed)
    return StereoScene(_finish(rng, left, sensor_sigma), _finish(rng, right, sensor_sigma),
                       disp, visible, dmax, seed)


def scene_pool(W: int, H: int, dmax: int, planes: int, seed: int, count: int,
               sensor_sigma: float = 2.0):
    """`count` pairs of one scene that differ only in their sensor noise.

    Drawing the planes and the warp once keeps a large pool cheap to make; the
    pool is used to cycle inputs through more memory than the GPU's L2 holds.
    """
    rng, left, right, disp, visible = _scene_base(W, H, dmax, planes, seed)
    out = []
    for _ in range(count):
        out.append(StereoScene(_finish(rng, left, sensor_sigma), _finish(rng, right, sensor_sigma),
                               disp, visible, dmax, seed))
    return out


def shift_pair(W: int, H: int, d0: int, seed: int = 0, channels: int = 3):
    """Textured noise image and a copy shifted left by d0 columns.

    right(x, y) = left(x + d0, y) for x + d0 < W; the last d0 columns of the
    right image are fresh noise. Every left pixel with x >= d0 is visible at
    disparity d0.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    left = rng.integers(0, 256, size=(H, W, channels), dtype=np.uint8)
    right = rng.integers(0, 256, size=(H, W, channels), dtype=np.uint8)
    if d0 < W:
        right[:, : W - d0] = left[:, d0:]
    return left, right

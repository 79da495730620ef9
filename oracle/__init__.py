"""CPU oracle for the paper's local stereo method (arXiv 2212.00488).

TEST INFRASTRUCTURE ONLY: only the test suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package. The library's
product path never calls it and it never calls the library.

The arithmetic lives in ``stereo_oracle.c`` (plain C, direct loops); this
module only marshals numpy arrays and strings the stages together in the order
of Sec. III of the paper:

  grey -> (downscale, Eq. 2) -> census + arms -> cost (Eqs. 3-6)
  -> aggregation along x then y (Eqs. 7-8) -> WTA (Eq. 9), both bases
  -> cross-check (Eq. 10) -> median -> bilateral fill (Eq. 11) -> (upscale)
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field

import numpy as np

from . import build as _build

_lib = None

_u8p = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_f32p = np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_int = ctypes.c_int
_dbl = ctypes.c_double


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.oracle_grey.argtypes = [_u8p, _int, _int, _u8p]
        L.oracle_downscale.argtypes = [_u8p, _int, _int, _u8p]
        L.oracle_census.argtypes = [_u8p, _int, _int, _u8p]
        L.oracle_arms.argtypes = [_u8p, _int, _int, _int, _int, _int, _u8p, _u8p, _u8p, _u8p]
        L.oracle_cost_tables.argtypes = [_dbl, _dbl, _int, _i32p, _i32p]
        L.oracle_volume_int.argtypes = [_u8p] * 8 + [_int] * 4 + [_i32p, _i32p, ctypes.c_void_p, _i64p]
        L.oracle_volume_int.restype = _int
        L.oracle_wta_int.argtypes = [_u8p] * 8 + [_int] * 4 + [_i32p, _i32p, _u8p, ctypes.c_void_p]
        L.oracle_wta_int.restype = _int
        L.oracle_wta_f64.argtypes = [_u8p] * 8 + [_int] * 4 + [_dbl, _dbl, _u8p, _f64p, _f64p]
        L.oracle_wta_f64.restype = _int
        L.oracle_crosscheck.argtypes = [_u8p, _u8p, _int, _int, _u8p]
        L.oracle_median3.argtypes = [_u8p, _int, _int, _u8p]
        L.oracle_fill.argtypes = [_u8p, _u8p, _u8p, _int, _int, _int, _int, _f32p]
        L.oracle_upscale.argtypes = [_f32p, _u8p, _u8p, _int, _int, _int, _int, _int, _f32p]
        L.oracle_diff.argtypes = [_f64p, _f64p] + [_u8p] * 6 + [_int] * 3 + [_f64p, _dbl, _f64p,
                                                                           ctypes.c_void_p, ctypes.c_void_p,
                                                                           ctypes.c_void_p, ctypes.c_void_p]
        L.oracle_diff.restype = _int
        L.oracle_set_threads.argtypes = [_int]
        L.oracle_set_threads.restype = _int
        _lib = L
    return _lib


def set_threads(n: int = 0) -> int:
    """Threads of the oracle's row loops (0: every processor); returns the
    count in effect. Results are the same for any count."""
    return lib().oracle_set_threads(int(n))


@dataclass
class Params:
    """The method's constants (Sec. V and the Table II footnote) and readings."""
    lambda_ad: float = 0.3
    lambda_mc: float = 2.3
    tc: int = 13          # brightness threshold delta of the arms
    wx: int = 21          # horizontal arm cap per side
    wy: int = 31          # vertical arm cap per side
    t_fill: int = 3       # T of the bilateral estimation
    downscale: int = 1    # 1: K = 2, m = 1 mean-pool and Dmax halved; 0: none
    cost_scale: int = 512  # integer mode: each cost term is round(scale * value)
    fill_mode: int = 0    # 0 bilateral estimation; 1 closer GCP (Fig. 5a); 2 smaller disparity (Fig. 5b)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def grey(rgb):
    rgb = _c(rgb, np.uint8)
    H, W = rgb.shape[:2]
    out = np.empty((H, W), np.uint8)
    lib().oracle_grey(rgb, W, H, out)
    return out


def downscale(g):
    g = _c(g, np.uint8)
    H, W = g.shape
    out = np.empty((H // 2, W // 2), np.uint8)
    lib().oracle_downscale(g, W, H, out)
    return out


def census(g):
    g = _c(g, np.uint8)
    Y, X = g.shape
    out = np.empty((Y, X), np.uint8)
    lib().oracle_census(g, X, Y, out)
    return out


def arms(g, wx=21, wy=31, tc=13):
    """Returns (hm, hp, vm, vp), each uint8 [Y][X]."""
    g = _c(g, np.uint8)
    Y, X = g.shape
    hm, hp, vm, vp = (np.empty((Y, X), np.uint8) for _ in range(4))
    lib().oracle_arms(g, X, Y, wx, wy, tc, hm, hp, vm, vp)
    return hm, hp, vm, vp


def cost_tables(lambda_ad=0.3, lambda_mc=2.3, scale=512):
    ad = np.empty(256, np.int32)
    mc = np.empty(7, np.int32)
    lib().oracle_cost_tables(lambda_ad, lambda_mc, scale, ad, mc)
    return ad, mc


def _base_args(gB, cB, gM, cM, armsB):
    hm, hp, vm, vp = armsB
    return [_c(gB, np.uint8), _c(cB, np.uint8), _c(gM, np.uint8), _c(cM, np.uint8),
            _c(hm, np.uint8), _c(hp, np.uint8), _c(vm, np.uint8), _c(vp, np.uint8)]


def volume_int(gB, cB, gM, cM, armsB, D, direction, p: Params = Params(), want_cost=False):
    """Aggregated volume CA[d][y][x] (int64) of one base; optionally the cost C too.

    direction -1: left base (match at x - d); +1: right base (match at x + d)."""
    Y, X = np.shape(gB)
    ad, mc = cost_tables(p.lambda_ad, p.lambda_mc, p.cost_scale)
    CA = np.empty((D, Y, X), np.int64)
    C = np.empty((D, Y, X), np.int64) if want_cost else None
    rc = lib().oracle_volume_int(*_base_args(gB, cB, gM, cM, armsB), X, Y, D, direction, ad, mc,
                                 C.ctypes.data if C is not None else None, CA)
    if rc != 0:
        raise MemoryError("oracle_volume_int")
    return (CA, C) if want_cost else CA


def wta_int(gB, cB, gM, cM, armsB, D, direction, p: Params = Params(), want_best=False):
    Y, X = np.shape(gB)
    ad, mc = cost_tables(p.lambda_ad, p.lambda_mc, p.cost_scale)
    disp = np.empty((Y, X), np.uint8)
    best = np.empty((Y, X), np.int64) if want_best else None
    rc = lib().oracle_wta_int(*_base_args(gB, cB, gM, cM, armsB), X, Y, D, direction, ad, mc, disp,
                              best.ctypes.data if best is not None else None)
    if rc != 0:
        raise MemoryError("oracle_wta_int")
    return (disp, best) if want_best else disp


def wta_f64(gB, cB, gM, cM, armsB, D, direction, p: Params = Params()):
    """FP64 mode: returns (disp, best, second) with the two lowest CA per pixel."""
    Y, X = np.shape(gB)
    disp = np.empty((Y, X), np.uint8)
    best = np.empty((Y, X), np.float64)
    second = np.empty((Y, X), np.float64)
    rc = lib().oracle_wta_f64(*_base_args(gB, cB, gM, cM, armsB), X, Y, D, direction,
                              p.lambda_ad, p.lambda_mc, disp, best, second)
    if rc != 0:
        raise MemoryError("oracle_wta_f64")
    return disp, best, second


def crosscheck(dl, dr):
    dl = _c(dl, np.uint8)
    Y, X = dl.shape
    out = np.empty((Y, X), np.uint8)
    lib().oracle_crosscheck(dl, _c(dr, np.uint8), X, Y, out)
    return out


def median3(d):
    d = _c(d, np.uint8)
    Y, X = d.shape
    out = np.empty((Y, X), np.uint8)
    lib().oracle_median3(d, X, Y, out)
    return out


def fill(dm, gcp, g, T=3, mode=0):
    """Sec. III-E fill of non-GCPs; mode 0 bilateral estimation, 1 the closer
    GCP (Fig. 5a), 2 the smaller disparity (Fig. 5b)."""
    dm = _c(dm, np.uint8)
    Y, X = dm.shape
    out = np.empty((Y, X), np.float32)
    lib().oracle_fill(dm, _c(gcp, np.uint8), _c(g, np.uint8), X, Y, T, mode, out)
    return out


def upscale(dp, gs, gf, T=3):
    dp = _c(dp, np.float32)
    Y, X = dp.shape
    H, W = np.shape(gf)
    out = np.empty((H, W), np.float32)
    lib().oracle_upscale(dp, _c(gs, np.uint8), _c(gf, np.uint8), X, Y, W, H, T, out)
    return out


def processed_dmax(dmax: int, downscale: int) -> int:
    """Disparity count after scaling down: Dmax is halved (Sec. I), rounded up."""
    return (dmax + 1) // 2 if downscale else dmax


@dataclass
class Result:
    disp: np.ndarray          # final float map (full-res units and size when downscaled)
    dl: np.ndarray            # D^L uint8 at processed size
    dr: np.ndarray            # D^R uint8
    gcp: np.ndarray           # GCP mask uint8 (0/1)
    dm: np.ndarray            # median-filtered D^L
    dplus: np.ndarray         # filled map, float, processed size and units
    grey_l: np.ndarray        # processed grey images
    grey_r: np.ndarray
    census_l: np.ndarray
    census_r: np.ndarray
    arms_l: tuple
    arms_r: tuple
    grey_full_l: np.ndarray = field(default=None)


def pipeline(left_rgb, right_rgb, dmax: int, p: Params = Params()) -> Result:
    """The whole method (Sec. III steps 1-8) on one RGB pair, integer cost mode."""
    gl_full, gr_full = grey(left_rgb), grey(right_rgb)
    if p.downscale:
        gl, gr = downscale(gl_full), downscale(gr_full)
    else:
        gl, gr = gl_full, gr_full
    D = processed_dmax(dmax, p.downscale)
    cl, cr = census(gl), census(gr)
    al = arms(gl, p.wx, p.wy, p.tc)
    ar = arms(gr, p.wx, p.wy, p.tc)
    dl = wta_int(gl, cl, gr, cr, al, D, -1, p)
    dr = wta_int(gr, cr, gl, cl, ar, D, +1, p)
    gcp = crosscheck(dl, dr)
    dm = median3(dl)
    dplus = fill(dm, gcp, gl, p.t_fill, p.fill_mode)
    if p.downscale:
        disp = upscale(dplus, gl, gl_full, p.t_fill)
    else:
        disp = dplus.copy()
    return Result(disp, dl, dr, gcp, dm, dplus, gl, gr, cl, cr, al, ar, gl_full)


def supports(left_rgb, right_rgb, p: Params = Params()):
    """Processed grey, census codes and arms of both images (Sec. III steps
    1-3), the inputs of the matching cost."""
    gl, gr = grey(left_rgb), grey(right_rgb)
    if p.downscale:
        gl, gr = downscale(gl), downscale(gr)
    return (gl, census(gl), arms(gl, p.wx, p.wy, p.tc)), (gr, census(gr), arms(gr, p.wx, p.wy, p.tc))


def wta_pair_f64(left_rgb, right_rgb, dmax: int, p: Params = Params()):
    """FP64 mode of the matching cost, both aggregations and the WTA for both
    bases (Eqs. 3-9 without quantisation). Returns ((D^L, best, second),
    (D^R, best, second))."""
    (gl, cl, al), (gr, cr, ar) = supports(left_rgb, right_rgb, p)
    D = processed_dmax(dmax, p.downscale)
    return wta_f64(gl, cl, gr, cr, al, D, -1, p), wta_f64(gr, cr, gl, cl, ar, D, +1, p)


def support_size(arms_b):
    """Cells in each anchor's cross support: the sum over the rows of its
    vertical arm of each row's horizontal width (Eqs. 7-8)."""
    hm, hp, vm, vp = (np.asarray(a, np.int64) for a in arms_b)
    width = hm + hp + 1
    Y, X = width.shape
    cum = np.vstack([np.zeros((1, X), np.int64), np.cumsum(width, axis=0)])
    ys = np.arange(Y)[:, None]
    xs = np.arange(X)[None, :]
    return cum[ys + vp + 1, xs] - cum[ys - vm, xs]


def grey_f(rgb):
    """Grey on [0, 1] of float RGB on [0, 1]: the integer path's BT.601 weights
    (77, 150, 29) / 256 without rounding."""
    rgb = np.asarray(rgb, np.float64)
    return (77.0 * rgb[..., 0] + 150.0 * rgb[..., 1] + 29.0 * rgb[..., 2]) / 256.0


def quantise(g):
    """The uint8 grey the frozen census codes and arms are computed from."""
    return np.clip(np.rint(np.asarray(g, np.float64) * 255.0), 0, 255).astype(np.uint8)


def diff_forward_backward(gL, gR, census_l, census_r, arms_l, D, theta, tau=0.1, go=None):
    """Differentiable form (FP64, left base): soft-argmin disparity and, when go
    is given, the gradient of sum(go * dhat) for gL, gR and theta
    (w_AD, w_MC, lambda_AD, lambda_MC). Arms and census codes are frozen."""
    gL = _c(gL, np.float64)
    gR = _c(gR, np.float64)
    Y, X = gL.shape
    th = _c(theta, np.float64)
    dhat = np.empty((Y, X), np.float64)
    hm, hp, vm, vp = (_c(a, np.uint8) for a in arms_l)
    args = [gL, gR, _c(census_l, np.uint8), _c(census_r, np.uint8), hm, hp, vm, vp, X, Y, D, th, tau, dhat]
    if go is None:
        rc = lib().oracle_diff(*args, None, None, None, None)
        if rc != 0:
            raise MemoryError("oracle_diff")
        return dhat
    go = _c(go, np.float64)
    g_l = np.empty((Y, X), np.float64)
    g_r = np.empty((Y, X), np.float64)
    g_t = np.empty(4, np.float64)
    rc = lib().oracle_diff(*args, go.ctypes.data, g_l.ctypes.data, g_r.ctypes.data, g_t.ctypes.data)
    if rc != 0:
        raise MemoryError("oracle_diff")
    return dhat, g_l, g_r, g_t

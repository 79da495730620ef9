"""ctypes binding of the C ABI in include/stereo.h (argument marshalling only).

Every function here has the name and arguments of its C counterpart. Pointers
are passed as integers (``tensor.data_ptr()``, ``stream.cuda_stream``). There
is no fallback: if ``lib/libstereo.so`` is missing or does not load, the
import raises.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libstereo.so")

STEREO_OK = 0
STEREO_EINVAL = -1
STEREO_ENOMEM = -2
STEREO_ECUDA = -3
STEREO_ETIMEOUT = -4

STAGE_SCALEDOWN = 0
STAGE_SUPPORT = 1
STAGE_COSTAGG = 2
STAGE_REFINE = 3
STAGE_UPSCALE = 4
NUM_STAGES = 5
STAGE_NAMES = ["SD", "W+-/W*+-", "C+CA_x+CA", "CC+Post+SU", "SU"]


class stereo_job(ctypes.Structure):
    _fields_ = [
        ("left_rgb", ctypes.c_void_p),
        ("right_rgb", ctypes.c_void_p),
        ("W", ctypes.c_int),
        ("H", ctypes.c_int),
        ("Dmax", ctypes.c_int),
        ("disp_out", ctypes.c_void_p),
        ("dl_out", ctypes.c_void_p),
        ("dr_out", ctypes.c_void_p),
        ("gcp_out", ctypes.c_void_p),
    ]


class stereo_params(ctypes.Structure):
    _fields_ = [
        ("lambda_ad", ctypes.c_double),
        ("lambda_mc", ctypes.c_double),
        ("tc", ctypes.c_int),
        ("wx", ctypes.c_int),
        ("wy", ctypes.c_int),
        ("t_fill", ctypes.c_int),
        ("downscale", ctypes.c_int),
        ("cost_scale", ctypes.c_int),
        ("fill_mode", ctypes.c_int),
    ]


_vp = ctypes.c_void_p
_i = ctypes.c_int
_ctxp = ctypes.c_void_p

_SIGNATURES = {
    "stereo_default_params": (None, [ctypes.POINTER(stereo_params)]),
    "stereo_create": (_i, [ctypes.POINTER(_vp), _i, ctypes.POINTER(stereo_params), ctypes.c_size_t]),
    "stereo_destroy": (None, [_ctxp]),
    "stereo_last_error": (ctypes.c_char_p, [_ctxp]),
    "stereo_compute": (_i, [_ctxp, _vp, _vp, _i, _i, _i, _vp, _vp, _vp, _vp, _vp]),
    "stereo_compute_host": (_i, [_ctxp, _vp, _vp, _i, _i, _i, _vp, _vp, _vp, _vp]),
    "stereo_compute_host_async": (_i, [_ctxp, _vp, _vp, _i, _i, _i, _vp, _vp, _vp, _vp]),
    "stereo_sync": (_i, [_ctxp]),
    "stereo_debug_planes": (_i, [_ctxp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "stereo_launch_stage": (_i, [_ctxp, _i, _vp]),
    "stereo_set_profiling": (_i, [_ctxp, _i]),
    "stereo_stage_ms": (_i, [_ctxp, ctypes.POINTER(ctypes.c_float), _i]),
    "stereo_last_launch_count": (_i, [_ctxp]),
    "stereo_set_tile": (_i, [_ctxp, _i]),
    "stereo_get_tile": (_i, [_ctxp, _i, _i, _i]),
    "stereo_set_wait_limit": (_i, [_ctxp, ctypes.c_uint32]),
    "stereo_compute_batch": (_i, [_ctxp, _i, ctypes.c_void_p, _vp]),
    "stereo_batch_tile": (_i, [_ctxp, ctypes.POINTER(ctypes.c_float), _i]),
    "stereo_job_bytes": (ctypes.c_size_t, [ctypes.POINTER(stereo_params), _i, _i, _i]),
    "stereo_tune_save": (_i, [_ctxp, ctypes.c_char_p]),
    "stereo_tune_load": (_i, [_ctxp, ctypes.c_char_p]),
    "stereo_diff_forward": (_i, [_ctxp, _i, _i, _i, _i, _vp, _vp, _vp, _vp, _vp, ctypes.c_float, _vp, _vp, _vp]),
    "stereo_diff_backward": (_i, [_ctxp, _i, _i, _i, _i, _vp, _vp, _vp, _vp, _vp, ctypes.c_float, _vp, _vp, _vp,
                                  _vp, _vp, _vp, _vp]),
    "stereo_compute_noalloc": (_i, [ctypes.POINTER(stereo_params), _vp, _vp, _i, _i, _i, _vp, _vp, _vp, _vp,
                                    _vp, ctypes.c_char_p, ctypes.c_size_t]),
    "stereo_measure_peaks": (_i, [_i, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                  ctypes.POINTER(ctypes.c_double)]),
}

_lib = None


def load():
    """Loads the library (once) and declares every exported function."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing; build it with paper_2212_00488_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class StereoError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"stereo error {code}: {msg}")
        self.code = code


def check(ctx, rc):
    if rc != STEREO_OK:
        msg = load().stereo_last_error(ctx) if ctx else b""
        raise StereoError(rc, (msg or b"").decode(errors="replace"))
    return rc


def stereo_default_params():
    p = stereo_params()
    load().stereo_default_params(ctypes.byref(p))
    return p


def stereo_create(device=0, params=None, mem_cap_bytes=0):
    ctx = _vp()
    p = params if params is not None else stereo_default_params()
    rc = load().stereo_create(ctypes.byref(ctx), device, ctypes.byref(p), mem_cap_bytes)
    if rc != STEREO_OK:
        raise StereoError(rc, "stereo_create failed (bad parameters, no sm_103 device, or CUDA error)")
    return ctx.value


def stereo_destroy(ctx):
    load().stereo_destroy(ctx)


def stereo_last_error(ctx):
    return (load().stereo_last_error(ctx) or b"").decode(errors="replace")


def stereo_compute(ctx, left, right, W, H, dmax, disp, dl=0, dr=0, gcp=0, stream=0):
    return check(ctx, load().stereo_compute(ctx, left, right, W, H, dmax, disp, dl or None, dr or None,
                                            gcp or None, stream or None))


def stereo_compute_host(ctx, left, right, W, H, dmax, disp, dl=0, dr=0, gcp=0):
    return check(ctx, load().stereo_compute_host(ctx, left, right, W, H, dmax, disp, dl or None, dr or None,
                                                 gcp or None))


def stereo_compute_host_async(ctx, left, right, W, H, dmax, disp, dl=0, dr=0, gcp=0):
    return check(ctx, load().stereo_compute_host_async(ctx, left, right, W, H, dmax, disp, dl or None, dr or None,
                                                       gcp or None))


def stereo_sync(ctx):
    return check(ctx, load().stereo_sync(ctx))


def stereo_debug_planes(ctx, grey_l=0, grey_r=0, census_l=0, census_r=0, arms_l=0, arms_r=0, dm=0, dplus=0,
                        stream=0):
    args = [a or None for a in (grey_l, grey_r, census_l, census_r, arms_l, arms_r, dm, dplus, stream)]
    return check(ctx, load().stereo_debug_planes(ctx, *args))


def stereo_launch_stage(ctx, stage, stream=0):
    return check(ctx, load().stereo_launch_stage(ctx, stage, stream or None))


def stereo_set_profiling(ctx, on):
    """on: False/0 off, True/1 every compute, n > 1 every n-th compute."""
    return check(ctx, load().stereo_set_profiling(ctx, int(on)))


def stereo_stage_ms(ctx, n=NUM_STAGES):
    """(mean per-stage ms, number of frames averaged)."""
    buf = (ctypes.c_float * n)()
    rc = load().stereo_stage_ms(ctx, buf, n)
    if rc < 0:
        check(ctx, rc)
    return list(buf), rc


def stereo_last_launch_count(ctx):
    return load().stereo_last_launch_count(ctx)


NUM_TILES = 9


def stereo_set_tile(ctx, tile):
    return check(ctx, load().stereo_set_tile(ctx, tile))


def stereo_set_wait_limit(ctx, polls):
    return check(ctx, load().stereo_set_wait_limit(ctx, polls))


def stereo_get_tile(ctx, W, H, dmax):
    rc = load().stereo_get_tile(ctx, W, H, dmax)
    if rc < 0:
        check(ctx, rc)
    return rc


def stereo_compute_batch(ctx, jobs, stream=0):
    """jobs: a sequence of stereo_job structures."""
    arr = (stereo_job * len(jobs))(*jobs)
    return check(ctx, load().stereo_compute_batch(ctx, len(jobs), ctypes.cast(arr, ctypes.c_void_p), stream or None))


def stereo_job_bytes(params, W, H, dmax):
    """Batch workspace bytes of one W x H frame (0 if the library rejects it)."""
    return int(load().stereo_job_bytes(ctypes.byref(params) if params is not None else None, W, H, dmax))


def stereo_batch_tile(ctx):
    """(tile of the last batch, autotuner ms per tile id or -1)."""
    buf = (ctypes.c_float * NUM_TILES)()
    t = load().stereo_batch_tile(ctx, buf, NUM_TILES)
    return t, list(buf)


def stereo_tune_save(ctx, path):
    rc = load().stereo_tune_save(ctx, path.encode())
    if rc < 0:
        check(ctx, rc)
    return rc


def stereo_tune_load(ctx, path):
    rc = load().stereo_tune_load(ctx, path.encode())
    if rc < 0:
        check(ctx, rc)
    return rc


def stereo_diff_forward(ctx, B, W, H, D, left, right, left_u8, right_u8, theta, tau, dhat, stats, stream=0):
    return check(ctx, load().stereo_diff_forward(ctx, B, W, H, D, left, right, left_u8, right_u8, theta, tau, dhat,
                                                 stats, stream or None))


def stereo_diff_backward(ctx, B, W, H, D, left, right, left_u8, right_u8, theta, tau, dhat, stats, grad_dhat,
                         grad_left, grad_right, grad_theta, stream=0):
    return check(ctx, load().stereo_diff_backward(ctx, B, W, H, D, left, right, left_u8, right_u8, theta, tau,
                                                  dhat, stats, grad_dhat, grad_left, grad_right, grad_theta,
                                                  stream or None))


def stereo_measure_peaks(device=0):
    """Measured whole-device rates: (int32 add/xor/min ops/s, popc/s, shared-memory load bytes/s)."""
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    check(None, load().stereo_measure_peaks(device, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return a.value, b.value, c.value

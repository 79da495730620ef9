"""PyTorch-facing wrapper of the C ABI: torch supplies device memory and the
current stream; every step of the method runs in the library's kernels.
"""
from __future__ import annotations

from dataclasses import dataclass

import torch

from . import _lib


@dataclass
class StereoOutput:
    disp: torch.Tensor            # float32, final disparity map
    dl: torch.Tensor | None = None
    dr: torch.Tensor | None = None
    gcp: torch.Tensor | None = None


CUDA_STREAM_LEGACY = 1   # cudaStreamLegacy: the handle of the legacy default stream


def stream_handle(s: torch.cuda.Stream) -> int:
    """The cudaStream_t to pass to the C ABI for a torch stream.

    torch's default stream has handle 0, which the ABI reads as "the context's
    own stream"; it is passed as cudaStreamLegacy instead so the library's work
    stays ordered with torch's."""
    return s.cuda_stream if s.cuda_stream != 0 else CUDA_STREAM_LEGACY


def processed_shape(W: int, H: int, dmax: int, downscale: bool):
    if downscale:
        return W // 2, H // 2, (dmax + 1) // 2
    return W, H, dmax


class Stereo:
    """One library context on one CUDA device.

    ``Stereo(device=0)(left, right, dmax)`` takes uint8 CUDA tensors [H, W, 3]
    (contiguous, HWC) and returns the float disparity map; the optional maps of
    the processed image are returned when ``maps=True``.
    """

    def __init__(self, device: int = 0, mem_cap_bytes: int = 0, **params):
        p = _lib.stereo_default_params()
        for k, v in params.items():
            if not hasattr(p, k):
                raise TypeError(f"unknown parameter {k}")
            setattr(p, k, v)
        self.params = p
        self.device = device
        self.ctx = _lib.stereo_create(device, p, mem_cap_bytes)

    def close(self):
        if getattr(self, "ctx", None):
            _lib.stereo_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def downscale(self) -> bool:
        return bool(self.params.downscale)

    def _check_image(self, t: torch.Tensor, name: str):
        if t.dtype != torch.uint8 or t.dim() != 3 or t.shape[2] != 3 or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous uint8 tensor [H, W, 3]")
        if t.device.type != "cuda" or t.device.index != self.device:
            raise ValueError(f"{name} must live on cuda:{self.device}")

    def __call__(self, left: torch.Tensor, right: torch.Tensor, dmax: int, maps: bool = False,
                 out: StereoOutput | None = None, stream: torch.cuda.Stream | None = None) -> StereoOutput:
        self._check_image(left, "left")
        self._check_image(right, "right")
        if left.shape != right.shape:
            raise ValueError("left and right must have the same shape")
        H, W = int(left.shape[0]), int(left.shape[1])
        X, Y, _ = processed_shape(W, H, dmax, self.downscale)
        dev = left.device
        if out is None:
            out = StereoOutput(torch.empty((H, W), dtype=torch.float32, device=dev))
            if maps:
                out.dl = torch.empty((Y, X), dtype=torch.uint8, device=dev)
                out.dr = torch.empty((Y, X), dtype=torch.uint8, device=dev)
                out.gcp = torch.empty((Y, X), dtype=torch.uint8, device=dev)
        s = stream if stream is not None else torch.cuda.current_stream(dev)
        _lib.stereo_compute(self.ctx, left.data_ptr(), right.data_ptr(), W, H, dmax, out.disp.data_ptr(),
                            out.dl.data_ptr() if out.dl is not None else 0,
                            out.dr.data_ptr() if out.dr is not None else 0,
                            out.gcp.data_ptr() if out.gcp is not None else 0, stream_handle(s))
        return out

    def debug_planes(self, X: int, Y: int, device=None):
        """Intermediates of the last call: grey, census, arms (both images), Dm, D+."""
        dev = torch.device("cuda", self.device) if device is None else device
        t = {k: torch.empty((Y, X), dtype=torch.uint8, device=dev)
             for k in ("grey_l", "grey_r", "census_l", "census_r", "dm")}
        t["arms_l"] = torch.empty((Y, X), dtype=torch.int32, device=dev)
        t["arms_r"] = torch.empty((Y, X), dtype=torch.int32, device=dev)
        t["dplus"] = torch.empty((Y, X), dtype=torch.float32, device=dev)
        s = torch.cuda.current_stream(dev)
        _lib.stereo_debug_planes(self.ctx, t["grey_l"].data_ptr(), t["grey_r"].data_ptr(),
                                 t["census_l"].data_ptr(), t["census_r"].data_ptr(), t["arms_l"].data_ptr(),
                                 t["arms_r"].data_ptr(), t["dm"].data_ptr(), t["dplus"].data_ptr(),
                                 stream_handle(s))
        return t

    def compute_host(self, left, right, dmax: int, disp, dl=None, dr=None, gcp=None, wait: bool = True):
        """Host-buffer variant (numpy arrays or CPU tensors, ideally pinned).
        wait=False only queues the copies and the pipeline on the context's
        stream; the buffers must stay untouched until sync()."""
        def ptr(a):
            if a is None:
                return 0
            return a.data_ptr() if isinstance(a, torch.Tensor) else a.ctypes.data
        H, W = int(left.shape[0]), int(left.shape[1])
        fn = _lib.stereo_compute_host if wait else _lib.stereo_compute_host_async
        fn(self.ctx, ptr(left), ptr(right), W, H, dmax, ptr(disp), ptr(dl), ptr(dr), ptr(gcp))

    def sync(self):
        """Waits for the context's stream; raises on a bounded-wait timeout."""
        _lib.stereo_sync(self.ctx)

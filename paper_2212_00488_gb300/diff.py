"""Differentiable form: soft-argmin disparity with gradients through the
cross aggregation (a torch.autograd.Function over the C ABI).

Forward and backward run in the library's kernels; torch supplies the tensors
and the current stream. The census codes and arms are frozen, computed from
the uint8 images of the pair; the float images, the mixing weights
(w_AD, w_MC) and the robust-function scales (lambda_AD, lambda_MC) are
differentiated.
"""
from __future__ import annotations

import torch

from . import _lib
from .stereo import Stereo, stream_handle


class StereoSoftArgmin(torch.autograd.Function):
    @staticmethod
    def forward(fctx, left, right, theta, left_u8, right_u8, D: int, tau: float, st: Stereo):
        for t, name in ((left, "left"), (right, "right")):
            if t.dtype != torch.float32 or t.dim() != 4 or t.shape[3] != 3 or not t.is_contiguous() or not t.is_cuda:
                raise ValueError(f"{name} must be a contiguous float32 CUDA tensor [B, H, W, 3]")
        for t in (left_u8, right_u8):
            if t.dtype != torch.uint8 or t.shape != left.shape or not t.is_contiguous():
                raise ValueError("the uint8 images must match the float images' shape")
        theta = theta.contiguous()
        B, H, W = int(left.shape[0]), int(left.shape[1]), int(left.shape[2])
        dhat = torch.empty((B, H, W), dtype=torch.float32, device=left.device)
        stats = torch.empty((B, H, W, 2), dtype=torch.float32, device=left.device)
        s = stream_handle(torch.cuda.current_stream(left.device))
        _lib.stereo_diff_forward(st.ctx, B, W, H, D, left.data_ptr(), right.data_ptr(), left_u8.data_ptr(),
                                 right_u8.data_ptr(), theta.data_ptr(), tau, dhat.data_ptr(), stats.data_ptr(), s)
        fctx.save_for_backward(left, right, theta, left_u8, right_u8, dhat, stats)
        fctx.D, fctx.tau, fctx.st = D, tau, st
        return dhat

    @staticmethod
    def backward(fctx, grad_dhat):
        left, right, theta, left_u8, right_u8, dhat, stats = fctx.saved_tensors
        B, H, W = int(left.shape[0]), int(left.shape[1]), int(left.shape[2])
        go = grad_dhat.contiguous()
        gl = torch.empty_like(left)
        gr = torch.empty_like(right)
        gt = torch.empty(4, dtype=torch.float32, device=left.device)
        s = stream_handle(torch.cuda.current_stream(left.device))
        _lib.stereo_diff_backward(fctx.st.ctx, B, W, H, fctx.D, left.data_ptr(), right.data_ptr(),
                                  left_u8.data_ptr(), right_u8.data_ptr(), theta.data_ptr(), fctx.tau,
                                  dhat.data_ptr(), stats.data_ptr(), go.data_ptr(), gl.data_ptr(), gr.data_ptr(),
                                  gt.data_ptr(), s)
        return gl, gr, gt, None, None, None, None, None


def soft_argmin_disparity(left, right, theta, left_u8, right_u8, D: int, tau: float = 0.1, st: Stereo | None = None):
    """dhat [B, H, W] of float RGB pairs [B, H, W, 3] on [0, 1]; theta = (w_AD, w_MC, lambda_AD, lambda_MC)."""
    if st is None:
        st = Stereo(left.device.index, downscale=0)
    return StereoSoftArgmin.apply(left, right, theta, left_u8, right_u8, D, tau, st)

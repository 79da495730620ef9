"""The allocation-free entry point against the regular one.

stereo_compute_noalloc serves callers that must not allocate device memory
while they run (a real-time frame loop that may not stall on or fail in an
allocation, or a program whose memory pool owns the device). It keeps every
intermediate in one fixed array inside the library. Its maps must equal
stereo_compute's exactly, on consecutive calls that reuse that array.
This file is collected last so that a failure here never hides another test.
"""
import ctypes

import numpy as np
import pytest

from paper_2212_00488_gb300 import scenes

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2212_00488_gb300 import build
    build.build()


def _noalloc(left, right, W, H, dmax, disp, dl, dr, gcp, stream, params=None):
    from paper_2212_00488_gb300 import _lib
    err = ctypes.create_string_buffer(256)
    p = params if params is not None else _lib.stereo_default_params()
    rc = _lib.load().stereo_compute_noalloc(ctypes.byref(p), left, right, W, H, dmax, disp, dl, dr, gcp, stream,
                                            err, len(err))
    return rc, err.value.decode()


def test_noalloc_matches_regular_entry_point_on_consecutive_calls():
    from paper_2212_00488_gb300 import Stereo
    from paper_2212_00488_gb300.stereo import stream_handle
    st = Stereo(0)
    s = torch.cuda.current_stream()
    for seed, (W, H, dmax) in enumerate([(1436, 992, 145), (640, 480, 64)]):
        sc = scenes.make_scene(W, H, dmax, planes=12, seed=40 + seed)
        lt = torch.from_numpy(sc.left).cuda()
        rt = torch.from_numpy(sc.right).cuda()
        ref = st(lt, rt, dmax, maps=True)
        X, Y = W // 2, H // 2
        disp = torch.full((H, W), -1.0, dtype=torch.float32, device="cuda")
        dl = torch.zeros((Y, X), dtype=torch.uint8, device="cuda")
        dr = torch.zeros((Y, X), dtype=torch.uint8, device="cuda")
        gcp = torch.zeros((Y, X), dtype=torch.uint8, device="cuda")
        rc, msg = _noalloc(lt.data_ptr(), rt.data_ptr(), W, H, dmax, disp.data_ptr(), dl.data_ptr(),
                           dr.data_ptr(), gcp.data_ptr(), stream_handle(s))
        assert rc == 0, msg
        torch.cuda.synchronize()
        assert torch.equal(disp, ref.disp)
        assert torch.equal(dl, ref.dl) and torch.equal(dr, ref.dr) and torch.equal(gcp, ref.gcp)
    st.close()


def test_noalloc_without_downscaling_and_other_parameters():
    # the path without downscaling: the processed grey is the full-resolution
    # grey and refine writes the filled map straight into disp_out; non-default
    # arm caps and threshold, two calls in a row on different frames
    from paper_2212_00488_gb300 import Stereo, _lib
    from paper_2212_00488_gb300.stereo import stream_handle
    kw = dict(downscale=0, wx=9, wy=15, tc=20)
    st = Stereo(0, **kw)
    p = _lib.stereo_default_params()
    for k, v in kw.items():
        setattr(p, k, v)
    s = torch.cuda.current_stream()
    W, H, dmax = 640, 480, 64
    for seed in (70, 71):
        sc = scenes.make_scene(W, H, dmax, planes=12, seed=seed)
        lt = torch.from_numpy(sc.left).cuda()
        rt = torch.from_numpy(sc.right).cuda()
        ref = st(lt, rt, dmax, maps=True)
        disp = torch.full((H, W), -1.0, dtype=torch.float32, device="cuda")
        dl = torch.zeros((H, W), dtype=torch.uint8, device="cuda")
        dr = torch.zeros((H, W), dtype=torch.uint8, device="cuda")
        gcp = torch.zeros((H, W), dtype=torch.uint8, device="cuda")
        rc, msg = _noalloc(lt.data_ptr(), rt.data_ptr(), W, H, dmax, disp.data_ptr(), dl.data_ptr(),
                           dr.data_ptr(), gcp.data_ptr(), stream_handle(s), params=p)
        assert rc == 0, msg
        torch.cuda.synchronize()
        assert torch.equal(disp, ref.disp)
        assert torch.equal(dl, ref.dl) and torch.equal(dr, ref.dr) and torch.equal(gcp, ref.gcp)
    st.close()


def test_noalloc_rejects_frames_beyond_its_fixed_scratch():
    x = torch.zeros((4000, 4000, 3), dtype=torch.uint8, device="cuda")
    d = torch.zeros((4000, 4000), dtype=torch.float32, device="cuda")
    rc, msg = _noalloc(x.data_ptr(), x.data_ptr(), 4000, 4000, 128, d.data_ptr(), 0, 0, 0, 0)
    assert rc == -2 and "scratch" in msg

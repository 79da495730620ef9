"""Host logic of the serving form: memory-budget admission (no GPU)."""
import pytest

from paper_2212_00488_gb300.serve import Admission, frame_bytes


def test_admission_is_fifo_and_never_exceeds_the_cap():
    a = Admission(100)
    for i, n in enumerate([40, 30, 50, 10, 20]):
        a.offer(i, n)
    first = [i for i, _ in a.admit()]
    assert first == [0, 1]                     # 40 + 30; the 50 must wait (FIFO, no skipping)
    assert a.used == 70 and a.peak == 70
    a.release(40)
    assert [i for i, _ in a.admit()] == [2, 3]  # 30 + 50 + 10 = 90
    a.release(30)
    a.release(50)
    assert [i for i, _ in a.admit()] == [4]
    assert a.peak <= a.cap and not a.waiting


def test_admission_rejects_requests_larger_than_the_cap():
    a = Admission(10)
    with pytest.raises(ValueError):
        a.offer("big", 11)
    with pytest.raises(ValueError):
        Admission(0)


@pytest.fixture(scope="module")
def _library():
    from paper_2212_00488_gb300 import build
    build.build()


def test_frame_bytes_is_the_librarys_figure_plus_the_output(_library):
    # the library reports a frame's batch workspace (host arithmetic, no GPU);
    # a request holds that plus its float output map
    from paper_2212_00488_gb300 import _lib
    p = _lib.stereo_default_params()
    for W, H, dmax in ((640, 480, 64), (1436, 992, 145), (1920, 1080, 192), (7, 5, 3)):
        assert frame_bytes(W, H, dmax, p) == _lib.stereo_job_bytes(p, W, H, dmax) + 4 * W * H
        assert frame_bytes(W, H, dmax) == frame_bytes(W, H, dmax, p)
    small, big = frame_bytes(640, 480, 64), frame_bytes(1920, 1080, 192)
    assert 0 < small < big
    # 1436 x 992 downscaled: about 12 bytes per pixel of workspace plus the output
    assert 14 * 1436 * 992 < frame_bytes(1436, 992, 145) < 18 * 1436 * 992
    # without downscaling every plane is at full resolution
    p.downscale = 0
    assert _lib.stereo_job_bytes(p, 640, 480, 64) > 35 * 640 * 480


def test_library_rejects_what_the_entry_points_reject(_library):
    from paper_2212_00488_gb300 import _lib
    p = _lib.stereo_default_params()
    assert _lib.stereo_job_bytes(p, 0, 480, 64) == 0
    assert _lib.stereo_job_bytes(p, 640, 480, 0) == 0
    assert _lib.stereo_job_bytes(p, 640, 480, 600) == 0      # 300 disparities after halving
    assert _lib.stereo_job_bytes(p, 1, 480, 64) == 0         # downscaling needs W >= 2
    p.wx = 300
    assert _lib.stereo_job_bytes(p, 640, 480, 64) == 0
    with pytest.raises(ValueError):
        frame_bytes(640, 480, 0)

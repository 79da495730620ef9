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


def test_frame_bytes_grows_with_the_frame():
    small, big = frame_bytes(640, 480), frame_bytes(1920, 1080)
    assert 0 < small < big
    # 1436 x 992: about 12 bytes per pixel of workspace plus the 4-byte output
    assert 14 * 1436 * 992 < frame_bytes(1436, 992) < 18 * 1436 * 992

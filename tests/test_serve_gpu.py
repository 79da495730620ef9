"""Serving form on the GPU: continuous batching with memory admission.

Requests of mixed resolution arrive while others run; every result must equal
the single-frame entry point's map for that pair exactly, and the admitted
bytes must never exceed the cap.
"""
import time

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


def _pairs():
    out = []
    for i, (W, H, dmax) in enumerate([(640, 480, 64), (1436, 992, 145), (320, 240, 32), (1920, 1080, 192)]):
        s = scenes.make_scene(W, H, dmax, planes=10, seed=60 + i)
        out.append((torch.from_numpy(s.left).cuda(), torch.from_numpy(s.right).cuda(), dmax))
    return out


def test_served_results_equal_solo_results_alone_and_in_the_mix():
    from paper_2212_00488_gb300 import Stereo
    from paper_2212_00488_gb300.serve import StereoServer
    pairs = _pairs()
    solo = Stereo(0)
    ref = [solo(l, r, d).disp.clone() for l, r, d in pairs]
    torch.cuda.synchronize()
    srv = StereoServer(0, mem_cap_bytes=2 << 30, lanes=2, max_batch=8)
    # alone: one request at a time
    for (l, r, d), want in zip(pairs, ref):
        got = srv.submit(l, r, d).result(timeout=60)
        torch.cuda.synchronize()
        assert torch.equal(got, want)
    # in the mix: 24 requests arriving in bursts while earlier ones run
    futs = []
    for k in range(24):
        l, r, d = pairs[k % len(pairs)]
        futs.append((k % len(pairs), srv.submit(l, r, d)))
        if k % 5 == 4:
            time.sleep(0.002)
    for i, f in futs:
        got = f.result(timeout=60)
        torch.cuda.synchronize()
        assert torch.equal(got, ref[i])
    st = srv.stats()
    srv.close()
    solo.close()
    assert st["completed"] == 28 and st["peak_admitted_bytes"] <= st["cap_bytes"]
    assert st["batches"] < 28          # requests were grouped
    assert st["p50_ms"] is not None and st["p99_ms"] >= st["p50_ms"]


def test_small_cap_admits_one_frame_at_a_time():
    from paper_2212_00488_gb300.serve import StereoServer, frame_bytes
    pairs = _pairs()
    l, r, d = pairs[1]
    cap = frame_bytes(1436, 992) + 1000
    srv = StereoServer(0, mem_cap_bytes=cap, lanes=2)
    futs = [srv.submit(l, r, d) for _ in range(6)]
    outs = [f.result(timeout=60) for f in futs]
    torch.cuda.synchronize()
    assert all(torch.equal(o, outs[0]) for o in outs)
    with pytest.raises(ValueError):
        srv.submit(*pairs[3])          # 1920x1080 does not fit the cap at all
    st = srv.stats()
    srv.close()
    assert st["peak_admitted_bytes"] <= cap and st["completed"] == 6

"""Serving form on the GPU: continuous batching with memory admission.

Requests of mixed resolution arrive while others run; every result must equal
the oracle's map for that pair (the method of Sec. III) exactly, alone and in
the mix, and the admitted bytes must never exceed the cap.
"""
import time

import pytest

import oracle
from paper_2212_00488_gb300 import scenes

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2212_00488_gb300 import build
    build.build()


SHAPES = [(640, 480, 64), (1436, 992, 145), (320, 240, 32), (1920, 1080, 192)]


def _scenes():
    return [scenes.make_scene(W, H, dmax, planes=10, seed=60 + i) for i, (W, H, dmax) in enumerate(SHAPES)]


def _pairs(scs=None):
    scs = scs or _scenes()
    return [(torch.from_numpy(s.left).cuda(), torch.from_numpy(s.right).cuda(), dmax)
            for s, (_, _, dmax) in zip(scs, SHAPES)]


def test_served_results_equal_oracle_results_alone_and_in_the_mix():
    from paper_2212_00488_gb300.serve import StereoServer
    scs = _scenes()
    pairs = _pairs(scs)
    ref = [torch.from_numpy(oracle.pipeline(s.left, s.right, dmax, oracle.Params()).disp).cuda()
           for s, (_, _, dmax) in zip(scs, SHAPES)]
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
    assert st["completed"] == 28 and st["peak_admitted_bytes"] <= st["cap_bytes"]
    assert st["batches"] < 28          # requests were grouped
    assert st["p50_ms"] is not None and st["p99_ms"] >= st["p50_ms"]


def test_small_cap_runs_one_frame_per_lane_at_a_time():
    # each of the two lanes owns half the cap, room for one 1436x992 frame;
    # its context is created with that share, so the library enforces it too
    from paper_2212_00488_gb300.serve import StereoServer, frame_bytes
    pairs = _pairs()
    l, r, d = pairs[1]
    cap = 2 * frame_bytes(1436, 992, 145) + 1000
    srv = StereoServer(0, mem_cap_bytes=cap, lanes=2)
    futs = [srv.submit(l, r, d) for _ in range(6)]
    outs = [f.result(timeout=60) for f in futs]
    torch.cuda.synchronize()
    assert all(torch.equal(o, outs[0]) for o in outs)
    with pytest.raises(ValueError):
        srv.submit(*pairs[3])          # 1920x1080 does not fit a lane's share
    st = srv.stats()
    srv.close()
    assert st["peak_admitted_bytes"] <= cap and st["completed"] == 6
    assert st["batches"] == 6          # one frame per batch: two do not fit a share


def test_a_bounded_wait_that_gives_up_fails_the_batch_futures():
    # with a wait limit of zero polls every wait in the fused kernel gives up
    # at once; the server reads the context's error word when the batch
    # completes and fails those requests instead of returning their maps
    from paper_2212_00488_gb300 import _lib
    from paper_2212_00488_gb300.serve import StereoServer
    l, r, d = _pairs()[2]
    srv = StereoServer(0, mem_cap_bytes=1 << 30, lanes=1, tile=0)
    _lib.stereo_set_wait_limit(srv.lanes[0].st.ctx, 0)
    f = srv.submit(l, r, d)
    with pytest.raises(_lib.StereoError) as e:
        f.result(timeout=60)
    assert e.value.code == _lib.STEREO_ETIMEOUT
    _lib.stereo_set_wait_limit(srv.lanes[0].st.ctx, 1 << 20)
    got = srv.submit(l, r, d).result(timeout=60)
    torch.cuda.synchronize()
    st = srv.stats()
    srv.close()
    sc = _scenes()[2]
    want = oracle.pipeline(sc.left, sc.right, d, oracle.Params()).disp
    assert (got.cpu().numpy() == want).all()
    assert st["failed"] == 1 and st["completed"] == 1

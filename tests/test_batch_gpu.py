"""Batched form: many pairs of uneven size in one call.

Every frame of a batch is the method of Sec. III (Eqs. 3-11) on that pair, so
each output is compared bit-exactly with the CPU oracle at every frame shape of
the batched workload (640x480/64, 1024x768/96, 1436x992/145, 1920x1080/192).
Frames of larger mixes are also compared with the single-frame entry point,
whatever tile shape the autotuner picks and across calls that reuse the
captured graph with other buffers.
"""
import os
import tempfile

import numpy as np
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


def _frames(shapes, seed):
    out = []
    for i, (W, H, dmax) in enumerate(shapes):
        s = scenes.make_scene(W, H, dmax, planes=8, seed=seed + i)
        out.append((torch.from_numpy(s.left).cuda(), torch.from_numpy(s.right).cuda(), W, H, dmax))
    return out


def _batch(st, frames, tile=None):
    from paper_2212_00488_gb300 import _lib
    from paper_2212_00488_gb300.stereo import stream_handle
    jobs, outs = [], []
    for lt, rt, W, H, dmax in frames:
        X, Y = W // 2, H // 2
        o = dict(disp=torch.full((H, W), -7.0, device="cuda"),
                 dl=torch.zeros((Y, X), dtype=torch.uint8, device="cuda"),
                 dr=torch.zeros((Y, X), dtype=torch.uint8, device="cuda"),
                 gcp=torch.zeros((Y, X), dtype=torch.uint8, device="cuda"))
        outs.append(o)
        jobs.append(_lib.stereo_job(lt.data_ptr(), rt.data_ptr(), W, H, dmax, o["disp"].data_ptr(),
                                    o["dl"].data_ptr(), o["dr"].data_ptr(), o["gcp"].data_ptr()))
    if tile is not None:
        _lib.stereo_set_tile(st.ctx, tile)
    _lib.stereo_compute_batch(st.ctx, jobs, stream_handle(torch.cuda.current_stream()))
    torch.cuda.synchronize()
    _lib.stereo_sync(st.ctx)
    return outs


def _check_against_solo(frames, outs):
    from paper_2212_00488_gb300 import Stereo
    solo = Stereo(0)
    for (lt, rt, W, H, dmax), o in zip(frames, outs):
        ref = solo(lt, rt, dmax, maps=True)
        torch.cuda.synchronize()
        assert torch.equal(o["disp"], ref.disp), (W, H, dmax)
        assert torch.equal(o["dl"], ref.dl) and torch.equal(o["dr"], ref.dr) and torch.equal(o["gcp"], ref.gcp)
    solo.close()


MENU = [(640, 480, 64), (1024, 768, 96), (1436, 992, 145), (1920, 1080, 192)]


def test_one_frame_of_each_menu_shape_matches_the_oracle():
    # one batch holding a frame of every shape of the batched workload; each
    # frame's float map, D^L, D^R and GCP mask against the oracle, element by
    # element (the largest frame first inside the persistent kernel, the
    # smallest last, so tiles of different frames share the launch)
    from paper_2212_00488_gb300 import Stereo
    frames, scs = [], []
    for i, (W, H, dmax) in enumerate(MENU):
        sc = scenes.make_scene(W, H, dmax, planes=40, seed=500 + i)
        scs.append(sc)
        frames.append((torch.from_numpy(sc.left).cuda(), torch.from_numpy(sc.right).cuda(), W, H, dmax))
    st = Stereo(0)
    outs = _batch(st, frames)
    st.close()
    for sc, (_, _, W, H, dmax), o in zip(scs, frames, outs):
        ref = oracle.pipeline(sc.left, sc.right, dmax, oracle.Params())
        what = f"{W}x{H}/{dmax}"
        for k, want in (("dl", ref.dl), ("dr", ref.dr), ("gcp", ref.gcp), ("disp", ref.disp)):
            got = o[k].cpu().numpy()
            bad = np.argwhere(got != want)
            assert bad.size == 0, f"{what} {k}: {len(bad)} mismatches, first {bad[:5].tolist()}"


def test_mixed_small_batch_equals_solo_and_autotunes():
    from paper_2212_00488_gb300 import Stereo, _lib
    frames = _frames([(320, 240, 32), (200, 150, 40), (401, 301, 64), (160, 120, 16), (90, 70, 9)], 3)
    st = Stereo(0)
    outs = _batch(st, frames)
    _check_against_solo(frames, outs)
    tile, tune_ms = _lib.stereo_batch_tile(st.ctx)
    assert 0 <= tile < _lib.NUM_TILES and tune_ms[tile] > 0 and min(t for t in tune_ms if t > 0) == tune_ms[tile]
    # the choice persists through a file and is reused without tuning
    path = os.path.join(tempfile.mkdtemp(), "tune.txt")
    assert _lib.stereo_tune_save(st.ctx, path) == 1
    st2 = Stereo(0)
    assert _lib.stereo_tune_load(st2.ctx, path) == 1
    outs2 = _batch(st2, frames)
    t2, ms2 = _lib.stereo_batch_tile(st2.ctx)
    assert t2 == tile and all(m == 0 for m in ms2)          # no tuning ran in that context
    for a, b in zip(outs, outs2):
        assert torch.equal(a["disp"], b["disp"])
    st.close()
    st2.close()


def test_paper_size_mix_equals_solo_with_every_fixed_tile_and_graph_update():
    from paper_2212_00488_gb300 import Stereo
    rng = np.random.default_rng(7)
    menu = [(640, 480, 64), (1024, 768, 96), (1436, 992, 145), (1920, 1080, 192)]
    shapes = [menu[i] for i in rng.integers(0, 4, size=16)]
    frames = _frames(shapes, 100)
    st = Stereo(0)
    outs = _batch(st, frames)
    _check_against_solo(frames, outs)
    # a second call with fresh output buffers updates the captured graph
    outs_b = _batch(st, frames)
    for a, b in zip(outs, outs_b):
        assert torch.equal(a["disp"], b["disp"])
    for tile in (0, 2, 4):
        outs_t = _batch(st, frames[:4], tile=tile)
        for a, b in zip(outs[:4], outs_t):
            assert torch.equal(a["disp"], b["disp"]) and torch.equal(a["dl"], b["dl"])
    st.close()


def test_job_bytes_bound_the_batch_workspace():
    # a context whose cap is the sum of its frames' stereo_job_bytes runs the
    # batch; a cap below the frames' layouts is refused with ENOMEM
    from paper_2212_00488_gb300 import Stereo, _lib
    frames = _frames([(640, 480, 64), (1024, 768, 96)], 9)
    p = _lib.stereo_default_params()
    need = sum(_lib.stereo_job_bytes(p, W, H, dmax) for _, _, W, H, dmax in frames)
    st = Stereo(0, mem_cap_bytes=need)
    outs = _batch(st, frames, tile=0)
    st.close()
    _check_against_solo(frames, outs)
    small = Stereo(0, mem_cap_bytes=need // 2)
    with pytest.raises(_lib.StereoError) as e:
        _batch(small, frames, tile=0)
    assert e.value.code == _lib.STEREO_ENOMEM
    small.close()


def test_batch_argument_errors():
    from paper_2212_00488_gb300 import Stereo, _lib
    st = Stereo(0)
    with pytest.raises(_lib.StereoError):
        _lib.stereo_compute_batch(st.ctx, [])
    x = torch.zeros((8, 8, 3), dtype=torch.uint8, device="cuda")
    d = torch.zeros((8, 8), device="cuda")
    job = _lib.stereo_job(x.data_ptr(), x.data_ptr(), 8, 8, 4, d.data_ptr(), None, None, None)
    with pytest.raises(_lib.StereoError):
        _lib.stereo_compute_batch(st.ctx, [job] * 33)
    bad = _lib.stereo_job(x.data_ptr(), x.data_ptr(), 8, 8, 0, d.data_ptr(), None, None, None)
    with pytest.raises(_lib.StereoError):
        _lib.stereo_compute_batch(st.ctx, [job, bad])
    st.close()

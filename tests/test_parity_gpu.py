"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Every cost in the library is integer (quantised tables, exact uint32 sums), so
every output is compared bit-exactly: grey, census codes, arms, D^L, D^R, the
GCP mask, the median map, the filled float map and the upscaled float map
(the float steps are single IEEE operations in the same order on both sides).
"""
import numpy as np
import pytest

import oracle
from paper_2212_00488_gb300 import scenes
from paper_2212_00488_gb300._lib import NUM_TILES

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2212_00488_gb300 import build
    build.build()


def _params(**kw):
    p = oracle.Params()
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def _run_gpu(left, right, dmax, p, tile=-1):
    from paper_2212_00488_gb300 import Stereo, _lib
    st = Stereo(0, lambda_ad=p.lambda_ad, lambda_mc=p.lambda_mc, tc=p.tc, wx=p.wx, wy=p.wy,
                t_fill=p.t_fill, downscale=p.downscale, cost_scale=p.cost_scale, fill_mode=p.fill_mode)
    _lib.stereo_set_tile(st.ctx, tile)
    lt = torch.from_numpy(np.ascontiguousarray(left)).cuda()
    rt = torch.from_numpy(np.ascontiguousarray(right)).cuda()
    out = st(lt, rt, dmax, maps=True)
    Y, X = out.dl.shape
    planes = st.debug_planes(X, Y)
    torch.cuda.synchronize()
    res = {k: v.cpu().numpy() for k, v in planes.items()}
    res.update(disp=out.disp.cpu().numpy(), dl=out.dl.cpu().numpy(), dr=out.dr.cpu().numpy(),
               gcp=out.gcp.cpu().numpy())
    st.close()
    return res


def _pack_arms(a):
    hm, hp, vm, vp = (x.astype(np.uint32) for x in a)
    return (hm | (hp << 8) | (vm << 16) | (vp << 24)).view(np.int32)


def _compare(g, r, what=""):
    assert np.array_equal(g["grey_l"], r.grey_l), what + " grey_l"
    assert np.array_equal(g["grey_r"], r.grey_r), what + " grey_r"
    assert np.array_equal(g["census_l"], r.census_l), what + " census_l"
    assert np.array_equal(g["census_r"], r.census_r), what + " census_r"
    assert np.array_equal(g["arms_l"], _pack_arms(r.arms_l)), what + " arms_l"
    assert np.array_equal(g["arms_r"], _pack_arms(r.arms_r)), what + " arms_r"
    for k in ("dl", "dr", "gcp", "dm"):
        bad = np.argwhere(g[k] != getattr(r, k))
        assert bad.size == 0, f"{what} {k}: {len(bad)} mismatches, first {bad[:5].tolist()}"
    assert np.array_equal(g["dplus"], r.dplus), what + " dplus"
    assert g["disp"].shape == r.disp.shape
    bad = np.argwhere(g["disp"] != r.disp)
    assert bad.size == 0, f"{what} disp: {len(bad)} mismatches, first {bad[:5].tolist()}"


def test_small_scene_no_downscale():
    # 360 x 248, Dmax 36, no downscaling: spans several 64-column strips, six
    # disparity slabs and a ragged last strip and slab
    s = scenes.make_scene(360, 248, 36, planes=12, seed=0)
    p = _params(downscale=0)
    _compare(_run_gpu(s.left, s.right, 36, p), oracle.pipeline(s.left, s.right, 36, p), "360x248/36")


def test_paper_shape_full_pipeline():
    # the paper's workload shape: 1436 x 992, Dmax 145 -> 718 x 496, D 73
    s = scenes.make_scene(1436, 992, 145, planes=40, seed=0)
    p = _params()
    _compare(_run_gpu(s.left, s.right, 145, p), oracle.pipeline(s.left, s.right, 145, p), "1436x992/145")


@pytest.mark.parametrize("W,H,dmax", [(1482, 994, 128), (1444, 960, 380)])
def test_other_middlebury_like_shapes(W, H, dmax):
    # the Pipes-like and Vintage-like shapes of Sec. V (D = 64 and 190 after
    # halving; 741 and 722 processed columns)
    s = scenes.make_scene(W, H, dmax, planes=40, seed=W)
    p = _params()
    _compare(_run_gpu(s.left, s.right, dmax, p), oracle.pipeline(s.left, s.right, dmax, p), f"{W}x{H}/{dmax}")


@pytest.mark.parametrize("tile", range(NUM_TILES))
def test_every_tile_shape(tile):
    # each tile shape of the fused kernel gives the oracle's result, on a frame
    # with ragged strips and slabs and both clipped image borders
    s = scenes.make_scene(300, 150, 50, planes=6, seed=12)
    p = _params(downscale=0)
    _compare(_run_gpu(s.left, s.right, 50, p, tile=tile), oracle.pipeline(s.left, s.right, 50, p), f"tile {tile}")


def _flat_blocks(W, H, shift, seed):
    # large flat blocks with faint noise: support arms run to their caps, so
    # vertical windows span the full 2 wy + 1 rows of the ring
    rng = np.random.default_rng(seed)
    base = np.kron(rng.integers(40, 220, size=(H // 64 + 1, W // 48 + 2)), np.ones((64, 48)))
    img = np.clip(base[:H, :W + shift] + rng.integers(-2, 3, size=(H, W + shift)), 0, 255).astype(np.uint8)
    left = np.repeat(img[:, shift:, None], 3, axis=2)
    right = np.repeat(img[:, :W, None], 3, axis=2)
    return np.ascontiguousarray(left), np.ascontiguousarray(right)


@pytest.mark.parametrize("tile", range(NUM_TILES))
def test_full_vertical_arms_every_tile(tile):
    left, right = _flat_blocks(170, 200, 7, seed=tile)
    p = _params(downscale=0)
    r = oracle.pipeline(left, right, 24, p)
    assert max(int(r.arms_l[2].max()), int(r.arms_l[3].max())) == p.wy     # arms reach the cap
    _compare(_run_gpu(left, right, 24, p, tile=tile), r, f"flat tile {tile}")


@pytest.mark.parametrize("W,H,dmax,ds", [
    (7, 5, 3, 0),        # narrower than a warp, fewer rows than the vertical arm cap
    (1, 9, 1, 0),        # one column, one disparity
    (33, 1, 40, 0),      # one row, more disparities than columns
    (65, 3, 7, 0),       # one column past a strip boundary
    (130, 70, 13, 0),    # ragged strip, slab of one
    (5, 4, 9, 1),        # downscaled to 2 x 2
    (257, 129, 64, 1),   # odd full-res size
    (600, 90, 300, 1),   # D = 150 after halving, wider than many strips
    (268, 67, 20, 1),    # fused grey + downscale: W = 8k + 4, odd H (last row's grey)
    (16, 3, 5, 1),       # fused grey + downscale: one output row, odd H
    (8192, 6, 20, 1),    # widest input: processed width 4096, the refine kernel's largest shared memory
    (4096, 3, 10, 0),    # processed width 4096 without downscaling (row kernel)
])
def test_edge_shapes(W, H, dmax, ds):
    s = scenes.make_scene(W, H, dmax, planes=3, seed=W * 7 + H)
    p = _params(downscale=ds)
    _compare(_run_gpu(s.left, s.right, dmax, p), oracle.pipeline(s.left, s.right, dmax, p), f"{W}x{H}/{dmax}")


@pytest.mark.parametrize("wx,wy,tc,scale", [(0, 0, 13, 512), (5, 9, 13, 512), (29, 31, 13, 512),
                                            (21, 31, 40, 512), (21, 31, 13, 2048), (3, 2, 1, 9),
                                            (21, 31, 0, 512),      # no pixel is similar: every arm 0
                                            (29, 31, 256, 512)])   # every pixel is similar: arms at the caps
def test_parameter_variants(wx, wy, tc, scale):
    s = scenes.make_scene(200, 120, 24, planes=6, seed=3)
    p = _params(downscale=0, wx=wx, wy=wy, tc=tc, cost_scale=scale)
    _compare(_run_gpu(s.left, s.right, 24, p), oracle.pipeline(s.left, s.right, 24, p), f"wx{wx} wy{wy}")


@pytest.mark.parametrize("wx,wy,scale", [(41, 31, 512), (61, 31, 512), (141, 27, 512), (141, 31, 480)])
def test_wide_windows_of_table_I(wx, wy, scale):
    # the W_x of Table I beyond 26 per side need the wider prefix tiles; flat
    # blocks 320 pixels wide let the horizontal arms run to the cap. At
    # wx = 141, wy = 31 a window sum can reach (283 * 63) P, which needs a cost
    # scale below 497 for the 24-bit aggregated cost of the WTA key
    rng = np.random.default_rng(wx + wy)
    W, H, shift = 420, 90, 5
    base = np.kron(rng.integers(40, 220, size=(H // 45 + 1, (W + shift) // 320 + 2)), np.ones((45, 320)))
    img = np.clip(base[:H, :W + shift] + rng.integers(-2, 3, size=(H, W + shift)), 0, 255).astype(np.uint8)
    left = np.ascontiguousarray(np.repeat(img[:, shift:, None], 3, axis=2))
    right = np.ascontiguousarray(np.repeat(img[:, :W, None], 3, axis=2))
    p = _params(downscale=0, wx=wx, wy=wy, cost_scale=scale)
    r = oracle.pipeline(left, right, 16, p)
    assert max(int(r.arms_l[0].max()), int(r.arms_l[1].max())) == wx     # arms reach the cap
    _compare(_run_gpu(left, right, 16, p), r, f"wx{wx} wy{wy}")


def test_key_range_is_checked():
    # (2 wx + 1)(2 wy + 1) P must stay below 2^24: wx = 141, wy = 31 at the
    # default scale is refused, one step lower in wy or scale is accepted
    from paper_2212_00488_gb300 import Stereo, _lib
    with pytest.raises(_lib.StereoError) as e:
        Stereo(0, wx=141, wy=31)
    assert e.value.code == _lib.STEREO_EINVAL
    Stereo(0, wx=141, wy=27).close()
    Stereo(0, wx=141, wy=31, cost_scale=480).close()
    with pytest.raises(_lib.StereoError):
        Stereo(0, wx=142)


@pytest.mark.parametrize("mode", [1, 2])
def test_fill_variants(mode):
    # the prior-art fills of Sec. III-E (Fig. 5), downscaled so the scale-up
    # runs on the filled map too
    s = scenes.make_scene(400, 300, 60, planes=8, seed=21 + mode)
    p = _params(fill_mode=mode)
    _compare(_run_gpu(s.left, s.right, 60, p), oracle.pipeline(s.left, s.right, 60, p), f"fill mode {mode}")


def test_max_disparities():
    # 256 processed disparities, the largest the uint8 maps and keys carry
    s = scenes.make_scene(300, 40, 256, planes=4, seed=8)
    p = _params(downscale=0)
    _compare(_run_gpu(s.left, s.right, 256, p), oracle.pipeline(s.left, s.right, 256, p), "D=256")


def test_constant_and_shift_invariants():
    p = _params(downscale=0)
    g = np.full((40, 90, 3), 120, np.uint8)
    r = _run_gpu(g, g, 20, p)
    assert (r["dl"] == 0).all() and (r["dr"] == 0).all()
    left, right = scenes.shift_pair(120, 40, 6, seed=4, channels=1)
    left, right = np.repeat(left, 3, axis=2), np.repeat(right, 3, axis=2)
    r = _run_gpu(left, right, 16, p)
    o = oracle.pipeline(left, right, 16, p)
    assert np.array_equal(r["dl"], o.dl) and np.array_equal(r["dr"], o.dr)
    assert (r["dl"][:, 6 + 21 + 2: 120 - 3 - 21] == 6).mean() > 0.99


def test_host_entry_point_matches_device_entry_point():
    from paper_2212_00488_gb300 import Stereo
    s = scenes.make_scene(400, 300, 60, planes=8, seed=5)
    st = Stereo(0)
    lt = torch.from_numpy(s.left).cuda()
    rt = torch.from_numpy(s.right).cuda()
    dev = st(lt, rt, 60, maps=True)
    torch.cuda.synchronize()
    disp = np.empty((300, 400), np.float32)
    dl = np.empty((150, 200), np.uint8)
    st.compute_host(s.left, s.right, 60, disp, dl=dl)
    assert np.array_equal(disp, dev.disp.cpu().numpy())
    assert np.array_equal(dl, dev.dl.cpu().numpy())
    st.close()


def test_async_host_calls_over_two_contexts():
    # frames queued alternately on two contexts without waiting equal the
    # device-buffer results frame by frame
    from paper_2212_00488_gb300 import Stereo
    frames = [scenes.make_scene(320, 240, 40, planes=6, seed=30 + k) for k in range(4)]
    ref = Stereo(0)
    want = []
    for f in frames:
        d = ref(torch.from_numpy(f.left).cuda(), torch.from_numpy(f.right).cuda(), 40).disp
        want.append(d.cpu().numpy())
    ref.close()
    a, b = Stereo(0), Stereo(0)
    outs = [torch.empty((240, 320), dtype=torch.float32).pin_memory() for _ in frames]
    ins = [(torch.from_numpy(f.left).pin_memory(), torch.from_numpy(f.right).pin_memory()) for f in frames]
    for k, (l, r) in enumerate(ins):
        (a, b)[k % 2].compute_host(l, r, 40, outs[k], wait=False)
    a.sync()
    b.sync()
    for k in range(len(frames)):
        assert np.array_equal(outs[k].numpy(), want[k])
    a.close()
    b.close()


def test_stage_relaunch_and_profiling():
    from paper_2212_00488_gb300 import Stereo, _lib
    from paper_2212_00488_gb300.stereo import stream_handle
    s = scenes.make_scene(300, 200, 40, planes=5, seed=6)
    st = Stereo(0)
    _lib.stereo_set_profiling(st.ctx, True)
    lt = torch.from_numpy(s.left).cuda()
    rt = torch.from_numpy(s.right).cuda()
    out = st(lt, rt, 40, maps=True)
    ms, nframes = _lib.stereo_stage_ms(st.ctx)
    assert nframes == 1
    assert len(ms) == 5 and all(t >= 0 for t in ms) and ms[_lib.STAGE_COSTAGG] > 0
    # grey + downscale, support, fused cost/aggregation/WTA, refine + scale-up
    assert _lib.stereo_last_launch_count(st.ctx) == 4 and ms[_lib.STAGE_UPSCALE] == 0
    first = out.dl.clone()
    for stage in range(_lib.NUM_STAGES):
        _lib.stereo_launch_stage(st.ctx, stage, stream_handle(torch.cuda.current_stream()))
    torch.cuda.synchronize()
    assert torch.equal(first, out.dl)
    st.close()


def test_sampled_profiling():
    # profiling every 3rd compute: 7 computes record frames 0, 3 and 6
    from paper_2212_00488_gb300 import Stereo, _lib
    s = scenes.make_scene(200, 100, 20, planes=4, seed=9)
    st = Stereo(0)
    lt = torch.from_numpy(s.left).cuda()
    rt = torch.from_numpy(s.right).cuda()
    _lib.stereo_set_profiling(st.ctx, 3)
    for _ in range(7):
        st(lt, rt, 20)
    ms, nframes = _lib.stereo_stage_ms(st.ctx)
    assert nframes == 3 and ms[_lib.STAGE_COSTAGG] > 0
    with pytest.raises(_lib.StereoError):
        _lib.stereo_set_profiling(st.ctx, -1)
    st.close()


def test_argument_errors():
    from paper_2212_00488_gb300 import Stereo, _lib
    st = Stereo(0)
    x = torch.zeros((8, 8, 3), dtype=torch.uint8, device="cuda")
    d = torch.zeros((8, 8), dtype=torch.float32, device="cuda")
    with pytest.raises(_lib.StereoError) as e:
        _lib.stereo_compute(st.ctx, x.data_ptr(), x.data_ptr(), 8, 8, 0, d.data_ptr())
    assert e.value.code == _lib.STEREO_EINVAL
    with pytest.raises(_lib.StereoError):
        _lib.stereo_compute(st.ctx, x.data_ptr(), x.data_ptr(), 8, 8, 600, d.data_ptr())
    with pytest.raises(_lib.StereoError):
        _lib.stereo_compute(st.ctx, 0, x.data_ptr(), 8, 8, 4, d.data_ptr())
    st.close()
    small = Stereo(0, mem_cap_bytes=1 << 16)
    big = torch.zeros((600, 800, 3), dtype=torch.uint8, device="cuda")
    with pytest.raises(_lib.StereoError) as e:
        small(big, big, 64)
    assert e.value.code == _lib.STEREO_ENOMEM
    small.close()
    with pytest.raises(_lib.StereoError):
        Stereo(0, wx=200)           # beyond the supported arm cap
    with pytest.raises(_lib.StereoError):
        Stereo(0, cost_scale=1 << 14)   # aggregated costs would overflow the 24-bit key
    with pytest.raises(_lib.StereoError):
        Stereo(0, wx=0, wy=0, cost_scale=40000)   # one cost would overflow the 16-bit table
    st = Stereo(0)
    with pytest.raises(_lib.StereoError):
        _lib.stereo_set_tile(st.ctx, _lib.NUM_TILES)
    assert 0 <= _lib.stereo_get_tile(st.ctx, 1436, 992, 145) < _lib.NUM_TILES
    st.close()


def test_bounded_wait_reports_timeout_and_context_recovers():
    # the fused kernel's producer/consumer waits are bounded: with a limit of
    # zero polls every wait gives up at once, the kernel returns early and the
    # host sees ETIMEOUT; no GPU state is harmed and the next frame is correct
    from paper_2212_00488_gb300 import Stereo, _lib
    s = scenes.make_scene(200, 100, 30, planes=4, seed=2)
    st = Stereo(0, downscale=0)
    lt = torch.from_numpy(s.left).cuda()
    rt = torch.from_numpy(s.right).cuda()
    _lib.stereo_set_wait_limit(st.ctx, 0)
    st(lt, rt, 30, maps=True)
    torch.cuda.synchronize()
    with pytest.raises(_lib.StereoError) as e:
        _lib.stereo_sync(st.ctx)
    assert e.value.code == _lib.STEREO_ETIMEOUT
    _lib.stereo_set_wait_limit(st.ctx, 1 << 20)
    out = st(lt, rt, 30, maps=True)
    torch.cuda.synchronize()
    _lib.stereo_sync(st.ctx)
    ref = oracle.pipeline(s.left, s.right, 30, _params(downscale=0))
    assert np.array_equal(out.dl.cpu().numpy(), ref.dl)
    st.close()

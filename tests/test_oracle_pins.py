"""Pins of the CPU oracle against what the paper and mathematics fix.

None of these tests retypes the oracle's formulas: they check hand-worked
values (tests/golden), closed forms, invariants, library special cases and
brute-force enumeration on tiny inputs, chosen so that a dropped term, a wrong
sign or index, or a transposed operand in the oracle fails one of them.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2212_00488_gb300 import scenes


def _load(golden_dir, name):
    with open(os.path.join(golden_dir, name)) as f:
        return json.load(f)


# --------------------------------------------------------------------------- grey, downscale

def test_grey_hand_values(golden_dir):
    g = _load(golden_dir, "grey_downscale.json")
    for case in g["grey"]:
        rgb = np.array(case["rgb"], np.uint8).reshape(1, 1, 3)
        assert int(oracle.grey(rgb)[0, 0]) == case["grey"], case


def test_grey_keeps_grey_pixels():
    # weights summing to one keep every grey level v -> v
    v = np.arange(256, dtype=np.uint8)
    rgb = np.stack([v, v, v], axis=-1).reshape(16, 16, 3)
    assert np.array_equal(oracle.grey(rgb).ravel(), v)


def test_downscale_hand_cases(golden_dir):
    g = _load(golden_dir, "grey_downscale.json")
    for case in g["downscale"]:
        img = np.zeros((case["H"], case["W"]), np.uint8)
        for x, y, v in case["pixels"]:
            img[y, x] = v
        assert np.array_equal(oracle.downscale(img), np.array(case["out"], np.uint8)), case["work"]


def test_downscale_linear_ramp_interior():
    # Eq. 2: the mean of a symmetric window of a linear image is its centre value
    H, W = 20, 26
    yy, xx = np.mgrid[0:H, 0:W]
    img = (3 * xx + 4 * yy + 7).astype(np.uint8)
    s = oracle.downscale(img)
    Y, X = s.shape
    assert (Y, X) == (10, 13)
    for y in range(1, Y):
        for x in range(1, X):
            if 2 * x + 1 < W and 2 * y + 1 < H:
                assert s[y, x] == img[2 * y, 2 * x]


def test_downscale_constant_and_odd_size():
    img = np.full((9, 7), 77, np.uint8)
    s = oracle.downscale(img)
    assert s.shape == (4, 3) and (s == 77).all()


# --------------------------------------------------------------------------- census

def test_census_hand_patches(golden_dir):
    g = _load(golden_dir, "census_arms.json")
    for case in g["census"]:
        patch = np.array(case["patch"], np.uint8)
        # embed the 3x5 patch with a margin of copies so that no clamping reaches it
        img = np.pad(patch, ((2, 2), (3, 3)), mode="edge")
        code = oracle.census(img)
        assert int(code[1 + 2, 2 + 3]) == case["code"], case["work"]


def test_census_ramps_closed_form():
    xx = np.tile(np.arange(40, dtype=np.int32) * 5, (12, 1)).astype(np.uint8)
    c = oracle.census(xx)
    # left neighbours darker: bits of (-1,-1), (-2,0), (-1,+1) -> 1 + 4 + 16
    assert (c[2:-2, 3:-3] == 21).all()
    yy = xx.T.copy()
    c = oracle.census(yy)
    # rows above darker: (-1,-1) and (+1,-1) -> 1 + 2
    assert (c[3:-3, 2:-2] == 3).all()
    assert (oracle.census(np.full((5, 9), 42, np.uint8)) == 0).all()


def test_census_mirror_permutes_bits():
    rng = np.random.default_rng(3)
    g = rng.integers(0, 256, size=(15, 23), dtype=np.uint8)
    a = oracle.census(g)
    b = oracle.census(g[:, ::-1].copy())[:, ::-1]
    # mirroring swaps dx -> -dx: bit pairs (0,1), (2,3), (4,5) exchange
    perm = np.zeros_like(a)
    for k, kk in [(0, 1), (1, 0), (2, 3), (3, 2), (4, 5), (5, 4)]:
        perm |= ((a >> k) & 1) << kk
    assert np.array_equal(perm, b)


# --------------------------------------------------------------------------- arms

def test_arms_hand_rows(golden_dir):
    g = _load(golden_dir, "census_arms.json")
    for case in g["arms_rows"]:
        row = np.array(case["row"], np.uint8)[None, :]
        hm, hp, vm, vp = oracle.arms(row, case["wx"], 31, case["tc"])
        x = case["x"]
        assert (int(hm[0, x]), int(hp[0, x])) == (case["hm"], case["hp"]), case["work"]
        assert vm[0, x] == 0 and vp[0, x] == 0
        # the same row as a column gives the same counts on the vertical arms
        hm2, hp2, vm2, vp2 = oracle.arms(row.T.copy(), 31, case["wx"], case["tc"])
        assert (int(vm2[x, 0]), int(vp2[x, 0])) == (case["hm"], case["hp"])


def test_arms_fig4_cross(golden_dir):
    c = _load(golden_dir, "census_arms.json")["fig4_cross"]
    n = c["size"]
    img = np.full((n, n), 200, np.uint8)
    img[5, 2:9] = 100
    img[1:10, 5] = 100
    hm, hp, vm, vp = oracle.arms(img, 21, 31, 13)
    x, y = c["centre"]
    assert (hm[y, x], hp[y, x], vm[y, x], vp[y, x]) == (c["hm"], c["hp"], c["vm"], c["vp"])


def test_arms_constant_image_reach_border_or_cap():
    Y, X = 70, 50
    hm, hp, vm, vp = oracle.arms(np.full((Y, X), 9, np.uint8), 21, 31, 13)
    xs = np.arange(X)[None, :]
    ys = np.arange(Y)[:, None]
    assert np.array_equal(hm, np.broadcast_to(np.minimum(21, xs), (Y, X)))
    assert np.array_equal(hp, np.broadcast_to(np.minimum(21, X - 1 - xs), (Y, X)))
    assert np.array_equal(vm, np.broadcast_to(np.minimum(31, ys), (Y, X)))
    assert np.array_equal(vp, np.broadcast_to(np.minimum(31, Y - 1 - ys), (Y, X)))


# --------------------------------------------------------------------------- cost tables

def test_cost_tables_endpoints_and_monotone():
    for scale in (512, 2048, 32768):
        ad, mc = oracle.cost_tables(0.3, 2.3, scale)
        assert ad[0] == 0 and mc[0] == 0
        assert (np.diff(ad) >= 0).all() and (np.diff(mc) > 0).all()
        assert ad[255] < scale and mc[6] < scale


def test_cost_tables_lambda_placement():
    # 1 - exp(-a/(255 lambda)) crosses 1 - 1/e at a = 255 * 0.3 = 76.5 and
    # 1 - exp(-h/2.3) crosses it at h = 2.3: a wrong lambda or scale moves these
    S = 32768
    ad, mc = oracle.cost_tables(0.3, 2.3, S)
    level = S * (1 - 1 / math.e)
    assert ad[76] < level < ad[77]
    assert mc[2] < level < mc[3]


def test_cost_tables_exponential_law():
    # 1 - f(a + b) = (1 - f(a)) (1 - f(b)) holds for any exponential cost; it
    # fails for a dropped term, a sign error or a linear stand-in
    S = 32768
    ad, mc = oracle.cost_tables(0.3, 2.3, S)
    qa = (S - ad.astype(np.float64)) / S
    for a in range(0, 128, 7):
        for b in range(0, 128, 11):
            assert abs(qa[a + b] - qa[a] * qa[b]) < 2.0 / S
    qm = (S - mc.astype(np.float64)) / S
    for a in range(4):
        for b in range(7 - a):
            assert abs(qm[a + b] - qm[a] * qm[b]) < 2.0 / S


# --------------------------------------------------------------------------- cost volume and aggregation

def _tiny_inputs(seed, X=14, Y=10, smooth=True):
    rng = np.random.default_rng(seed)
    gl = rng.integers(60, 200, size=(Y, X)).astype(np.int32)
    if smooth:
        # mixed texture: some runs of similar values so that arms vary
        gl = (gl // 24) * 24 + rng.integers(0, 6, size=(Y, X))
    gl = gl.astype(np.uint8)
    gr = np.roll(gl, -2, axis=1)
    gr[:, -2:] = rng.integers(0, 256, size=(Y, 2))
    gr = np.clip(gr.astype(np.int32) + rng.integers(-3, 4, size=(Y, X)), 0, 255).astype(np.uint8)
    return gl, gr


def _support(arms, x, y):
    hm, hp, vm, vp = arms
    pts = []
    for s in range(-int(vm[y, x]), int(vp[y, x]) + 1):
        yy = y + s
        for t in range(-int(hm[yy, x]), int(hp[yy, x]) + 1):
            pts.append((x + t, yy))
    return pts


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_aggregation_equals_support_enumeration(seed):
    # Eqs. 7-8: the aggregated cost is the sum of C over the 2-D support set of
    # the anchor (its vertical span, each row with that row's own x arms)
    gl, gr = _tiny_inputs(seed)
    Y, X = gl.shape
    D = 6
    cl, cr = oracle.census(gl), oracle.census(gr)
    al, ar = oracle.arms(gl, 4, 3, 13), oracle.arms(gr, 4, 3, 13)
    for (gB, cB, gM, cM, aB, direction) in [(gl, cl, gr, cr, al, -1), (gr, cr, gl, cl, ar, +1)]:
        CA, C = oracle.volume_int(gB, cB, gM, cM, aB, D, direction, want_cost=True)
        for y in range(Y):
            for x in range(X):
                pts = _support(aB, x, y)
                for d in range(D):
                    assert CA[d, y, x] == sum(int(C[d, yy, xx]) for xx, yy in pts)


def test_cost_volume_special_values():
    gl, gr = _tiny_inputs(4)
    Y, X = gl.shape
    D = 5
    cl, cr = oracle.census(gl), oracle.census(gr)
    al = oracle.arms(gl, 4, 3, 13)
    ad, mc = oracle.cost_tables(0.3, 2.3, 512)
    P = int(ad[255] + mc[6])
    _, C = oracle.volume_int(gl, cl, gr, cr, al, D, -1, want_cost=True)
    for d in range(D):
        assert (C[d, :, :d] == P).all()           # left base: x - d < 0 has no match
    # identical images at d = 0 cost nothing; elsewhere the cost is positive
    _, C0 = oracle.volume_int(gl, cl, gl, cl, al, 1, -1, want_cost=True)
    assert (C0 == 0).all()
    assert (C[0] >= 0).all() and (C <= P).all()


def test_right_base_reuse_identity():
    # Eq. 6: C^R(x, y, d) = C^L(x + d, y, d); the oracle computes C^R directly
    gl, gr = _tiny_inputs(5)
    Y, X = gl.shape
    D = 6
    cl, cr = oracle.census(gl), oracle.census(gr)
    al, ar = oracle.arms(gl, 4, 3, 13), oracle.arms(gr, 4, 3, 13)
    _, CL = oracle.volume_int(gl, cl, gr, cr, al, D, -1, want_cost=True)
    _, CR = oracle.volume_int(gr, cr, gl, cl, ar, D, +1, want_cost=True)
    ad, mc = oracle.cost_tables(0.3, 2.3, 512)
    P = int(ad[255] + mc[6])
    for d in range(D):
        assert np.array_equal(CR[d, :, : X - d], CL[d, :, d:])
        assert (CR[d, :, X - d:] == P).all()


# --------------------------------------------------------------------------- WTA invariants

def _supports(g, p):
    return oracle.census(g), oracle.arms(g, p.wx, p.wy, p.tc)


def test_constant_image_gives_zero_disparity():
    g = np.full((20, 30), 128, np.uint8)
    p = oracle.Params(downscale=0)
    c, a = _supports(g, p)
    assert (oracle.wta_int(g, c, g, c, a, 9, -1, p) == 0).all()
    assert (oracle.wta_int(g, c, g, c, a, 9, +1, p) == 0).all()


@pytest.mark.parametrize("d0", [0, 3, 7])
def test_pure_shift_recovers_the_shift(d0):
    left, right = scenes.shift_pair(64, 24, d0, seed=11, channels=1)
    gl, gr = left[..., 0].copy(), right[..., 0].copy()
    p = oracle.Params(downscale=0)
    cl, al = _supports(gl, p)
    cr, ar = _supports(gr, p)
    D = 12
    dl = oracle.wta_int(gl, cl, gr, cr, al, D, -1, p)
    dr = oracle.wta_int(gr, cr, gl, cl, ar, D, +1, p)
    X = gl.shape[1]
    lo, hi = d0 + p.wx + 2, X - 3 - p.wx
    assert (dl[:, lo:hi] == d0).all()
    assert (dr[:, p.wx + 2: X - d0 - 3 - p.wx] == d0).all()


def test_mirror_symmetry_of_the_two_bases():
    # with a mirror-symmetric census, arms, out-of-image penalty and tie rule,
    # D^R(L, R) equals the mirror of D^L(mirror R, mirror L) exactly
    s = scenes.make_scene(96, 40, 14, planes=5, seed=21)
    p = oracle.Params(downscale=0)
    gl, gr = oracle.grey(s.left), oracle.grey(s.right)
    cl, al = _supports(gl, p)
    cr, ar = _supports(gr, p)
    dr = oracle.wta_int(gr, cr, gl, cl, ar, 14, +1, p)
    fl, fr = gr[:, ::-1].copy(), gl[:, ::-1].copy()
    cfl, afl = _supports(fl, p)
    cfr, _ = _supports(fr, p)
    dl_m = oracle.wta_int(fl, cfl, fr, cfr, afl, 14, -1, p)
    assert np.array_equal(dr, dl_m[:, ::-1])


def test_integer_mode_matches_fp64_except_near_ties():
    # the integer mode rounds each term to 1/scale: a support of n cells moves
    # by at most n/scale, so decisions can differ only where the FP64 winner's
    # lead is within 2 n / scale
    s = scenes.make_scene(120, 60, 16, planes=6, seed=5)
    p = oracle.Params(downscale=0)
    gl, gr = oracle.grey(s.left), oracle.grey(s.right)
    cl, al = _supports(gl, p)
    cr, _ = _supports(gr, p)
    D = 16
    di = oracle.wta_int(gl, cl, gr, cr, al, D, -1, p)
    df, best, second = oracle.wta_f64(gl, cl, gr, cr, al, D, -1, p)
    hm, hp, vm, vp = al
    Y, X = gl.shape
    n = np.zeros((Y, X))
    width = hm.astype(np.int64) + hp + 1
    for y in range(Y):
        for x in range(X):
            n[y, x] = width[y - vm[y, x]: y + vp[y, x] + 1, x].sum()
    bound = 2 * n / p.cost_scale
    clear = (second - best) > bound
    assert clear.mean() > 0.5
    assert np.array_equal(di[clear], df[clear])


@pytest.mark.parametrize("scale", [512, 2048])
def test_integer_mode_at_the_paper_shape_differs_only_inside_the_tie_band(scale):
    # 1436 x 992, Dmax 145 -> 718 x 496, D 73, both bases: every pixel whose
    # integer-mode disparity differs from the FP64 mode's (Eqs. 3-5 without
    # quantisation) has an FP64 lead of at most 2 n / scale (n cells in its
    # support, each term rounded by at most half a unit of 1/scale)
    oracle.set_threads(0)
    s = scenes.make_scene(1436, 992, 145, planes=40, seed=0)
    p = oracle.Params(cost_scale=scale)
    (gl, cl, al), (gr, cr, ar) = oracle.supports(s.left, s.right, p)
    D = oracle.processed_dmax(145, 1)
    dli = oracle.wta_int(gl, cl, gr, cr, al, D, -1, p)
    dri = oracle.wta_int(gr, cr, gl, cl, ar, D, +1, p)
    (dlf, bl, sl), (drf, br, sr) = oracle.wta_pair_f64(s.left, s.right, 145, p)
    for di, df, best, second, a in ((dli, dlf, bl, sl, al), (dri, drf, br, sr, ar)):
        band = (second - best) <= 2 * oracle.support_size(a) / scale
        differ = di != df
        assert not (differ & ~band).any()
        assert band.mean() < 0.06 and differ.mean() < 1e-3


def test_support_size_is_the_brute_force_count():
    g = oracle.grey(scenes.make_scene(40, 30, 8, planes=3, seed=2).left)
    a = oracle.arms(g, 5, 4, 13)
    hm, hp, vm, vp = a
    n = oracle.support_size(a)
    for y in range(30):
        for x in range(40):
            want = sum(int(hm[y + t, x]) + int(hp[y + t, x]) + 1 for t in range(-int(vm[y, x]), int(vp[y, x]) + 1))
            assert n[y, x] == want


# --------------------------------------------------------------------------- cross-check, median, fill, upscale

def test_crosscheck_hand_and_pairing():
    dl = np.array([[0, 1, 1, 2, 0]], np.uint8)
    dr = np.array([[0, 1, 2, 9, 0]], np.uint8)
    # x=0: k=0, dr[0]=0 yes; x=1: k=1, dr[0]=0 no; x=2: k=1, dr[1]=1 yes;
    # x=3: k=2, dr[1]=1 no; x=4: k=0, dr[4]=0 yes
    assert oracle.crosscheck(dl, dr).tolist() == [[1, 0, 1, 0, 1]]
    k = np.full((3, 6), 2, np.uint8)
    assert (oracle.crosscheck(k, k) == (np.arange(6) >= 2)).all()


def test_crosscheck_mirror_swap_keeps_matched_pairs():
    rng = np.random.default_rng(9)
    Y, X = 7, 30
    dl = rng.integers(0, 4, size=(Y, X)).astype(np.uint8)
    dr = rng.integers(0, 4, size=(Y, X)).astype(np.uint8)
    g = oracle.crosscheck(dl, dr)
    g2 = oracle.crosscheck(dr[:, ::-1].copy(), dl[:, ::-1].copy())
    pairs = {(y, x, x - int(dl[y, x])) for y in range(Y) for x in range(X) if g[y, x]}
    pairs2 = set()
    for y in range(Y):
        for xp in range(X):
            if g2[y, xp]:
                u = X - 1 - xp
                k = int(dr[y, u])
                pairs2.add((y, u + k, u))
    assert pairs == pairs2


def test_median_matches_library_filter():
    sp = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(2)
    d = rng.integers(0, 60, size=(17, 23)).astype(np.uint8)
    ref = sp.median_filter(d, size=3, mode="nearest")
    assert np.array_equal(oracle.median3(d), ref)
    assert (oracle.median3(np.full((4, 5), 7, np.uint8)) == 7).all()


def test_fill_hand_rows(golden_dir):
    g = _load(golden_dir, "fill.json")
    for case in g["rows"]:
        gcp = np.array([case["gcp"]], np.uint8)
        dm = np.array([case["dm"]], np.uint8)
        gr = np.array([case["grey"]], np.uint8)
        out = oracle.fill(dm, gcp, gr, g["T"])
        assert out[0].tolist() == [float(v) for v in case["out"]], case["work"]


def test_fill_variants_hand_rows(golden_dir):
    g = _load(golden_dir, "fill_variants.json")
    for case in g["rows"]:
        gcp = np.array([case["gcp"]], np.uint8)
        dm = np.array([case["dm"]], np.uint8)
        gr = np.zeros_like(dm)
        for mode, name in ((1, "closer"), (2, "smaller")):
            out = oracle.fill(dm, gcp, gr, 3, mode)
            assert out[0].tolist() == [float(v) for v in case[name]], (name, case["work"])


def test_fill_variants_bound_the_gcps():
    # every filled value of the prior-art modes is one of the row's GCP values
    # (or 0 in a row without GCPs), and the smaller-disparity mode never
    # exceeds the closer-GCP mode between two GCPs
    rng = np.random.default_rng(4)
    gcp = (rng.random((20, 40)) < 0.2).astype(np.uint8)
    dm = rng.integers(0, 60, size=(20, 40)).astype(np.uint8)
    g = rng.integers(0, 255, size=(20, 40)).astype(np.uint8)
    closer, smaller = oracle.fill(dm, gcp, g, 3, 1), oracle.fill(dm, gcp, g, 3, 2)
    for y in range(20):
        vals = set(dm[y][gcp[y] == 1].astype(float).tolist()) or {0.0}
        assert set(closer[y].tolist()) <= vals and set(smaller[y].tolist()) <= vals
        idx = np.flatnonzero(gcp[y])
        if len(idx) >= 2:
            inner = slice(idx[0], idx[-1] + 1)
            assert (smaller[y][inner] <= closer[y][inner]).all()


def test_upscale_closed_forms():
    Y, X = 6, 9
    H, W = 2 * Y, 2 * X
    gs = np.zeros((Y, X), np.uint8)
    gf = np.zeros((H, W), np.uint8)
    c = np.full((Y, X), 7.25, np.float32)
    assert (oracle.upscale(c, gs, gf, 3) == 14.5).all()
    # a ramp along x in low-res units becomes the full-res column index
    ramp = np.tile(np.arange(X, dtype=np.float32), (Y, 1))
    up = oracle.upscale(ramp, gs, gf, 3)
    assert np.array_equal(up[:, : W - 1], np.tile(np.arange(W - 1, dtype=np.float32), (H, 1)))
    assert (up[:, W - 1] == 2 * (X - 1)).all()
    # a ramp along y interpolates linearly in y
    ramp_y = np.tile(np.arange(Y, dtype=np.float32)[:, None], (1, X))
    up = oracle.upscale(ramp_y, gs, gf, 3)
    assert np.array_equal(up[: H - 1], np.tile(np.arange(H - 1, dtype=np.float32)[:, None], (1, W)))


def test_upscale_edge_picks_closer_brightness():
    Y, X = 1, 2
    dp = np.array([[10.0, 30.0]], np.float32)          # differ by 20 > T
    gs = np.array([[100, 200]], np.uint8)
    gf = np.zeros((2, 4), np.uint8)
    gf[0, 1] = 120                                      # closer to the left low-res pixel
    out = oracle.upscale(dp, gs, gf, 3)
    assert out[0].tolist() == [20.0, 20.0, 60.0, 60.0]
    gf[0, 1] = 150                                      # equidistant: the right side
    assert oracle.upscale(dp, gs, gf, 3)[0, 1] == 60.0


# --------------------------------------------------------------------------- whole pipeline

def test_pipeline_shift_without_downscale():
    # equal channels keep the full 0..255 grey spread of the noise, so that
    # one-pixel supports cannot tie at a wrong disparity
    left, right = scenes.shift_pair(80, 30, 5, seed=3, channels=1)
    left, right = np.repeat(left, 3, axis=2), np.repeat(right, 3, axis=2)
    p = oracle.Params(downscale=0)
    r = oracle.pipeline(left, right, 10, p)
    lo, hi = 5 + p.wx + 2, 80 - 3 - p.wx
    # a one-pixel support can still tie at a wrong disparity by chance; the
    # median and the fill remove such isolated pixels
    assert (r.dl[1:-1, lo:hi] == 5).mean() > 0.99
    assert (r.gcp[1:-1, lo:hi] == 1).mean() > 0.99
    assert (r.disp[1:-1, lo:hi] == 5.0).all()


def test_pipeline_shapes_with_downscale():
    s = scenes.make_scene(101, 67, 20, planes=4, seed=1)
    r = oracle.pipeline(s.left, s.right, 20, oracle.Params())
    assert r.dl.shape == (33, 50) and r.disp.shape == (67, 101)
    assert r.dl.max() < oracle.processed_dmax(20, 1) == 10

"""Pins of the FP64 differentiable form of the oracle (soft-argmin over the
normalised cross aggregation, frozen census codes and arms)."""
import numpy as np
import pytest

import oracle


def _setup(seed=0, Y=9, X=14, shift=2):
    rng = np.random.default_rng(seed)
    base = rng.uniform(0.1, 0.9, (Y, X))
    gl = np.round(base * 6) / 6 + rng.uniform(-0.02, 0.02, (Y, X))     # patches, so arms vary
    gr = np.roll(gl, -shift, axis=1) + rng.normal(0, 0.01, (Y, X))
    ql, qr = oracle.quantise(gl), oracle.quantise(gr)
    return gl, gr, oracle.census(ql), oracle.census(qr), oracle.arms(ql, 4, 3, 13)


THETA = np.array([1.0, 0.7, 0.3, 2.3])


def _loss(gl, gr, cl, cr, al, D, th, go):
    return float((oracle.diff_forward_backward(gl, gr, cl, cr, al, D, th) * go).sum())


def _kink_distance(gl, gr, D, y, x):
    """Smallest |gL - gR| over the cells that involve pixel (y, x) of either
    image: a central difference of step h is valid when this exceeds h."""
    X = gl.shape[1]
    dl = [abs(gl[y, x] - gr[y, x - d]) for d in range(D) if x - d >= 0]
    dr = [abs(gl[y, x + d] - gr[y, x]) for d in range(D) if x + d < X]
    return min(dl + dr)


@pytest.mark.parametrize("seed", [0, 1])
def test_gradient_matches_central_differences(seed):
    gl, gr, cl, cr, al = _setup(seed)
    D = 6
    go = np.random.default_rng(seed + 9).normal(size=gl.shape)
    _, g_l, g_r, g_t = oracle.diff_forward_backward(gl, gr, cl, cr, al, D, THETA, go=go)
    h = 1e-3
    for k in range(4):
        tp, tm = THETA.copy(), THETA.copy()
        tp[k] += h
        tm[k] -= h
        fd = (_loss(gl, gr, cl, cr, al, D, tp, go) - _loss(gl, gr, cl, cr, al, D, tm, go)) / (2 * h)
        assert abs(fd - g_t[k]) <= 1e-5 + 1e-4 * abs(g_t[k]), (k, fd, g_t[k])
    rng = np.random.default_rng(seed + 3)
    checked = 0
    for _ in range(40):
        y, x = int(rng.integers(0, gl.shape[0])), int(rng.integers(0, gl.shape[1]))
        # step 1e-3 away from the |.| kink; a fine step anywhere
        for step, rtol in ((h, 1e-3), (1e-6, 1e-5)):
            if step == h and _kink_distance(gl, gr, D, y, x) <= 3 * h:
                continue
            for img, g in ((gl, g_l), (gr, g_r)):
                keep = img[y, x]
                img[y, x] = keep + step
                lp = _loss(gl, gr, cl, cr, al, D, THETA, go)
                img[y, x] = keep - step
                lm = _loss(gl, gr, cl, cr, al, D, THETA, go)
                img[y, x] = keep
                fd = (lp - lm) / (2 * step)
                assert abs(fd - g[y, x]) <= 1e-6 + rtol * abs(g[y, x]), (y, x, step, fd, g[y, x])
                checked += 1
    assert checked >= 60


def test_constant_image_gives_the_mean_disparity():
    # every in-image cost is zero, so the softmax is uniform over d
    Y, X, D = 8, 20, 5
    g = np.full((Y, X), 0.5)
    q = oracle.quantise(g)
    c = oracle.census(q)
    arm = oracle.arms(q, 3, 2, 13)
    dhat = oracle.diff_forward_backward(g, g, c, c, arm, D, THETA)
    inner = dhat[:, (D - 1) + 3:]            # whole support at x >= D - 1
    assert np.allclose(inner, (D - 1) / 2.0, atol=1e-12)


def test_small_temperature_reaches_the_wta():
    # with grey values on the 1/255 grid and w = (1, 1) the costs are exactly
    # the FP64 WTA oracle's; dividing by the support size does not move the
    # argmin, so as tau -> 0 the soft-argmin lands on the WTA disparity
    rng = np.random.default_rng(4)
    Y, X, D = 12, 24, 7
    ql = (np.round(rng.uniform(30, 220, (Y, X)) / 20) * 20).astype(np.uint8) + rng.integers(0, 4, (Y, X)).astype(np.uint8)
    qr = np.roll(ql, -3, axis=1)
    gl, gr = ql / 255.0, qr / 255.0
    cl, cr = oracle.census(ql), oracle.census(qr)
    al = oracle.arms(ql, 4, 3, 13)
    tau = 1e-4
    dhat = oracle.diff_forward_backward(gl, gr, cl, cr, al, D, np.array([1.0, 1.0, 0.3, 2.3]), tau=tau)
    p = oracle.Params(downscale=0, wx=4, wy=3, tc=13)
    dw, best, second = oracle.wta_f64(ql, cl, qr, cr, al, D, -1, p)
    hm, hp, vm, vp = al
    n = np.zeros((Y, X))
    width = hm.astype(np.int64) + hp + 1
    for y in range(Y):
        for x in range(X):
            n[y, x] = width[y - vm[y, x]: y + vp[y, x] + 1, x].sum()
    clear = (second - best) / n > 40 * tau
    assert clear.mean() > 0.5
    assert np.all(np.abs(dhat[clear] - dw[clear]) < 1e-9)

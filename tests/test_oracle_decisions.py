"""Pins of the oracle's FP32 decisions (Sec. 3 tiling and depth order, Eq.
3dgs thresholds) against their FP64 definitions.

The composite / clamp decisions and the tile lists are taken in FP32 with
correctly rounded operations in a stated order (the kernel's precision, so that
both sides decide identically).  What that must preserve is checked here
against FP64:
- the thresholds l = 2 ln(sigma / alpha_min) agree with the FP64 logarithm;
- the FP32 record (centre, conic, Sigma2D) agrees with the FP64 projection to
  FP32 rounding;
- a term is composited by the FP32 rule exactly when sigma exp(-q/2) >=
  alpha_min in FP64, except within 1e-5 (relative) of the threshold;
- the tile lists hold every tile with a composited pixel (brute force over
  every pixel), lie inside the support box, come within a fraction of a pixel of
  the FP64 support ellipse, hold no Gaussian twice, and are in (key, index)
  order."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2501_13975_b300 import synth


def _cfg(**kw):
    c = O.default_config(**kw)
    return {k: (float(np.float32(v)) if isinstance(v, float) else v) for k, v in c.items()}


def _scenes():
    yield synth.tiny_scene(seed=1, n=1000), synth.ring_cameras(4, 128)[0]
    yield synth.tiny_scene(seed=4, n=300, log_scale=(-1.0, 0.3)), synth.ring_cameras(4, 200, height=150)[1]
    yield synth.tiny_scene(seed=9, n=700), synth.ring_cameras(4, 90)[3]


def test_thresholds_match_the_fp64_logarithm():
    rng = np.random.default_rng(3)
    for amin in (1 / 255, 1e-3, 0.05):
        sc = synth.tiny_scene(seed=2, n=2000)
        sc.opacity = rng.uniform(amin, 1.0, sc.n).astype(np.float32)
        sc.opacity[:5] = [amin, 1.0, 0.99, 0.995, 2 * amin]
        cfg = _cfg(alpha_min=amin)
        cam = synth.ring_cameras(4, 64)[0]
        d = O.dec32(sc, cam, cfg)
        pr = O.project(sc, cam, cfg)
        vis = ~pr["culled"] & (sc.opacity >= np.float32(amin))
        sg = sc.opacity.astype(np.float64)
        l64 = 2 * np.log(sg / np.float32(amin).astype(np.float64))
        assert np.all(np.abs(d[11][vis] - l64[vis]) <= 1e-6 * np.maximum(1, l64[vis]))
        amax = np.float64(np.float32(cfg["alpha_max"]))
        hi = vis & (sg > amax)
        assert np.all(np.abs(d[12][hi] - 2 * np.log(sg[hi] / amax)) <= 1e-6)
        assert np.all(d[12][vis & ~hi] == -1)


def test_record_matches_fp64_projection():
    for sc, cam in _scenes():
        cfg = _cfg()
        d = O.dec32(sc, cam, cfg).astype(np.float64)
        pr = O.project(sc, cam, cfg)
        vis = ~pr["culled"] & (sc.opacity >= np.float32(cfg["alpha_min"]))
        assert vis.sum() > 100
        assert np.abs(d[0:2, vis] - pr["pix"][:, vis]).max() <= 2e-4
        con = pr["conic"][:, vis]
        assert np.abs(d[2:5, vis] - con).max() <= 1e-5 * np.abs(con).max(0).max()
        assert np.all(np.abs(d[2:5, vis] - con) <= 1e-4 * np.abs(con).max(0))
        sig = pr["sigma2d"][:, vis]
        det = sig[0] * sig[2] - sig[1] ** 2
        assert np.all(np.abs(d[13, vis] - det / sig[2] ** 2) <= 1e-4 * det / sig[2] ** 2)
        assert np.array_equal(d[9].astype(np.float32), pr["key"])


def test_term_decisions_match_fp64_except_at_the_threshold():
    """Every (pixel, Gaussian) term: FP32 decision vs sigma exp(-q/2) >=
    alpha_min in FP64 (no early stop: t_min = 0)."""
    for sc, cam in _scenes():
        cfg = _cfg(t_min=0.0)
        d = O.dec32(sc, cam, cfg)
        pr = O.project(sc, cam, cfg)
        vis = np.nonzero(~pr["culled"] & (sc.opacity >= np.float32(cfg["alpha_min"])))[0]
        ys, xs = np.mgrid[0:cam.height, 0:cam.width]
        xs, ys = xs.ravel().astype(np.float32), ys.ravel().astype(np.float32)
        n32 = np.zeros(xs.size, np.int64)
        n64 = np.zeros(xs.size, np.int64)
        near = np.zeros(xs.size, np.int64)
        for k in vis:
            ca, cb, cc, l = (np.float32(v) for v in d[[2, 3, 4, 11], k])
            dx = (xs - np.float32(d[0, k])).astype(np.float32)
            dy = (ys - np.float32(d[1, k])).astype(np.float32)
            a = np.float32(ca * dx + np.float32(cb * dy))       # one rounding per operation (fma emulated in FP64)
            a = (cb.astype(np.float64) * dy + a).astype(np.float32)
            q = (dx.astype(np.float64) * a + np.float32(np.float32(cc * dy) * dy)).astype(np.float32)
            c32 = q <= l
            X, Y = xs - pr["pix"][0, k], ys - pr["pix"][1, k]
            A, B, Cc = pr["conic"][:, k]
            q64 = A * X * X + 2 * B * X * Y + Cc * Y * Y
            with np.errstate(divide="ignore"):
                r = np.log(pr["opacity"][k] * np.exp(-0.5 * q64) / cfg["alpha_min"])
            c64 = r >= 0
            n32 += c32
            n64 += c64
            near += (np.abs(r) < 1e-5) & (c32 != c64)
            assert np.all((c32 == c64) | (np.abs(r) < 1e-5)), (k, np.abs(r[c32 != c64]).min())
        img = O.render(sc, cam, cfg)
        assert np.array_equal(img["ncontrib"].ravel(), n32)   # the renderer applies the same rule


def _band_reach64(pr, cfg, k, x0, y0, widen):
    """FP64 statement of the tile test: over the pixel rows [ylo, yhi] of the
    tile inside the padded support's height, the x-extent of the ellipse
    |x - k1 y| <= sqrt(k2 (ry^2 - y^2)) (continuous y: the extremes at the
    rows nearest +-y*) widened by the margin 1e-3 (|k1| + sqrt(k2)) ry + 0.05
    (+ widen), meets an integer column of the tile."""
    px, py = pr["pix"][:, k]
    sxx, sxy, syy = pr["sigma2d"][:, k]
    ell = 2 * np.log(pr["opacity"][k] / cfg["alpha_min"])
    ry = np.sqrt(ell * syy) * 1.0005 + 0.02
    k1, k2 = sxy / syy, (sxx * syy - sxy * sxy) / syy ** 2
    ystar = k1 * ry / np.sqrt(k2 + k1 * k1)
    marg = 0.05 + 1e-3 * (abs(k1) + np.sqrt(k2)) * ry + widen
    ylo, yhi = max(y0, np.ceil(py - ry)), min(y0 + 15, np.floor(py + ry))
    if ylo > yhi:
        return False
    ya, yb = ylo - py, yhi - py
    yr, yl = min(max(ystar, ya), yb), min(max(-ystar, ya), yb)
    xr = px + k1 * yr + np.sqrt(max(k2 * (ry * ry - yr * yr), 0)) + marg
    xl = px + k1 * yl - np.sqrt(max(k2 * (ry * ry - yl * yl), 0)) - marg
    return max(np.ceil(xl), x0) <= min(np.floor(xr), x0 + 15)


@pytest.mark.parametrize("case", [0, 1, 2])
def test_tile_lists_cover_the_support_and_follow_the_ellipse(case):
    sc, cam = list(_scenes())[case]
    cfg = _cfg()
    ranges, ids = O.tile_lists(sc, cam, cfg)
    touch, _ = O.tile_touch(sc, cam, 16, cfg)
    d = O.dec32(sc, cam, cfg)
    pr = O.project(sc, cam, cfg)
    key = pr["key"]
    tx = (cam.width + 15) // 16
    rect_lo, rect_hi = d[15].view(np.uint32), d[16].view(np.uint32)
    listed = {}
    for t in range(ranges.shape[0]):
        lst = ids[ranges[t, 0]:ranges[t, 1]].tolist()
        assert lst == sorted(lst, key=lambda k: (key[k], k)), t
        assert len(set(lst)) == len(lst)
        need = set(np.nonzero(touch[t] == 1)[0].tolist())
        assert need <= set(lst), (t, need - set(lst))      # every composited pixel's tile is listed
        for k in lst:
            listed[(t, k)] = True
    # every tile of every support box: listed exactly when the FP64 band test says so
    # (up to 0.01 px of FP32 rounding either way)
    for k in np.nonzero(d[10] > 0)[0]:
        lo, hi = int(rect_lo[k]), int(rect_hi[k])
        for tyy in range(lo >> 16, hi >> 16):
            for txx in range(lo & 0xFFFF, hi & 0xFFFF):
                t = tyy * tx + txx
                x0, y0 = txx * 16, tyy * 16
                if (t, k) in listed:
                    assert _band_reach64(pr, cfg, k, x0, y0, 0.01), (t, k)
                else:
                    assert not _band_reach64(pr, cfg, k, x0, y0, -0.01), (t, k)
    # the lists follow the ellipses: fewer entries than the boxes' tiles
    assert 0 < len(ids) < d[10].sum()

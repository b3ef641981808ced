"""Host-side checks of the arithmetic the pair emission relies on (no GPU).

1. Support ellipse per tile row.  The support { d : d^T A d <= l } of a
   Gaussian (A = Sigma^-1, l = 2 ln(sigma / alpha_min)) is, per pixel row y
   (relative to the centre), |x - k1 y| <= sqrt(k2 (ry^2 - y^2)) with
   k1 = Sigma_xy / Sigma_yy, k2 = det Sigma / Sigma_yy^2, ry^2 = l Sigma_yy.
   Over the integer pixel rows of one tile row, the emission takes the largest
   x at the row nearest y* = k1 ry / sqrt(k2 + k1^2) (the ellipse's rightmost
   point) and the smallest at the row nearest -y*.  The test restates that
   rule in FP64 and checks it against brute force over every pixel: a tile
   that holds a support pixel is always kept, and a kept tile holds a pixel
   within the margin of the support.

2. Row and column of a pair.  rel / w is taken as trunc(fl(rel * fl(1 / w)))
   in FP32 and corrected by one step either way; this is exact for every
   rel < 2^20 (the product is within 0.25 of the quotient)."""
import numpy as np
import pytest

TILE = 16


def _span_keeps(px, py, sxx, sxy, syy, ell, tx, ty, marg_rel=1e-3, marg_abs=0.05):
    """The emission's rule for tile (tx, ty), in FP64 (no rectangle clip)."""
    det = sxx * syy - sxy * sxy
    k1, k2 = sxy / syy, det / (syy * syy)
    ry = np.sqrt(ell * syy)
    ystar = k1 * ry / np.sqrt(k2 + k1 * k1)
    marg = marg_abs + marg_rel * (abs(k1) + np.sqrt(k2)) * ry
    ylo = max(ty * TILE, np.ceil(py - ry))
    yhi = min(ty * TILE + TILE - 1, np.floor(py + ry))
    if ylo > yhi:
        return False
    ya, yb = ylo - py, yhi - py
    yr, yl = min(max(ystar, ya), yb), min(max(-ystar, ya), yb)
    hr = np.sqrt(max(k2 * (ry * ry - yr * yr), 0.0))
    hl = np.sqrt(max(k2 * (ry * ry - yl * yl), 0.0))
    xr, xl = px + k1 * yr + hr + marg, px + k1 * yl - hl - marg
    return max(np.ceil(xl), tx * TILE) <= min(np.floor(xr), tx * TILE + TILE - 1)


def _random_gaussian(rng):
    ang = rng.uniform(0, np.pi)
    s1, s2 = np.exp(rng.uniform(np.log(0.6), np.log(60.0), 2))
    c, s = np.cos(ang), np.sin(ang)
    R = np.array([[c, -s], [s, c]])
    S = R @ np.diag([s1 * s1, s2 * s2]) @ R.T + 0.3 * np.eye(2)   # the low-pass term
    sigma = rng.uniform(0.01, 0.99)
    ell = 2 * np.log(sigma / (1.0 / 255.0))
    px, py = rng.uniform(20, 236, 2)
    return px, py, S[0, 0], S[0, 1], S[1, 1], ell


@pytest.mark.parametrize("seed", range(6))
def test_tile_rule_keeps_every_support_tile(seed):
    rng = np.random.default_rng(seed)
    gx, gy = np.meshgrid(np.arange(256), np.arange(256))
    kept_total = box_total = 0
    for _ in range(40):
        px, py, sxx, sxy, syy, ell = _random_gaussian(rng)
        if ell <= 0:
            continue
        A = np.linalg.inv(np.array([[sxx, sxy], [sxy, syy]]))
        dx, dy = gx - px, gy - py
        q = A[0, 0] * dx * dx + 2 * A[0, 1] * dx * dy + A[1, 1] * dy * dy
        inside = q <= ell
        rx, ry = np.sqrt(ell * sxx), np.sqrt(ell * syy)
        lam = np.linalg.eigvalsh(A).max()
        for ty in range(16):
            for tx in range(16):
                blk = inside[ty * TILE:(ty + 1) * TILE, tx * TILE:(tx + 1) * TILE]
                keep = _span_keeps(px, py, sxx, sxy, syy, ell, tx, ty)
                if blk.any():
                    assert keep, (seed, tx, ty)
                if keep:
                    # a kept tile holds a pixel within the margin of the support
                    qb = q[ty * TILE:(ty + 1) * TILE, tx * TILE:(tx + 1) * TILE]
                    delta = 0.06 + 1e-3 * (rx + ry) * 2
                    assert np.sqrt(qb.min()) <= np.sqrt(ell) + delta * np.sqrt(lam), (seed, tx, ty)
                # the rectangle's tiles, for the count below
                in_box = (tx * TILE <= px + rx and tx * TILE + TILE - 1 >= px - rx
                          and ty * TILE <= py + ry and ty * TILE + TILE - 1 >= py - ry)
                kept_total += keep and in_box
                box_total += in_box
    # elongated, rotated footprints: the ellipse leaves a good share of its box
    assert kept_total < 0.9 * box_total, (kept_total, box_total)


def test_quotient_by_reciprocal_is_exact():
    f32 = np.float32
    rels = np.concatenate([np.arange(0, 70000, dtype=np.int64),
                           np.random.default_rng(3).integers(0, 1 << 20, 200000)])
    for w in list(range(1, 300)) + [1000, 4095, 4096, 65535]:
        inv = f32(1.0) / f32(w)
        row = (rels.astype(f32) * inv).astype(np.int64)          # FP32 product, truncation
        rem = rels - row * w
        row = np.where(rem < 0, row - 1, np.where(rem >= w, row + 1, row))
        rem = np.where(rem < 0, rem + w, np.where(rem >= w, rem - w, rem))
        assert np.array_equal(row, rels // w), w
        assert np.array_equal(rem, rels % w), w

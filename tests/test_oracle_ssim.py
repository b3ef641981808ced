"""Pins of the oracle's SSIM value (Sec. 4.2 SSIM loss, read as Wang et al.
2004 SSIM per channel: 11x11 Gaussian window of sigma 1.5, normalised,
zero-padded "same" windows, C1 = 0.01^2, C2 = 0.03^2) and of the secondary
views' downsampling (Sec. 4.3), against what the mathematics fixes:

- an impulse image: the window moments around it are the window itself;
- two constant images: interior SSIM = (2ab + C1) / (a^2 + b^2 + C1), and at
  the zero-padded border a closed form in the window mass inside the image;
- random images: the moments equal scipy.ndimage.gaussian_filter (a library
  routine) with the same sigma, radius and zero padding;
- L_S equals the mean of 1 - SSIM over channels and pixels;
- a downsampled camera maps a point at full-resolution pixel pi to
  (pi + 1/2)/f - 1/2; a box-filtered linear ramp has a closed form.

A wrong window sigma or normalisation, C1 and C2 swapped, or sample (N - 1)
moments fail at least one of these."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2501_13975_b300 import synth

C1, C2 = 0.01 ** 2, 0.03 ** 2


def _window_1d(sigma=1.5, radius=5):
    i = np.arange(-radius, radius + 1, dtype=np.float64)
    w = np.exp(-i * i / (2.0 * sigma * sigma))
    return w / w.sum()


def test_impulse_moments_are_the_window():
    H = W = 31
    img = np.zeros((3, H, W))
    img[1, 15, 15] = 1.0
    _, mom = O.ssim_map(img, np.zeros_like(img), O.default_config())
    w = _window_1d()
    win = np.outer(w, w)
    # mu_x at centre p is w(15 - p): the window (symmetric) around the impulse
    np.testing.assert_allclose(mom[1, 0, 10:21, 10:21], win, rtol=0, atol=1e-15)
    np.testing.assert_allclose(mom[1, 2, 10:21, 10:21], win, rtol=0, atol=1e-15)   # x^2 = x for a 0/1 image
    assert abs(mom[1, 0].sum() - 1.0) < 1e-13                                       # normalised
    assert np.all(mom[1, 0][:10] == 0) and np.all(mom[1, 0][21:] == 0)              # radius 5
    assert np.all(mom[0] == 0) and np.all(mom[1, 1] == 0) and np.all(mom[1, 4] == 0)


@pytest.mark.parametrize("a,b", [(0.3, 0.7), (0.9, 0.05), (0.5, 0.5)])
def test_constant_images_closed_form(a, b):
    H, W = 24, 29
    img = np.full((3, H, W), a)
    tgt = np.full((3, H, W), b)
    ss, _ = O.ssim_map(img, tgt, O.default_config())
    inner = ss[:, 5:H - 5, 5:W - 5]
    np.testing.assert_allclose(inner, (2 * a * b + C1) / (a * a + b * b + C1), rtol=1e-10, atol=0)
    # border: the window mass M inside the image makes mu = a M, var = a^2 M (1 - M), cov = a b M (1 - M)
    w = _window_1d()
    mx = np.array([w[max(0, 5 - x):min(11, W + 5 - x)].sum() for x in range(W)])
    my = np.array([w[max(0, 5 - y):min(11, H + 5 - y)].sum() for y in range(H)])
    M = np.outer(my, mx)
    V = M * (1 - M)
    want = (2 * a * b * M * M + C1) * (2 * a * b * V + C2) / (((a * a + b * b) * M * M + C1) * ((a * a + b * b) * V + C2))
    np.testing.assert_allclose(ss[2], want, rtol=1e-10, atol=0)


def test_moments_match_a_library_gaussian_filter():
    from scipy.ndimage import gaussian_filter
    rng = np.random.default_rng(11)
    img = rng.uniform(0, 1, (3, 27, 34))
    tgt = np.clip(img + rng.normal(0, 0.1, img.shape), 0, 1)
    ss, mom = O.ssim_map(img, tgt, O.default_config())
    f = lambda z: gaussian_filter(z, sigma=1.5, truncate=5 / 1.5, mode="constant", cval=0.0)
    for c in range(3):
        x, y = img[c], tgt[c]
        want = [f(x), f(y), f(x * x), f(y * y), f(x * y)]
        for i in range(5):
            np.testing.assert_allclose(mom[c, i], want[i], rtol=0, atol=1e-14)
        mx, my = want[0], want[1]
        vx, vy, cxy = want[2] - mx * mx, want[3] - my * my, want[4] - mx * my
        s = (2 * mx * my + C1) * (2 * cxy + C2) / ((mx * mx + my * my + C1) * (vx + vy + C2))
        np.testing.assert_allclose(ss[c], s, rtol=1e-11, atol=1e-13)
    L = O.loss(img, tgt, O.default_config(), derivs=False)
    assert abs(L["lssim"] - np.mean(1.0 - ss)) < 1e-13


@pytest.mark.parametrize("f", [2, 3])
def test_downsampled_camera_keeps_pixel_centres(f):
    """Output pixel m covers input pixels f m .. f m + f - 1, whose centre is
    f m + (f - 1)/2: a point at input pixel pi lands at (pi + 1/2)/f - 1/2."""
    cam = synth.ring_cameras(4, 120, height=90)[1]
    dc = O.downsample_camera(cam, f)
    assert (dc.width, dc.height) == (120 // f, 90 // f)
    rng = np.random.default_rng(3)
    pts = rng.uniform(-1, 1, (3, 50))

    def pix(c):
        V = np.asarray(c.viewmat, np.float64).reshape(3, 4)
        t = V[:, :3] @ pts + V[:, 3:]
        return np.stack([c.fx * t[0] / t[2] + c.cx, c.fy * t[1] / t[2] + c.cy])

    np.testing.assert_allclose(pix(dc), (pix(cam) + 0.5) / f - 0.5, rtol=0, atol=1e-9)


@pytest.mark.parametrize("f", [2, 3])
def test_box_filtered_ramp_closed_form(f):
    H, W = 12, 18
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    img = np.stack([0.2 + 0.03 * x - 0.01 * y, 0.5 * np.ones_like(x), 0.01 * x * 0 + 0.07 * y])
    out = O.downsample_image(img, f)
    n, m = np.mgrid[0:H // f, 0:W // f].astype(np.float64)
    cx, cy = f * m + (f - 1) / 2, f * n + (f - 1) / 2
    np.testing.assert_allclose(out[0], 0.2 + 0.03 * cx - 0.01 * cy, rtol=0, atol=1e-14)
    np.testing.assert_allclose(out[1], 0.5, rtol=0, atol=1e-15)
    np.testing.assert_allclose(out[2], 0.07 * cy, rtol=0, atol=1e-14)
    # a block-constant image is reproduced exactly
    rng = np.random.default_rng(5)
    blocks = rng.uniform(0, 1, (3, H // f, W // f))
    big = np.repeat(np.repeat(blocks, f, 1), f, 2)
    np.testing.assert_allclose(O.downsample_image(big, f), blocks, rtol=0, atol=1e-15)

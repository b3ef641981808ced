"""Pins of the oracle's loss derivatives and Newton blocks by central finite
differences of the loss itself (Eq. local_hessian_gradient; loss equations of
Sec. 4.2). The blocks come from second-order jets; the FD side only renders
and evaluates the loss, so a dropped term, wrong sign or wrong index in the
jet path fails here."""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from oracle import oracle as O
from tests.oracle_scenes import NOTHRESH, micro_camera, micro_scene


def _loss(handle, cam, target, cfg):
    img = O.render(handle, cam, cfg)["image"]
    return O.loss(img, target, cfg, derivs=False)["loss"]


def _perturb(handle, group, k, i, eps, primary, ch=0):
    h = O._SceneHandle(handle)
    if group == O.POS:
        h.mean[i, k] += eps
    elif group == O.SCALE:
        h.scale[i, k] += eps
    elif group == O.OPACITY:
        h.opacity[k] += eps
    elif group == O.COLOR:
        h.sh[ch, i, k] += eps
    elif group == O.ROT:
        o = primary.center()
        a = h.mean[:, k] - o
        a /= np.linalg.norm(a)
        w, x, y, z = h.quat[:, k]
        r = Rotation.from_rotvec(eps * a) * Rotation.from_quat([x, y, z, w])
        qx, qy, qz, qw = r.as_quat()
        if qw * w + qx * x + qy * y + qz * z < 0:
            qx, qy, qz, qw = -qx, -qy, -qz, -qw
        h.quat[:, k] = [qw, qx, qy, qz]
    return h


def _fd_blocks(group, handle, k, cam, primary, target, cfg, eps, ch=0, hessian=True):
    S = O.sh_count(handle.sh_degree)
    D = O.group_dims(group, S)
    f = lambda hh: _loss(hh, cam, target, cfg)
    g = np.zeros(D)
    H = np.zeros((D, D))
    L0 = f(handle)
    P = lambda i, s: _perturb(handle, group, k, i, s, primary, ch)
    for i in range(D):
        Lp, Lm = f(P(i, eps)), f(P(i, -eps))
        g[i] = (Lp - Lm) / (2 * eps)
        if hessian:
            H[i, i] = (Lp - 2 * L0 + Lm) / eps ** 2
    if hessian:
        for i in range(D):
            for j in range(i + 1, D):
                def PP(si, sj):
                    hh = _perturb(handle, group, k, i, si, primary, ch)
                    return f(_perturb(hh, group, k, j, sj, primary, ch))
                H[i, j] = H[j, i] = (PP(eps, eps) - PP(eps, -eps) - PP(-eps, eps) + PP(-eps, -eps)) / (4 * eps ** 2)
    return g, H


def _unpack(Hp, D):
    H = np.zeros((D, D))
    kk = 0
    for a in range(D):
        for b in range(a, D):
            H[a, b] = H[b, a] = Hp[kk]
            kk += 1
    return H


def _setup(n=3, seed=0, sh_degree=0, lam=0.0, secondary=False):
    cfg = dict(NOTHRESH, lambda_ssim=lam)
    sc = micro_scene(n, seed, sh_degree)
    primary = micro_camera()
    view = micro_camera(eye=(0.6, -0.3, 0.2), target=(0.0, 0.0, 4.0)) if secondary else primary
    tgt_scene = micro_scene(n, seed + 100, sh_degree)
    target = O.render(tgt_scene, view, cfg)["image"]
    h = O.scene_handle(sc)
    img = O.render(h, view, cfg)["image"]
    L = O.loss(img, target, cfg)
    return cfg, h, view, primary, target, L


EPS = {O.POS: 2e-4, O.ROT: 2e-4, O.SCALE: 1e-4, O.OPACITY: 1e-4, O.COLOR: 1e-3}


@pytest.mark.parametrize("group", O.GROUPS)
@pytest.mark.parametrize("lam", [0.0, 0.2])
def test_gradient_matches_fd(group, lam):
    sh_degree = 1 if group == O.COLOR else 0
    cfg, h, view, primary, target, L = _setup(seed=1 + group, sh_degree=sh_degree, lam=lam, secondary=(group == O.ROT))
    blk = O.accum(group, h, view, primary, L["e"], L["h"], cfg)
    S = O.sh_count(sh_degree)
    for k in range(h.n):
        for ch in (range(3) if group == O.COLOR else [0]):
            gfd, _ = _fd_blocks(group, h, k, view, primary, target, cfg, EPS[group], ch, hessian=False)
            gj = blk["g"][ch, :, k] if group == O.COLOR else blk["g"][:, k]
            scale = max(np.abs(gfd).max(), 1e-12)
            assert np.abs(gj - gfd).max() <= 2e-5 * scale + 1e-12, (group, k, ch, gj, gfd)


@pytest.mark.parametrize("group", O.GROUPS)
def test_hessian_matches_fd_l2(group):
    """At lambda = 0 the pixel-diagonal loss Hessian is exact, so the block is
    the exact second derivative of the loss in the group's variables."""
    sh_degree = 1 if group == O.COLOR else 0
    cfg, h, view, primary, target, L = _setup(seed=11 + group, sh_degree=sh_degree, lam=0.0,
                                              secondary=(group in (O.ROT, O.POS)))
    blk = O.accum(group, h, view, primary, L["e"], L["h"], cfg)
    S = O.sh_count(sh_degree)
    D = O.group_dims(group, S)
    for k in range(h.n):
        for ch in (range(3) if group == O.COLOR else [0]):
            _, Hfd = _fd_blocks(group, h, k, view, primary, target, cfg, EPS[group], ch)
            Hp = blk["H"][ch, :, k] if group == O.COLOR else blk["H"][:, k]
            Hj = _unpack(Hp, D)
            scale = max(np.abs(Hfd).max(), 1e-12)
            assert np.abs(Hj - Hfd).max() <= 2e-4 * scale, (group, k, ch, Hj, Hfd)


def test_color_sh3_gradient_and_hessian():
    cfg, h, view, primary, target, L = _setup(n=2, seed=31, sh_degree=3, lam=0.0, secondary=True)
    blk = O.accum(O.COLOR, h, view, primary, L["e"], L["h"], cfg)
    k, ch = 1, 2
    gfd, Hfd = _fd_blocks(O.COLOR, h, k, view, primary, target, cfg, 1e-3, ch)
    assert np.allclose(blk["g"][ch, :, k], gfd, rtol=0, atol=2e-5 * np.abs(gfd).max())
    Hj = _unpack(blk["H"][ch, :, k], 16)
    assert np.abs(Hj - Hfd).max() <= 2e-4 * np.abs(Hfd).max()


@pytest.mark.parametrize("lam", [0.0, 0.2])
def test_pixel_loss_derivatives_fd(lam):
    """e = dL/dc exactly and h = d2L/dc_q^2 (the pixel-diagonal entry), by FD of
    the loss in one pixel value at a time (SSIM windows are zero-padded, so
    border pixels are included)."""
    rng = np.random.default_rng(5)
    img = rng.uniform(0, 1, (3, 24, 20))
    tgt = np.clip(img + rng.normal(0, 0.1, img.shape), 0, 1)
    cfg = dict(lambda_ssim=lam)
    L = O.loss(img, tgt, cfg)
    eps = 1e-4
    for (c, y, x) in [(0, 0, 0), (1, 5, 7), (2, 23, 19), (0, 12, 0), (1, 11, 10)]:
        def f(d):
            im = img.copy()
            im[c, y, x] += d
            return O.loss(im, tgt, cfg, derivs=False)["loss"]
        Lp, L0, Lm = f(eps), f(0.0), f(-eps)
        e_fd = (Lp - Lm) / (2 * eps)
        h_fd = (Lp - 2 * L0 + Lm) / eps ** 2
        assert abs(L["e"][c, y, x] - e_fd) <= 1e-7 * abs(e_fd) + 1e-12
        assert abs(L["h"][c, y, x] - h_fd) <= 1e-4 * abs(h_fd) + 1e-9


def test_ssim_identical_images():
    """SSIM of an image with itself is 1 everywhere: L_S = 0, e = 0."""
    rng = np.random.default_rng(6)
    img = rng.uniform(0, 1, (3, 16, 16))
    L = O.loss(img, img, dict(lambda_ssim=0.2))
    assert abs(L["lssim"]) < 1e-12 and abs(L["l2"]) == 0.0
    assert np.abs(L["e"]).max() < 1e-12


@pytest.mark.parametrize("group", [O.POS, O.SCALE, O.ROT])
def test_blocks_fd_through_frustum_clamp(group):
    """A Gaussian whose centre lies beyond the frustum clamp (tx/tz = 1.05 >
    1.3 * 24/40): its covariance uses the clamped ratio, and the jet-derived
    gradient and Hessian still match FD of the loss."""
    sc = micro_scene(2, 41)
    sc.mean[:, 1] = [4.2, 0.1, 4.0]
    sc.scale[:, 1] = [1.2, 0.9, 1.5]
    sc.opacity[1] = 0.7
    cfg = dict(NOTHRESH, lambda_ssim=0.0)
    cam = micro_camera()
    h = O.scene_handle(sc)
    target = O.render(micro_scene(2, 42), cam, cfg)["image"]
    img = O.render(h, cam, cfg)["image"]
    L = O.loss(img, target, cfg)
    blk = O.accum(group, h, cam, cam, L["e"], L["h"], cfg)
    D = O.group_dims(group, 1)
    gfd, Hfd = _fd_blocks(group, h, 1, cam, cam, target, cfg, EPS[group])
    assert np.abs(blk["g"][:, 1] - gfd).max() <= 2e-5 * np.abs(gfd).max()
    assert np.abs(_unpack(blk["H"][:, 1], D) - Hfd).max() <= 2e-4 * np.abs(Hfd).max()

"""Pins of the oracle's method variants.

Gauss-Newton blocks (the local Gauss-Newton variant Sec. 6 proposes for the
expensive position Hessian): H = sum_p sum_ch h_ch(p) J J^T with J = dc_ch(p)/dy.
The pin builds J by central finite differences of the rendered image (no jets)
and the pixel-diagonal loss Hessian h from the loss routine; at lambda = 0
(h = 1/(3|I|) > 0) the blocks are positive semidefinite, while the full
Newton blocks of the same scene are not.

Group order (Sec. 5, optimisation order): a sweep with a permuted order equals
the per-group steps (render every view, accumulate, solve, apply) composed in
that order from the oracle's single-step routines.

Jacobi over groups (the single-render sweep variant): equals every view
rendered once, every group accumulated and solved at that state, and the steps
applied with the position last, composed from the same routines."""
import numpy as np
import pytest

from oracle import oracle as O
from tests.oracle_scenes import NOTHRESH, micro_camera, micro_scene
from tests.test_oracle_derivatives import EPS, _perturb, _unpack


def _jacobian_fd(group, handle, k, cam, primary, cfg, eps, ch=0):
    """J[a] = d image / d y_a for Gaussian k (central differences of the render)."""
    S = O.sh_count(handle.sh_degree)
    D = O.group_dims(group, S)
    J = []
    for a in range(D):
        ip = O.render(_perturb(handle, group, k, a, eps, primary, ch), cam, cfg)["image"]
        im = O.render(_perturb(handle, group, k, a, -eps, primary, ch), cam, cfg)["image"]
        J.append((ip - im) / (2 * eps))
    return np.stack(J)          # [D][3][H][W]


def _scene(seed, lam, n=3):
    cfg = dict(NOTHRESH, lambda_ssim=lam)
    sc = micro_scene(n, seed, 0)
    cam = micro_camera()
    target = O.render(micro_scene(n, seed + 100, 0), cam, cfg)["image"]
    h = O.scene_handle(sc)
    img = O.render(h, cam, cfg)["image"]
    return cfg, h, cam, target, O.loss(img, target, cfg)


@pytest.mark.parametrize("group", [O.POS, O.ROT, O.SCALE])
@pytest.mark.parametrize("lam", [0.0, 0.2])
def test_gauss_newton_block_is_h_weighted_jacobian_product(group, lam):
    cfg, h, cam, target, L = _scene(51 + group, lam)
    gn = O.accum(group, h, cam, cam, L["e"], L["h"], dict(cfg, gauss_newton=1))
    full = O.accum(group, h, cam, cam, L["e"], L["h"], cfg)
    D = O.group_dims(group, 1)
    for k in range(h.n):
        J = _jacobian_fd(group, h, k, cam, cam, cfg, EPS[group]).reshape(D, -1)
        H_fd = (J * L["h"].reshape(1, -1)) @ J.T
        Hg = _unpack(gn["H"][:, k], D)
        scale = max(np.abs(H_fd).max(), 1e-12)
        assert np.abs(Hg - H_fd).max() <= 2e-4 * scale, (group, k, Hg, H_fd)
        # the gradient is the same in both variants (up to the order of the
        # oracle's threaded sums)
        assert np.allclose(gn["g"][:, k], full["g"][:, k], rtol=1e-12, atol=1e-15)


def test_gauss_newton_blocks_psd_where_full_blocks_are_not():
    """lambda = 0: h > 0, so every Gauss-Newton block is PSD; the full blocks of
    the same scene (away from the optimum) include indefinite ones."""
    n_indef = 0
    for seed in (61, 62, 63, 64):
        cfg, h, cam, target, L = _scene(seed, 0.0, n=4)
        assert np.all(L["h"] > 0)
        for group in (O.POS, O.SCALE):
            gn = O.accum(group, h, cam, cam, L["e"], L["h"], dict(cfg, gauss_newton=1))
            full = O.accum(group, h, cam, cam, L["e"], L["h"], cfg)
            for k in range(h.n):
                Hg = _unpack(gn["H"][:, k], 3)
                if np.abs(Hg).max() == 0:
                    continue
                assert np.linalg.eigvalsh(Hg).min() >= -1e-10 * np.abs(Hg).max()
                n_indef += np.linalg.eigvalsh(_unpack(full["H"][:, k], 3)).min() < -1e-6 * np.abs(Hg).max()
    assert n_indef > 0


def _composed_sweep(scene, cams, targets, knn, t, cfg, order):
    """The sweep written out from single steps, in `order` (Sec. 4.2; views of
    Sec. 4.3: primary full resolution, secondaries downsampled)."""
    K, f = cfg["knn_k"], cfg["downsample"]
    h = O._SceneHandle(O.scene_handle(scene))
    for group in order:
        S = O.sh_count(h.sh_degree)
        acc = None
        for vi in range(K + 1):
            v = t if vi == 0 else int(knn[t, vi - 1])
            cam, tgt = cams[v], targets[v]
            if vi > 0 and f > 1:
                cam, tgt = O.downsample_camera(cams[v], f), O.downsample_image(targets[v], f)
            img = O.render(h, cam, cfg)["image"]
            L = O.loss(img, tgt, cfg)
            acc = O.accum(group, h, cam, cams[t], L["e"], L["h"], cfg, out=acc)
        step = O.solve(group, h, cams[t], acc["g"], acc["H"], cfg)
        h = O.apply(group, h, cams[t], step["step"], cfg)
    return h


def test_sweep_follows_group_order():
    cfg = dict(O.default_config(), lambda_ssim=0.2, knn_k=2, downsample=2)
    sc = micro_scene(5, 71, 1)
    cams = [micro_camera(eye=(0.3 * np.cos(a), 0.3 * np.sin(a), 0.0), target=(0.0, 0.0, 4.0))
            for a in np.linspace(0, 2 * np.pi, 4, endpoint=False)]
    gt = micro_scene(5, 72, 1)
    targets = np.stack([O.render(gt, c, cfg)["image"] for c in cams])
    knn = np.array([[1, 3], [0, 2], [1, 3], [0, 2]], np.int32)
    order = (4, 2, 0, 3, 1)
    got, _, _ = O.sweep(sc, cams, targets, knn, 0, dict(cfg, group_order=order))
    want = _composed_sweep(sc, cams, targets, knn, 0, cfg, order)
    for name in ("mean", "quat", "scale", "opacity", "sh"):
        a, b = getattr(got, name), getattr(want, name)
        assert np.allclose(a, b, rtol=0, atol=1e-12 * max(1.0, np.abs(b).max())), name
    # and it differs from the default order (the order matters)
    dflt, _, _ = O.sweep(sc, cams, targets, knn, 0, cfg)
    assert not np.allclose(dflt.mean, got.mean, rtol=0, atol=1e-9)


def test_bad_group_order_rejected():
    with pytest.raises(ValueError):
        O.cfg_struct(dict(group_order=(0, 1, 2, 3, 3)))


def _views(cams, targets, knn, t, cfg):
    K, f = cfg["knn_k"], cfg["downsample"]
    out = []
    for vi in range(K + 1):
        v = t if vi == 0 else int(knn[t, vi - 1])
        cam, tgt = cams[v], targets[v]
        if vi > 0 and f > 1:
            cam, tgt = O.downsample_camera(cams[v], f), O.downsample_image(targets[v], f)
        out.append((cam, tgt))
    return out


def test_jacobi_over_groups_sweep():
    cfg = dict(O.default_config(), lambda_ssim=0.2, knn_k=2, downsample=2)
    sc = micro_scene(5, 81, 1)
    cams = [micro_camera(eye=(0.3 * np.cos(a), 0.3 * np.sin(a), 0.0), target=(0.0, 0.0, 4.0))
            for a in np.linspace(0, 2 * np.pi, 4, endpoint=False)]
    gt = micro_scene(5, 82, 1)
    targets = np.stack([O.render(gt, c, cfg)["image"] for c in cams])
    knn = np.array([[1, 3], [0, 2], [1, 3], [0, 2]], np.int32)
    t = 1
    got, losses, _ = O.sweep(sc, cams, targets, knn, t, dict(cfg, group_jacobi=1))
    h0 = O._SceneHandle(O.scene_handle(sc))
    acc = {q: None for q in O.GROUPS}
    for vi, (cam, tgt) in enumerate(_views(cams, targets, knn, t, cfg)):
        L = O.loss(O.render(h0, cam, cfg)["image"], tgt, cfg)
        if vi == 0:
            assert np.isclose(losses[0], L["loss"], rtol=1e-12) and np.all(losses[1:] == 0)
        for q in O.GROUPS:
            acc[q] = O.accum(q, h0, cam, cams[t], L["e"], L["h"], cfg, out=acc[q])
    steps = {q: O.solve(q, h0, cams[t], acc[q]["g"], acc[q]["H"], cfg)["step"] for q in O.GROUPS}
    want = h0
    for q in (O.ROT, O.SCALE, O.OPACITY, O.COLOR, O.POS):
        want = O.apply(q, want, cams[t], steps[q], cfg)
    for name in ("mean", "quat", "scale", "opacity", "sh"):
        a, b = getattr(got, name), getattr(want, name)
        assert np.allclose(a, b, rtol=0, atol=1e-12 * max(1.0, np.abs(b).max())), name
    # and it differs from the series sweep
    ser, _, _ = O.sweep(sc, cams, targets, knn, t, cfg)
    assert not np.allclose(ser.quat, got.quat, rtol=0, atol=1e-9)


@pytest.mark.parametrize("group", O.GROUPS)
def test_gradient_step_is_minus_lr_times_gradient(group):
    """First-order baseline: where no trust radius or bound binds, the step is
    exactly -lr g of the (finite-difference pinned) gradient; for opacity the
    barrier's gradient a (-1/s + 1/(1 - s)) is included."""
    sh = 1 if group == O.COLOR else 0
    cfg = dict(NOTHRESH, lambda_ssim=0.2, trust_pos=1e9, trust_rot=1e9, trust_color=1e9, scale_trust=1e9,
               frac_to_boundary=0.999999)
    sc = micro_scene(4, 91, sh)
    cam = micro_camera()
    target = O.render(micro_scene(4, 191, sh), cam, cfg)["image"]
    h = O.scene_handle(sc)
    L = O.loss(O.render(h, cam, cfg)["image"], target, cfg)
    blk = O.accum(group, h, cam, cam, L["e"], L["h"], cfg)
    lr = [0.0] * 5
    lr[group] = 1e-3
    st = O.solve(group, h, cam, blk["g"], blk["H"], dict(cfg, gd_lr=lr))["step"]
    want = -1e-3 * blk["g"]
    if group == O.OPACITY:
        s = h.opacity
        want = -1e-3 * (blk["g"] + O.default_config(**cfg)["barrier_alpha"] * (-1.0 / s + 1.0 / (1.0 - s)))
    assert np.abs(st.reshape(want.shape) - want).max() <= 1e-14 + 1e-12 * np.abs(want).max()


def test_small_gradient_step_lowers_the_loss():
    """The sign: a small step along -g lowers the loss of every group."""
    cfg = dict(NOTHRESH, lambda_ssim=0.2)
    sc = micro_scene(4, 93, 1)
    cam = micro_camera()
    target = O.render(micro_scene(4, 193, 1), cam, cfg)["image"]
    h = O.scene_handle(sc)
    L0 = O.loss(O.render(h, cam, cfg)["image"], target, cfg)
    for group in O.GROUPS:
        blk = O.accum(group, h, cam, cam, L0["e"], L0["h"], cfg)
        lr = [0.0] * 5
        lr[group] = 1e-2 / max(np.abs(blk["g"]).max(), 1e-12) * 1e-3
        st = O.solve(group, h, cam, blk["g"], blk["H"], dict(cfg, gd_lr=lr))["step"]
        h1 = O.apply(group, h, cam, st, cfg)
        L1 = O.loss(O.render(h1, cam, cfg)["image"], target, cfg, derivs=False)["loss"]
        assert L1 < L0["loss"], (group, L1, L0["loss"])

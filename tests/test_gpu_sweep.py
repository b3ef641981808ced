"""Sweep-level parity (Sec. 4.2 group order, Sec. 4.3 secondary targets) and
full-size sampled parity on the scene-scale workload."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2501_13975_b300 import synth  # noqa: E402
from tests.gpu_common import ambiguous_gaussians, oracle_cfg  # noqa: E402


def _scene_setup(n=300, size=64, seed=1):
    sc = synth.tiny_scene(n=n, seed=seed)
    gt = synth.perturbed(sc, seed=2, sd=0.05)
    cams = synth.ring_cameras(4, size)
    return sc, gt, cams


@pytest.mark.parametrize("order", [(0, 1, 2, 3, 4), (4, 2, 0, 3, 1)])
def test_native_sweep_equals_call_sequence(order):
    """gs2_sweep (native driver) = the same sequence of individual C-ABI calls
    (project, raster, accumulate per view with downsampled secondaries, solve,
    apply per group, in the configured group order, which also decides which
    pass sorts by depth and which reuse the order); differences only from
    atomic summation order."""
    from paper_2501_13975_b300 import gs2
    sc, gt, cams = _scene_setup()
    ctx = gs2.Context(sc.n, 64, 64, 0, config=dict(group_order=order))
    ocfg = oracle_cfg(ctx.config)
    targets = [torch.tensor(O.render(gt, c, ocfg)["image"].astype(np.float32), device="cuda") for c in cams]
    centres = np.stack([c.center() for c in cams]).astype(np.float32)
    sphere = ctx.bounding_sphere(gs2.DeviceScene.from_host(sc)).cpu().numpy()
    knn = gs2.camera_knn(centres, sphere, 3)
    t = 1
    a = gs2.DeviceScene.from_host(sc)
    la = torch.zeros(10, dtype=torch.float64, device="cuda")
    ctx.sweep(a, cams, targets, knn, t, la)
    b = gs2.DeviceScene.from_host(sc)
    lb = torch.zeros(10, dtype=torch.float64, device="cuda")
    views = [t] + list(knn[t])
    for group in order:
        blocks = ctx.blocks_buffer(group, sc.n, 0, 4)
        for slot, v in enumerate(views):
            if slot == 0:
                cam, tgt = cams[v], targets[v]
            else:
                cam, tgt = gs2.camera_downsample(cams[v], 2), ctx.downsample(targets[v], 2)
            proj = ctx.project(b, cam)
            img, rs = ctx.raster_fwd(b, cam, proj)
            ctx.accum(group, b, cam, cams[t], proj, rs, img, tgt, slot, blocks,
                      loss=lb[2 * group:2 * group + 2] if slot == 0 else None)
        step = ctx.solve(group, blocks, 4, b, cams[t])
        ctx.apply(group, step, b, cams[t])
    torch.cuda.synchronize()
    for name in ("mean", "quat", "scale", "opacity", "sh"):
        x, y = getattr(a, name), getattr(b, name)
        d = float((x - y).abs().max())
        assert d <= 1e-4 * max(1.0, float(y.abs().max())), (name, d)
    assert torch.allclose(la, lb, rtol=1e-5, atol=0)


def test_jacobi_over_groups_equals_call_sequence():
    """group_jacobi: gs2_sweep = every view projected and rendered once, every
    group accumulated from that render into its own blocks, all solved, and
    the steps applied with the position last (individual C-ABI calls)."""
    from paper_2501_13975_b300 import gs2
    sc, gt, cams = _scene_setup()
    ctx = gs2.Context(sc.n, 64, 64, 0, config=dict(group_jacobi=1))
    ocfg = oracle_cfg(ctx.config)
    targets = [torch.tensor(O.render(gt, c, ocfg)["image"].astype(np.float32), device="cuda") for c in cams]
    centres = np.stack([c.center() for c in cams]).astype(np.float32)
    sphere = ctx.bounding_sphere(gs2.DeviceScene.from_host(sc)).cpu().numpy()
    knn = gs2.camera_knn(centres, sphere, 3)
    t = 3
    a = gs2.DeviceScene.from_host(sc)
    ctx.sweep(a, cams, targets, knn, t)
    b = gs2.DeviceScene.from_host(sc)
    views = [t] + list(knn[t])
    blocks = {g: ctx.blocks_buffer(g, sc.n, 0, 4) for g in gs2.GROUPS}
    for slot, v in enumerate(views):
        if slot == 0:
            cam, tgt = cams[v], targets[v]
        else:
            cam, tgt = gs2.camera_downsample(cams[v], 2), ctx.downsample(targets[v], 2)
        proj = ctx.project(b, cam)
        img, rs = ctx.raster_fwd(b, cam, proj)
        for g in gs2.GROUPS:
            ctx.accum(g, b, cam, cams[t], proj, rs, img, tgt, slot, blocks[g])
    steps = {g: ctx.solve(g, blocks[g], 4, b, cams[t]) for g in gs2.GROUPS}
    for g in (gs2.ROT, gs2.SCALE, gs2.OPACITY, gs2.COLOR, gs2.POS):
        ctx.apply(g, steps[g], b, cams[t])
    torch.cuda.synchronize()
    ctx.check()
    for name in ("mean", "quat", "scale", "opacity", "sh"):
        x, y = getattr(a, name), getattr(b, name)
        d = float((x - y).abs().max())
        assert d <= 1e-4 * max(1.0, float(y.abs().max())), (name, d)


@pytest.mark.parametrize("lanes", [0, 1])
def test_profile_counts_every_stage(lanes):
    """With profiling on, one sweep (4 views x 5 groups) times 20 binnings,
    20 compositings, 20 loss passes and 20 accumulations, and its counters
    match the views' pixels and the tile lists' pairs."""
    from paper_2501_13975_b300 import gs2
    sc, gt, cams = _scene_setup()
    ctx = gs2.Context(sc.n, 64, 64, 0)
    ocfg = oracle_cfg(ctx.config)
    targets = [torch.tensor(O.render(gt, c, ocfg)["image"].astype(np.float32), device="cuda") for c in cams]
    centres = np.stack([c.center() for c in cams]).astype(np.float32)
    sphere = ctx.bounding_sphere(gs2.DeviceScene.from_host(sc)).cpu().numpy()
    knn = gs2.camera_knn(centres, sphere, 3)
    ctx.set_tuning(view_lanes=lanes)
    a = gs2.DeviceScene.from_host(sc)
    ctx.profile(True)
    ctx.sweep(a, cams, targets, knn, 0)
    p = ctx.profile_read()
    ctx.profile(False)
    ctx.check()
    assert p["stage_count"] == dict(binning=20, compositing=20, loss=20)
    assert all(p["stage_ms"][k] > 0 for k in ("binning", "compositing", "loss"))
    assert list(p["accum_launches"]) == [4, 4, 4, 4, 4]
    assert np.all(p["accum_ms"] > 0)
    assert list(p["binnings"]) == [4, 4, 4, 4, 4]
    assert list(p["pixels"]) == [64 * 64 + 3 * 32 * 32] * 5
    assert np.all(p["pairs"] > 0) and np.all(p["evaluations"] > 0)
    # the tile lists keep the tiles the support ellipses reach: a subset of the sorted pairs
    assert np.all(p["listed"] > 0) and np.all(p["listed"] <= p["pairs"])


@pytest.mark.parametrize("variant", [{}, {"group_order": (4, 2, 0, 3, 1)}, {"gauss_newton": 1},
                                     {"group_jacobi": 1}, {"gd_lr": (2.0, 20.0, 0.5, 2.0, 20.0)}],
                         ids=["paper", "order-42031", "gauss-newton", "jacobi-groups", "gradient-steps"])
def test_sweep_parity_with_oracle(variant):
    """One full native sweep on the GPU vs the oracle's sweep (FP64 state
    throughout, so the two drift apart by FP32 rounding from group to group):
    the primary loss seen by each group agrees to 1e-3 and every parameter row,
    the quaternions included, moves by the same update: every Gaussian within
    2e-3 of its update (the lockstep test of test_gpu_steps checks each
    group's step against its propagated bound).  Also for a
    permuted group order, Gauss-Newton blocks, Jacobi over groups and
    gradient steps."""
    from paper_2501_13975_b300 import gs2
    sc, gt, cams = _scene_setup(n=300, size=64)
    ctx = gs2.Context(sc.n, 64, 64, 0, config=variant)
    ocfg = oracle_cfg(ctx.config)
    tg_np = np.stack([O.render(gt, c, ocfg)["image"] for c in cams]).astype(np.float32)
    targets = [torch.tensor(x, device="cuda") for x in tg_np]
    sphere = O.bounding_sphere(sc)
    centres = np.stack([c.center() for c in cams])
    nb, _ = O.knn(centres, sphere, 3)
    knn = gs2.camera_knn(centres.astype(np.float32), sphere.astype(np.float32), 3)
    assert np.array_equal(nb, knn)
    t = 2
    ds = gs2.DeviceScene.from_host(sc)
    losses = torch.zeros(10, dtype=torch.float64, device="cuda")
    ctx.sweep(ds, cams, targets, knn, t, losses)
    torch.cuda.synchronize()
    h, olosses, _ = O.sweep(sc, cams, tg_np.astype(np.float64), nb, t, ocfg)
    gl = losses.cpu().numpy().reshape(5, 2)
    gl = gl[:, 0] + ocfg["lambda_ssim"] * gl[:, 1]
    assert np.allclose(gl, olosses, rtol=1e-3), (gl, olosses)
    got = ds.to_host()
    fr = {}
    for name in ("mean", "quat", "scale", "opacity", "sh"):
        x0 = getattr(sc, name).astype(np.float64).reshape(-1, sc.n)
        xo = getattr(h, name).reshape(-1, sc.n)
        xg = getattr(got, name).astype(np.float64).reshape(-1, sc.n)
        if name == "quat":   # q and -q are the same rotation; compare unit quaternions
            xg = xg / np.linalg.norm(xg, axis=0)
            xo = xo / np.linalg.norm(xo, axis=0)
        upd = np.linalg.norm(xo - x0, axis=0)
        err = np.linalg.norm(xg - xo, axis=0)
        ok = err <= 2e-3 * upd + 1e-6
        fr[name] = float(ok.mean())
    print(variant, "fraction of Gaussians within 2e-3 of their update:", fr)
    for name, f in fr.items():
        assert f == 1.0, (name, f)


def _crop(cam, x0, y0, w, h):
    """A window of cam as a camera of its own, with cam's frustum clamp limits."""
    lx = float(np.float32(1.3) * (np.float32(0.5) * np.float32(cam.width)) / np.float32(cam.fx))
    ly = float(np.float32(1.3) * (np.float32(0.5) * np.float32(cam.height)) / np.float32(cam.fy))
    return synth.Camera(w, h, cam.fx, cam.fy, cam.cx - x0, cam.cy - y0, cam.viewmat, lx, ly)


@pytest.fixture(scope="module")
def scene_workload():
    gt = synth.spread_scene()
    cams = synth.trajectory_cameras()
    return gt, cams


def test_full_size_render_sampled(scene_workload):
    """Scene workload at full size (1M Gaussians, 1600x1040, the bench's
    configuration): the GPU image on three 8x8 windows equals the oracle's
    brute-force render of those pixels (crop cameras) within 1e-5."""
    from paper_2501_13975_b300 import gs2
    gt, cams = scene_workload
    cam = cams[17]
    ctx = gs2.Context(gt.n, cam.width, cam.height, 3, 48_000_000)
    ds = gs2.DeviceScene.from_host(gt)
    proj = ctx.project(ds, cam)
    img, _ = ctx.raster_fwd(ds, cam, proj)
    torch.cuda.synchronize()
    ctx.check()
    img = img.cpu().numpy()
    ocfg = oracle_cfg(ctx.config)
    checked = 0
    worst = []
    for (x0, y0) in [(792, 516), (100, 900), (1500, 40)]:
        r = O.render(gt, _crop(cam, x0, y0, 8, 8), ocfg)
        ok = r["margin"] >= 1e-4
        d = np.abs(img[:, y0:y0 + 8, x0:x0 + 8] - r["image"]).max(0)
        nc = r["ncontrib"]
        mag = np.abs(r["image"]).max(0)
        for yy, xx in zip(*np.nonzero(ok)):
            worst.append((float(d[yy, xx]), int(nc[yy, xx]), float(mag[yy, xx])))
        checked += int(ok.sum())
    worst.sort(reverse=True)
    print("worst (diff, ncontrib, |c|):", worst[:8])
    assert checked >= 150
    assert worst[0][0] <= 1e-5, worst[:8]


def test_full_size_tile_lists_bit_exact(scene_workload):
    """Scene workload at full size (1M Gaussians, 1600x1040, about 15M listed
    pairs): the GPU's tile lists equal the oracle's plain-loop binning, every
    tile, Gaussian for Gaussian, in (depth key, index) order."""
    from paper_2501_13975_b300 import gs2
    gt, cams = scene_workload
    cam = cams[17]
    ctx = gs2.Context(gt.n, cam.width, cam.height, 3, 48_000_000)
    ocfg = oracle_cfg(ctx.config)
    ds = gs2.DeviceScene.from_host(gt)
    proj = ctx.project(ds, cam)
    ctx.raster_fwd(ds, cam, proj)
    torch.cuda.synchronize()
    ctx.check()
    ranges, ids, m = ctx.debug_tiles(cam.width, cam.height, capacity=48_000_000)
    ranges = ranges.cpu().numpy().astype(np.int64)
    ids = ids.cpu().numpy().view(np.uint32)
    oranges, oids = O.tile_lists(gt, cam, ocfg)
    oranges = oranges.astype(np.int64)
    glen, olen = ranges[:, 1] - ranges[:, 0], oranges[:, 1] - oranges[:, 0]
    assert len(oids) > 5_000_000
    assert np.array_equal(glen, olen), np.nonzero(glen != olen)[0][:5]
    ne = olen > 0
    assert np.array_equal(ranges[ne, 0], oranges[ne, 0])
    assert np.array_equal(ids[:len(oids)], oids)


@pytest.mark.parametrize("group", [0, 2])
def test_full_size_blocks_on_crop_view(scene_workload, group):
    """All 1M Gaussians (SH degree 3) against a 32x24 crop view of a scene
    camera (L2 loss, so a decision near a threshold affects only its own pixel):
    the GPU's blocks equal the oracle's within the block tolerances
    (position and scaling; the oracle's 16-variable colour jets for 1M
    Gaussians would need ~11 GB, colour at full size is covered by the
    sampled render)."""
    from paper_2501_13975_b300 import gs2
    from tests.test_gpu_parity import _colour_full
    from tests.gpu_common import rel_err
    gt, cams = scene_workload
    train = synth.perturbed(gt, seed=4, sd=0.02)
    cam = _crop(cams[5], 780, 500, 32, 24)
    ctx = gs2.Context(gt.n, 32, 24, 3, 8_000_000, dict(lambda_ssim=0.0))
    ocfg = oracle_cfg(ctx.config)
    target = O.render(gt, cam, ocfg)["image"].astype(np.float32)
    ds = gs2.DeviceScene.from_host(train)
    proj = ctx.project(ds, cam)
    img, rs = ctx.raster_fwd(ds, cam, proj)
    blocks = ctx.blocks_buffer(group, train.n, 3, 1)
    ctx.accum(group, ds, cam, cam, proj, rs, img, torch.tensor(target, device="cuda"), 0, blocks)
    torch.cuda.synchronize()
    ctx.check()
    orc = O.render(train, cam, ocfg)
    L = O.loss(orc["image"], target, ocfg)
    ob = O.accum(group, train, cam, cam, L["e"], L["h"], ocfg)
    amb, _ = ambiguous_gaussians(O, train, cam, ocfg, orc["margin"], thresh=2e-5)
    b = blocks.cpu().numpy()
    n = train.n
    if group == 4:
        g, H = _colour_full(b, 1, 16, n)
    else:
        g = b[:3 * n].reshape(3, n)
        H = b[3 * n:9 * n].reshape(6, n)
    keep = ~amb & (ob["npix"] > 0)
    assert keep.sum() >= 20
    gs = np.maximum(ob["gabs"], 1e-6 * ob["gabs"].max())
    hs = np.maximum(ob["Habs"], 1e-6 * ob["Habs"].max())
    assert rel_err(g[..., keep], ob["g"][..., keep], gs[..., keep]) <= 1e-4
    assert rel_err(H[..., keep], ob["H"][..., keep], hs[..., keep]) <= 1e-3

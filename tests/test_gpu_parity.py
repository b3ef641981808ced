"""GPU (CUDA path through the C ABI) vs FP64 oracle, element by element on the
same seeded inputs.

Tolerances: images <= 1e-5 max abs, gradients <= 1e-4 relative, Hessian
blocks <= 1e-3 relative, tile binning and sort order bit-exact.  "Relative" for a block entry is relative to the oracle's sum
of absolute per-pixel terms of that entry (the scale FP32 accumulation error
grows with), floored at 1e-6 of the largest such scale.  Whether a term is
composited or clamped, and which tiles list a Gaussian, are FP32 decisions
that the oracle takes identically; only the early stop at t_min is taken in
FP64 by the oracle, and terms within 2e-5 (relative) of it are excluded and
counted (the result of such a decision is not unique between FP32 and FP64)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2501_13975_b300 import synth  # noqa: E402
from tests.gpu_common import ambiguous_gaussians, oracle_cfg, rel_err  # noqa: E402


@pytest.fixture(scope="module")
def gs2():
    from paper_2501_13975_b300 import gs2 as m
    return m


def _setup(gs2, scene, cams, cfg=None, max_sh=3, max_pairs=0):
    gcfg = gs2.default_config(**(cfg or {}))
    W = max(c.width for c in cams)
    H = max(c.height for c in cams)
    ctx = gs2.Context(scene.n, W, H, max_sh, max_pairs, gcfg)
    return ctx, gcfg, oracle_cfg(gcfg)


def _tiny(n=1000, size=128, sh=0, seed=1):
    sc = synth.tiny_scene(seed=seed, n=n, sh_degree=sh)
    if sh > 0:
        rng = np.random.default_rng(seed + 50)
        sc.sh[:, 1:, :] = rng.normal(0, 0.1, sc.sh[:, 1:, :].shape).astype(np.float32)
    cams = synth.ring_cameras(4, size)
    return sc, cams


def _render_both(gs2, ctx, ocfg, sc, cam):
    ds = gs2.DeviceScene.from_host(sc)
    proj = ctx.project(ds, cam)
    img, rs = ctx.raster_fwd(ds, cam, proj)
    torch.cuda.synchronize()
    ctx.check()
    orc = O.render(sc, cam, ocfg)
    return ds, proj, img, rs, orc


@pytest.mark.parametrize("size", [128, 100])
def test_project_parity_and_keys(gs2, size):
    """The projection's decision fields (centre, conic, thresholds l and lmax,
    k2, padded ry, tile rectangle, tiles touched, depth key) are bit-identical
    to the oracle's FP32 decision record; the colour matches the FP64 oracle."""
    sc, cams = _tiny(sh=3, size=size)
    ctx, gcfg, ocfg = _setup(gs2, sc, cams)
    ds = gs2.DeviceScene.from_host(sc)
    for cam in cams[:2]:
        proj = ctx.project(ds, cam)
        out, keys = ctx.debug_proj(proj, sc.n)
        out = out.cpu().numpy()
        keys = keys.cpu().numpy().view(np.uint32)
        pr = O.project(sc, cam, ocfg)
        dec = O.dec32(sc, cam, ocfg)
        vis = (~pr["culled"]) & (pr["opacity"] >= ocfg["alpha_min"])
        assert (out[10] > 0).sum() > 100
        assert np.all(out[10][~vis] == 0)
        assert np.array_equal(keys, pr["key"].view(np.uint32))
        for row in (0, 1, 2, 3, 4, 5, 10, 11, 12, 13, 14, 15, 16):
            a, b = out[row][vis].view(np.uint32), dec[row][vis].view(np.uint32)
            assert np.array_equal(a, b), (row, np.nonzero(a != b)[0][:5])
        assert rel_err(out[6:9, vis], pr["color"][:, vis], 1.0) < 1e-5


def _lists(ranges, ids):
    return [ids[r0:r1].tolist() for r0, r1 in ranges]


@pytest.mark.parametrize("size,n,big", [(128, 1000, False), (100, 700, False), (40, 300, False), (512, 300, True)])
def test_binning_and_sort_bit_exact(gs2, size, n, big):
    """Every tile list equals the oracle's plain-loop binning of the same FP32
    support test, Gaussian for Gaussian and in the same (depth key, index)
    order.  The large case has footprints of about 20 tile rows, where a box
    holds many tiles the ellipse misses."""
    if big:
        sc = synth.tiny_scene(seed=4, n=n, sh_degree=0, log_scale=(-1.0, 0.3))
        cams = synth.ring_cameras(4, size)
    else:
        sc, cams = _tiny(n=n, size=size)
    ntile = ((size + 15) // 16) ** 2
    ctx, gcfg, ocfg = _setup(gs2, sc, cams, max_pairs=n * ntile if big else 0)
    for cam in cams[:2]:
        ds, proj, img, rs, orc = _render_both(gs2, ctx, ocfg, sc, cam)
        ranges, ids, m = ctx.debug_tiles(cam.width, cam.height, capacity=n * ntile if big else 16 * n)
        got = _lists(ranges.cpu().numpy(), ids.cpu().numpy())
        oranges, oids = O.tile_lists(sc, cam, ocfg)
        want = _lists(oranges, oids)
        assert len(got) == len(want)
        bad = [t for t in range(len(want)) if got[t] != want[t]]
        assert not bad, (bad[:5], got[bad[0]], want[bad[0]])
        assert int(ranges[:, 1].max()) == len(oids) <= m   # sorted pairs past the lists are box tiles the ellipses miss


@pytest.mark.parametrize("size,n,sh", [(128, 1000, 0), (100, 700, 3), (33, 200, 1)])
def test_raster_parity(gs2, size, n, sh):
    sc, cams = _tiny(n=n, size=size, sh=sh)
    ctx, gcfg, ocfg = _setup(gs2, sc, cams)
    for cam in cams[:2]:
        ds, proj, img, rs, orc = _render_both(gs2, ctx, ocfg, sc, cam)
        img = img.cpu().numpy()
        ok = orc["margin"] >= 1e-4
        assert (~ok).mean() <= 1e-3, (~ok).sum()
        assert np.abs(img - orc["image"])[:, ok].max() <= 1e-5
        tf, last = ctx.raster_state(rs, cam.width, cam.height)
        assert np.abs(tf.cpu().numpy() - orc["tfinal"])[ok].max() <= 1e-5


def test_empty_scene_renders_black(gs2):
    sc, cams = _tiny(n=50, size=48)
    sc.opacity[:] = 1e-3    # below alpha_min: nothing is rendered
    ctx, gcfg, ocfg = _setup(gs2, sc, cams)
    ds, proj, img, rs, orc = _render_both(gs2, ctx, ocfg, sc, cams[0])
    assert float(img.abs().max()) == 0.0
    tf, _ = ctx.raster_state(rs, 48, 48)
    assert float(tf.min()) == 1.0


@pytest.mark.parametrize("lam", [0.0, 0.2])
@pytest.mark.parametrize("shape", [(3, 128, 128), (3, 75, 100), (3, 9, 13)])
def test_loss_derivs_parity(gs2, lam, shape):
    rng = np.random.default_rng(7)
    img = rng.uniform(0, 1, shape).astype(np.float32)
    tgt = np.clip(img + rng.normal(0, 0.15, shape), 0, 1).astype(np.float32)
    ctx = gs2.Context(10, shape[2], shape[1], 0, 0, dict(lambda_ssim=lam))
    loss = torch.zeros(2, dtype=torch.float64, device="cuda")
    e, h = ctx.loss_derivs(torch.tensor(img, device="cuda"), torch.tensor(tgt, device="cuda"), loss)
    L = O.loss(img, tgt, oracle_cfg(ctx.config))
    e = e.cpu().numpy()
    h = h.cpu().numpy()
    assert rel_err(e, L["e"], np.abs(L["e"]).max()) < 5e-5
    assert rel_err(h, L["h"], np.abs(L["h"]).max()) < 5e-5
    lv = loss.cpu().numpy()
    assert abs(lv[0] - L["l2"]) <= 1e-5 * L["l2"]
    if lam:
        assert abs(lv[1] - L["lssim"]) <= 1e-4 * L["lssim"]


def _colour_full(blocks, n_views, S, n):
    """Assemble H_ch = sum_v s b b^T, g_ch = sum_v a b from the factored slots (FP64)."""
    b = blocks.reshape(n_views, 6 + S, n).astype(np.float64)
    g = np.zeros((3, S, n))
    H = np.zeros((3, S * (S + 1) // 2, n))
    iu = np.triu_indices(S)
    for v in range(n_views):
        bb = b[v, 6:]
        for ch in range(3):
            g[ch] += b[v, ch] * bb
            outer = bb[:, None, :] * bb[None, :, :]
            H[ch] += b[v, 3 + ch] * outer[iu[0], iu[1]]
    return g, H


def _blocks_case(gs2, group, sh=0, lam=0.2, secondary=False, n=1000, size=128, extra=None, tuning=None,
                 opacity_scale=1.0):
    sc, cams = _tiny(n=n, size=size, sh=sh)
    if opacity_scale != 1.0:   # fainter Gaussians: long walks through the tile lists
        sc.opacity = (sc.opacity * opacity_scale).astype(np.float32)
    ctx, gcfg, ocfg = _setup(gs2, sc, cams, dict(lambda_ssim=lam, **(extra or {})))
    if tuning:
        ctx.set_tuning(**tuning)
    gt = synth.perturbed(sc, seed=2, sd=0.05)
    primary = cams[0]
    view = O.downsample_camera(cams[1], 2) if secondary else primary
    vcam = synth.Camera(view.width, view.height, view.fx, view.fy, view.cx, view.cy,
                        np.asarray(view.viewmat, np.float32))
    target = O.render(gt, vcam, ocfg)["image"].astype(np.float32)
    ds, proj, img, rs, orc = _render_both(gs2, ctx, ocfg, sc, vcam)
    S = (sh + 1) ** 2
    blocks = ctx.blocks_buffer(group, sc.n, sh, 1)
    ctx.accum(group, ds, vcam, primary, proj, rs, img, torch.tensor(target, device="cuda"), 0, blocks)
    torch.cuda.synchronize()
    ctx.check()
    L = O.loss(orc["image"], target, ocfg)
    ob = O.accum(group, sc, vcam, primary, L["e"], L["h"], ocfg)
    amb, _ = ambiguous_gaussians(O, sc, vcam, ocfg, orc["margin"], thresh=2e-5, dilate=(10 if lam else 0))
    b = blocks.cpu().numpy()
    if group == O.COLOR:
        g, H = _colour_full(b, 1, S, sc.n)
    else:
        D = 3 if group in (O.POS, O.SCALE) else 1
        g = b[: D * sc.n].reshape(D, sc.n)
        H = b[D * sc.n: (D + D * (D + 1) // 2) * sc.n].reshape(D * (D + 1) // 2, sc.n)
    return dict(sc=sc, g=g, H=H, ob=ob, amb=amb, ctx=ctx, ocfg=ocfg, ds=ds, cams=cams, vcam=vcam,
                primary=primary, blocks=blocks, target=target, rs=rs)


def _check_blocks(r, gtol=1e-4, htol=1e-3):
    """Entries relative to the oracle's sum of absolute per-pixel terms (the
    scale the FP32 accumulation error grows with; floored at 1e-6 of the
    largest), plus the plain relative error |got - want| / |want| on the
    entries that do not cancel (|want| >= half their absolute-term sum), where
    it is at most twice the first.  Gaussians touched by an ambiguous
    decision are excluded, counted, and held to 5% of the contributors."""
    ob, amb = r["ob"], r["amb"]
    contrib = ob["npix"] > 0
    keep = ~amb & contrib
    excl = int((amb & contrib).sum())
    gs = np.maximum(ob["gabs"], 1e-6 * ob["gabs"].max())
    hs = np.maximum(ob["Habs"], 1e-6 * ob["Habs"].max())
    eg = rel_err(r["g"][..., keep], ob["g"][..., keep], gs[..., keep])
    eh = rel_err(r["H"][..., keep], ob["H"][..., keep], hs[..., keep])
    plain = {}
    for name, got, want, absv in (("g", r["g"], ob["g"], ob["gabs"]), ("H", r["H"], ob["H"], ob["Habs"])):
        sel = (np.abs(want) >= 0.5 * absv) & (absv > 1e-6 * absv.max()) & keep
        plain[name] = float(np.max(np.abs(got[sel] - want[sel]) / np.abs(want[sel]))) if sel.any() else 0.0
    print(f"excluded {excl} of {int(contrib.sum())} contributors; scaled g {eg:.2e} H {eh:.2e}; "
          f"plain relative on non-cancelling entries g {plain['g']:.2e} H {plain['H']:.2e}")
    assert excl <= 0.05 * contrib.sum(), (excl, int(contrib.sum()))
    assert eg <= gtol, eg
    assert eh <= htol, eh
    assert plain["g"] <= 2 * gtol and plain["H"] <= 2 * htol, plain
    # zero where the oracle has no contribution
    assert np.all(r["g"][..., ob["npix"] == 0] == 0)


@pytest.mark.parametrize("group", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("lam", [0.0, 0.2])
def test_blocks_parity_primary(gs2, group, lam):
    r = _blocks_case(gs2, group, sh=(1 if group == O.COLOR else 0), lam=lam)
    _check_blocks(r)


@pytest.mark.parametrize("group", [0, 1, 2])
@pytest.mark.parametrize("lam", [0.0, 0.2])
def test_blocks_parity_gauss_newton(gs2, group, lam):
    """Gauss-Newton blocks (the e-weighted second derivatives left out, Sec. 6)
    against the oracle's Gauss-Newton blocks."""
    r = _blocks_case(gs2, group, lam=lam, extra=dict(gauss_newton=1))
    _check_blocks(r)


@pytest.mark.parametrize("group", [0, 3, 4])
def test_blocks_parity_ragged_tiles(gs2, group):
    """90x90 view: the last tile row and column are ragged (10 of 16), so
    some accumulation threads have their first pixel inside and their second
    (four rows below) outside, and some have both outside."""
    r = _blocks_case(gs2, group, sh=(1 if group == O.COLOR else 0), lam=0.2, n=700, size=90)
    _check_blocks(r)


@pytest.mark.parametrize("px", [2, 4])
@pytest.mark.parametrize("case", [dict(lam=0.0), dict(lam=0.2), dict(lam=0.2, n=700, size=90),
                                  dict(lam=0.2, sh=3, secondary=True, n=1500, size=96),
                                  dict(lam=0.2, extra=dict(gauss_newton=1))],
                         ids=["l2", "ssim", "ragged", "secondary-sh3", "gauss-newton"])
def test_blocks_parity_position_pixels_per_thread(gs2, case, px):
    """The position accumulation with two pixels per thread (a warp per 8x8
    block) and with four (tuning accum_px = 4, the default: two warps per
    tile, one warp reduction per 128 pixels) against the oracle."""
    r = _blocks_case(gs2, O.POS, tuning=dict(accum_px=px), **case)
    assert r["ctx"].tuning()["accum_px"] == px
    _check_blocks(r)


@pytest.mark.parametrize("px", [2, 4])
@pytest.mark.parametrize("case", [dict(lam=0.2, sh=1, n=700, size=90),
                                  dict(lam=0.2, sh=3, secondary=True, n=1500, size=96)],
                         ids=["ragged", "secondary-sh3"])
def test_blocks_parity_colour_pixels_per_thread(gs2, case, px):
    """The colour accumulation, which also follows accum_px: one pixel pair
    per lane (a warp per 8x8 block) and two pairs (a warp per 8x16 column,
    e and h staged in shared memory) against the oracle."""
    r = _blocks_case(gs2, O.COLOR, tuning=dict(accum_px=px), **case)
    assert r["ctx"].tuning()["accum_px"] == px
    _check_blocks(r)


@pytest.mark.parametrize("group", [0, 1, 2, 4])
def test_blocks_parity_secondary_sh3(gs2, group):
    """Downsampled secondary view, primary-view axes, SH degree 3 colour path."""
    r = _blocks_case(gs2, group, sh=3, lam=0.2, secondary=True, n=1500, size=96)
    _check_blocks(r)


def _random_blocks(group, n, S, rng):
    """Random solver inputs: mostly SPD blocks, some indefinite, some zero."""
    if group == O.COLOR:
        return None
    D = 3 if group in (O.POS, O.SCALE) else 1
    g = rng.standard_normal((D, n)) * 10.0 ** rng.uniform(-3, 1, n)
    Hp = np.zeros((D * (D + 1) // 2, n))
    for k in range(n):
        Q, _ = np.linalg.qr(rng.standard_normal((D, D)))
        ev = 10.0 ** rng.uniform(-2, 2, D) * 10.0 ** rng.uniform(-2, 1)
        if k % 7 == 3:
            ev[0] = -ev[0]
        Hf = Q @ np.diag(ev) @ Q.T
        Hp[:, k] = Hf[np.triu_indices(D)]
    g[:, ::11] = 0.0
    Hp[:, ::11] = 0.0
    return g.astype(np.float32), Hp.astype(np.float32)


@pytest.mark.parametrize("group", [0, 1, 2, 3, 4])
def test_gradient_step_parity_same_inputs(gs2, group):
    """First-order baseline (gd_lr): GPU FP32 gradient step vs the oracle's
    FP64 one on identical (FP32) blocks, with the learning rate chosen so that
    some steps are clipped by the trust radii or bounds and some are not."""
    rng = np.random.default_rng(200 + group)
    n = 3000
    sh = 3 if group == O.COLOR else 0
    S = (sh + 1) ** 2
    sc = synth.tiny_scene(n=n, seed=4, sh_degree=sh)
    cams = synth.ring_cameras(4, 64)
    primary = cams[2]
    lr = [0.0] * 5
    lr[group] = {0: 0.05, 1: 0.3, 2: 0.02, 3: 0.05, 4: 0.5}[group]
    ctx, gcfg, ocfg = _setup(gs2, sc, cams, dict(gd_lr=lr))
    ds = gs2.DeviceScene.from_host(sc)
    if group == O.COLOR:
        nv = 4
        slots = np.zeros((nv, 6 + S, n), np.float32)
        slots[:, 0:3] = rng.standard_normal((nv, 3, n))
        slots[:, 3:6] = 10.0 ** rng.uniform(-2, 1, (nv, 3, n))
        slots[:, 6:] = rng.standard_normal((nv, S, n))
        g, H = _colour_full(slots.reshape(-1), nv, S, n)
        ref = O.solve(group, sc, primary, g, H, ocfg)["step"]
        got = ctx.solve(group, torch.tensor(slots.reshape(-1), device="cuda"), nv, ds, primary)
        got = got.cpu().numpy()[: 3 * S * n].reshape(3, S, n)
    else:
        g, Hp = _random_blocks(group, n, S, rng)
        g[:, ::17] = 0.0
        Hp[:, ::17] = 0.0
        blocks = torch.tensor(np.concatenate([g.reshape(-1), Hp.reshape(-1)]), device="cuda")
        got = ctx.solve(group, blocks, 1, ds, primary).cpu().numpy().reshape(-1, n)
        ref = O.solve(group, sc, primary, g.astype(np.float64), Hp.astype(np.float64), ocfg)["step"]
        assert np.all(got[:, ::17] == 0)
    scale = np.abs(ref).max()
    assert scale > 0
    assert np.abs(got - ref).max() <= 1e-5 * scale + 1e-30


@pytest.mark.parametrize("group", [0, 1, 2, 3, 4])
def test_solver_parity_same_inputs(gs2, group):
    """GPU FP32 solve vs the oracle's FP64 solve on identical (FP32) blocks:
    steps within max(1e-3, 1e-5 cond) relative; identical status decisions
    except where the oracle's damping decision was within 1e-3 of its threshold."""
    rng = np.random.default_rng(100 + group)
    n = 3000
    sh = 3 if group == O.COLOR else 0
    S = (sh + 1) ** 2
    sc = synth.tiny_scene(n=n, seed=3, sh_degree=sh)
    cams = synth.ring_cameras(4, 64)
    primary = cams[1]
    ctx, gcfg, ocfg = _setup(gs2, sc, cams)
    ds = gs2.DeviceScene.from_host(sc)
    if group == O.COLOR:
        nv = 4
        slots = np.zeros((nv, 6 + S, n), np.float32)
        slots[:, 0:3] = rng.standard_normal((nv, 3, n))
        slots[:, 3:6] = 10.0 ** rng.uniform(-2, 1, (nv, 3, n))
        slots[:, 6:] = rng.standard_normal((nv, S, n))
        slots[1, :, ::13] = 0.0
        g, H = _colour_full(slots.reshape(-1), nv, S, n)
        blocks = torch.tensor(slots.reshape(-1), device="cuda")
        os_ = O.solve(group, sc, primary, g, H, ocfg)
        ref = os_["step"]
        got = ctx.solve(group, blocks, nv, ds, primary).cpu().numpy()[: 3 * S * n].reshape(3, S, n)
        ok = (os_["status"] == 0) & (os_["info"][:, 1] > 1e-3)
        d = np.linalg.norm(got - ref, axis=1)
        nrm = np.maximum(np.linalg.norm(ref, axis=1), 1e-30)
        tol = np.maximum(1e-3, 1e-5 * os_["cond"])
        assert np.all((d <= tol * nrm)[ok]), np.max((d / nrm / tol)[ok])
        return
    g, Hp = _random_blocks(group, n, S, rng)
    blocks = torch.tensor(np.concatenate([g.reshape(-1), Hp.reshape(-1)]), device="cuda")
    nf = torch.zeros(1, dtype=torch.int32, device="cuda")
    got = ctx.solve(group, blocks, 1, ds, primary, n_failed=nf).cpu().numpy().reshape(-1, n)
    os_ = O.solve(group, sc, primary, g.astype(np.float64), Hp.astype(np.float64), ocfg)
    ref = os_["step"]
    ok = (os_["status"] == 0) & (os_["info"][1] > 1e-3)
    assert ok.sum() > 0.5 * n
    d = np.linalg.norm(got - ref, axis=0)
    nrm = np.maximum(np.linalg.norm(ref, axis=0), 1e-30)
    tol = np.maximum(1e-3, 1e-5 * os_["cond"])
    frac = (d / nrm / tol)[ok]
    assert np.all(frac <= 1.0), (np.max(frac), np.nonzero(ok)[0][np.argmax(frac)])
    assert np.all(got[:, os_["status"] == 2] == 0)
    clear = os_["info"][1] > 1e-3
    assert int(nf.item()) >= int(((os_["status"] == 1) & clear).sum())


def test_apply_parity(gs2):
    """Updates applied to the same FP32 parameters with the same steps."""
    sc, cams = _tiny(n=400, size=64, sh=1)
    ctx, gcfg, ocfg = _setup(gs2, sc, cams)
    rng = np.random.default_rng(3)
    primary = cams[2]
    for group in O.GROUPS:
        ds = gs2.DeviceScene.from_host(sc)
        S = 4
        shape = {0: (3,), 1: (1,), 2: (3,), 3: (1,), 4: (3 * S,)}[group]
        step = (0.01 * rng.standard_normal(shape + (sc.n,))).astype(np.float32)
        if group == O.SCALE:
            step = (0.1 * sc.scale * rng.standard_normal(sc.scale.shape)).astype(np.float32)
        ctx.apply(group, torch.tensor(step.reshape(-1), device="cuda"), ds, primary)
        h = O.apply(group, sc, primary, step.reshape((3, S, sc.n)) if group == O.COLOR else step.reshape(-1, sc.n),
                    ocfg)
        got = ds.to_host()
        for name in ("mean", "quat", "scale", "opacity", "sh"):
            a = getattr(got, name).astype(np.float64)
            b = getattr(h, name)
            assert np.abs(a - b).max() <= 2e-6 * max(1.0, np.abs(b).max()), (group, name)

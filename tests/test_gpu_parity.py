"""GPU (CUDA path through the C ABI) vs FP64 oracle, element by element on the
same seeded inputs.

Tolerances (stated by the build target): images <= 1e-5 max abs, gradients
<= 1e-4 relative, Hessian blocks <= 1e-3 relative, tile binning and sort
order bit-exact.  "Relative" for a block entry is relative to the oracle's sum
of absolute per-pixel terms of that entry (the scale FP32 accumulation error
grows with), floored at 1e-6 of the largest such scale.  Decisions that sit
within 1e-4 (relative) of a threshold in the oracle are excluded and counted
(the result of such a decision is not unique between FP32 and FP64)."""
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
    sc, cams = _tiny(sh=3, size=size)
    ctx, gcfg, ocfg = _setup(gs2, sc, cams)
    ds = gs2.DeviceScene.from_host(sc)
    for cam in cams[:2]:
        proj = ctx.project(ds, cam)
        out, keys = ctx.debug_proj(proj, sc.n)
        out = out.cpu().numpy().astype(np.float64)
        keys = keys.cpu().numpy().view(np.uint32)
        pr = O.project(sc, cam, ocfg)
        vis = (~pr["culled"]) & (pr["opacity"] >= ocfg["alpha_min"])
        assert (out[10] > 0).sum() > 100
        assert np.all(out[10][~vis] == 0)
        assert np.array_equal(keys[vis], pr["key"][vis].view(np.uint32))
        assert rel_err(out[0:2, vis], pr["pix"][:, vis], 1.0) < 2e-4          # pixels
        con = pr["conic"][:, vis]
        assert rel_err(out[2:5, vis], con, np.abs(con).max(0)) < 1e-4
        assert rel_err(out[6:9, vis], pr["color"][:, vis], 1.0) < 1e-5


@pytest.mark.parametrize("size,n,big", [(128, 1000, False), (100, 700, False), (40, 300, False), (512, 300, True)])
def test_binning_and_sort_bit_exact(gs2, size, n, big):
    """Every tile list is sorted by (FP32 depth key, index), holds every
    Gaussian that has a pixel with alpha >= alpha_min in the tile, and no
    Gaussian twice; an extra entry lies within the Gaussian's support box and
    within a fraction of a pixel of its support ellipse (the lists follow the
    ellipse, not its box).  The large case has footprints of about 20 tile rows,
    where a box holds many tiles the ellipse misses."""
    if big:
        sc = synth.tiny_scene(seed=4, n=n, sh_degree=0, log_scale=(-1.0, 0.3))
        cams = synth.ring_cameras(4, size)
    else:
        sc, cams = _tiny(n=n, size=size)
    ntile = ((size + 15) // 16) ** 2
    ctx, gcfg, ocfg = _setup(gs2, sc, cams, max_pairs=n * ntile if big else 0)
    cam = cams[0]
    ds, proj, img, rs, orc = _render_both(gs2, ctx, ocfg, sc, cam)
    ranges, ids, m = ctx.debug_tiles(cam.width, cam.height, capacity=n * ntile if big else 16 * n)
    ranges = ranges.cpu().numpy()
    ids = ids.cpu().numpy()
    touch, rect = O.tile_touch(sc, cam, 16, ocfg)
    pr = O.project(sc, cam, ocfg)
    key = pr["key"]
    tx = (cam.width + 15) // 16
    listed = int(ranges[:, 1].max())   # sorted pairs past it are tiles the ellipses miss
    assert listed <= m
    for t in range(ranges.shape[0]):
        lst = ids[ranges[t, 0]:ranges[t, 1]]
        order = sorted(lst.tolist(), key=lambda k: (key[k], k))
        assert lst.tolist() == order, f"tile {t} not in (key, index) order"
        need = set(np.nonzero(touch[t] == 1)[0].tolist())
        assert need <= set(lst.tolist()), f"tile {t} misses {need - set(lst.tolist())}"
        assert len(set(lst.tolist())) == len(lst), f"tile {t} lists a Gaussian twice"
        x0, y0 = (t % tx) * 16, (t // tx) * 16
        gx, gy = np.meshgrid(np.arange(x0, min(x0 + 16, cam.width)), np.arange(y0, min(y0 + 16, cam.height)))
        for k in set(lst.tolist()) - need:
            r = rect[:, k]
            assert r[0] - 1 <= x0 + 15 and r[2] + 1 >= x0 and r[1] - 1 <= y0 + 15 and r[3] + 1 >= y0, (t, k)
            # an extra entry is a tile the support ellipse nearly reaches: some
            # pixel lies within delta of { d^T A d <= l } (sqrt(q) is a norm
            # with Lipschitz constant sqrt(lambda_max(A)))
            a, b, c = pr["conic"][:, k]
            dx, dy = gx - pr["pix"][0, k], gy - pr["pix"][1, k]
            q = a * dx * dx + 2 * b * dx * dy + c * dy * dy
            lam = 0.5 * (a + c) + np.hypot(0.5 * (a - c), b)
            ell = 2 * np.log(pr["opacity"][k] / ocfg["alpha_min"])
            delta = 0.2 + 5e-3 * (r[2] - r[0] + r[3] - r[1])
            assert np.sqrt(q.min()) <= np.sqrt(ell) + delta * np.sqrt(lam), (t, k, q.min(), ell)
    # the lists cover the support ellipses, not their bounding rectangles
    with np.errstate(invalid="ignore"):
        px0, py0 = np.maximum(np.ceil(rect[0]), 0), np.maximum(np.ceil(rect[1]), 0)
        px1, py1 = np.minimum(np.floor(rect[2]), cam.width - 1), np.minimum(np.floor(rect[3]), cam.height - 1)
        vis = (~pr["culled"]) & (pr["opacity"] > ocfg["alpha_min"]) & (px0 <= px1) & (py0 <= py1)
    box = (px1 // 16 - px0 // 16 + 1) * (py1 // 16 - py0 // 16 + 1)
    assert listed < box[vis].sum(), (listed, box[vis].sum())


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


def _blocks_case(gs2, group, sh=0, lam=0.2, secondary=False, n=1000, size=128, extra=None):
    sc, cams = _tiny(n=n, size=size, sh=sh)
    ctx, gcfg, ocfg = _setup(gs2, sc, cams, dict(lambda_ssim=lam, **(extra or {})))
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
                primary=primary, blocks=blocks, target=target)


def _check_blocks(r, gtol=1e-4, htol=1e-3):
    ob, amb = r["ob"], r["amb"]
    keep = ~amb & (ob["npix"] > 0)
    assert keep.sum() >= 0.5 * (ob["npix"] > 0).sum(), (keep.sum(), amb.sum())
    gs = np.maximum(ob["gabs"], 1e-6 * ob["gabs"].max())
    hs = np.maximum(ob["Habs"], 1e-6 * ob["Habs"].max())
    eg = rel_err(r["g"][..., keep], ob["g"][..., keep], gs[..., keep])
    eh = rel_err(r["H"][..., keep], ob["H"][..., keep], hs[..., keep])
    assert eg <= gtol, eg
    assert eh <= htol, eh
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


@pytest.mark.parametrize("group", [0, 1, 2, 4])
def test_blocks_parity_secondary_sh3(gs2, group):
    """Downsampled secondary view, primary-view axes, SH degree 3 colour path."""
    r = _blocks_case(gs2, group, sh=3, lam=0.2, secondary=True, n=1500, size=96)
    _check_blocks(r)


def _damped(Hf, mu0, tries):
    """The oracle's accepted damping shift for a dense block (numpy, for tolerance scales)."""
    m = np.abs(np.diag(Hf)).mean()
    mu = mu0
    for _ in range(tries + 1):
        A = Hf + mu * m * np.eye(Hf.shape[0])
        if np.linalg.eigvalsh(A).min() > 0:
            return A
        mu *= 10
    return None


def _full(Hp, D):
    H = np.zeros((D, D))
    iu = np.triu_indices(D)
    H[iu] = Hp
    H[(iu[1], iu[0])] = Hp
    return H


@pytest.mark.parametrize("group", [1, 3, 4])
def test_newton_steps_end_to_end(gs2, group):
    """Blocks accumulated on the GPU and solved on the GPU vs the oracle doing
    both: the step error bound is the block tolerances (g 1e-4, H 1e-3 of their
    absolute-term scales) propagated through the damped inverse,
    |dx| <= 1e-3 |x| + |H~^-1| (1e-4 |gabs| + 1e-3 |Habs| |x|)."""
    sh = 1 if group == O.COLOR else 0
    r = _blocks_case(gs2, group, sh=sh, lam=0.2)
    ctx, ds, primary, ob, ocfg = r["ctx"], r["ds"], r["primary"], r["ob"], r["ocfg"]
    step = ctx.solve(group, r["blocks"], 1, ds, primary).cpu().numpy()
    os_ = O.solve(group, r["sc"], primary, ob["g"], ob["H"], ocfg)
    n, S = r["sc"].n, (sh + 1) ** 2
    keep = ~r["amb"] & (ob["npix"] > 0)
    checked = 0
    for k in np.nonzero(keep)[0]:
        chans = range(3) if group == O.COLOR else [None]
        for ch in chans:
            if group == O.COLOR:
                st = os_["status"][ch, k]
                if st != 0 or os_["info"][ch, 1, k] < 1e-3:
                    continue
                Hf = _full(ob["H"][ch, :, k], S)
                ga, Ha = np.abs(ob["gabs"][ch, :, k]).sum(), np.abs(ob["Habs"][ch, :, k]).sum()
                x = os_["step"][ch, :, k]
                y = step[(ch * S) * n + k: (ch * S + S) * n + k: n]
            else:
                st = os_["status"][k]
                if st != 0 or os_["info"][1, k] < 1e-3:
                    continue
                Hf = ob["H"][:, k].reshape(1, 1).copy()
                if group == O.OPACITY:
                    sg = float(r["sc"].opacity[k])
                    a = ocfg["barrier_alpha"]
                    Hf += a * (1 / sg ** 2 + 1 / (1 - sg) ** 2)
                ga, Ha = ob["gabs"][0, k], ob["Habs"][0, k]
                x = os_["step"][:, k]
                y = step[k:k + 1]
            A = _damped(Hf, ocfg["damping_mu0"], ocfg["damping_tries"])
            inv = np.linalg.norm(np.linalg.inv(A), 2)
            bound = 1e-3 * np.linalg.norm(x) + inv * (1e-4 * ga + 1e-3 * Ha * np.linalg.norm(x))
            if group == O.OPACITY:   # fraction-to-boundary clipping is 1-Lipschitz
                bound += 1e-6
            assert np.linalg.norm(y - x) <= bound, (k, ch, y, x, bound)
            checked += 1
    assert checked > 100


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

"""Mixed-precision policy (precision = 1): FP64 accumulation of the per-warp
FP32 partial sums and FP64 re-solves of blocks with condition estimate > 1e6.
Reports the error against the FP64 oracle per block type for both modes
(run with -s to see the table) and checks that the mixed path is not less
accurate and stays within the parity tolerances."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2501_13975_b300 import synth  # noqa: E402
from tests.gpu_common import ambiguous_gaussians, oracle_cfg  # noqa: E402
from tests.test_gpu_parity import _colour_full  # noqa: E402

NAMES = ("position", "rotation", "scaling", "opacity", "colour")


def _case(gs2, group, precision):
    sh = 3 if group == O.COLOR else 0
    sc = synth.tiny_scene(n=1500, seed=17, sh_degree=sh)
    if sh:
        sc.sh[:, 1:, :] = np.random.default_rng(3).normal(0, 0.1, sc.sh[:, 1:, :].shape).astype(np.float32)
    cams = synth.ring_cameras(4, 128)
    gt = synth.perturbed(sc, seed=18, sd=0.05)
    ctx = gs2.Context(sc.n, 128, 128, 3, 0, dict(precision=precision))
    ocfg = oracle_cfg(ctx.config)
    primary = cams[0]
    ds = gs2.DeviceScene.from_host(sc)
    nv = 4
    blocks = ctx.blocks_buffer(group, sc.n, sh, nv)
    ob = None
    for slot, v in enumerate([0, 1, 2, 3]):
        cam = primary if slot == 0 else O.downsample_camera(cams[v], 2)
        cam = synth.Camera(cam.width, cam.height, cam.fx, cam.fy, cam.cx, cam.cy,
                           np.asarray(cam.viewmat, np.float32))
        tgt = O.render(gt, cam, ocfg)["image"].astype(np.float32)
        proj = ctx.project(ds, cam)
        img, rs = ctx.raster_fwd(ds, cam, proj)
        ctx.accum(group, ds, cam, primary, proj, rs, img, torch.tensor(tgt, device="cuda"), slot, blocks)
        r = O.render(sc, cam, ocfg)
        L = O.loss(r["image"], tgt, ocfg)
        ob = O.accum(group, sc, cam, primary, L["e"], L["h"], ocfg, out=ob)
        amb_v, _ = ambiguous_gaussians(O, sc, cam, ocfg, r["margin"], thresh=2e-5, dilate=10)
        amb = amb_v if slot == 0 else (amb | amb_v)
    step = ctx.solve(group, blocks, nv, ds, primary).cpu().numpy()
    torch.cuda.synchronize()
    b = blocks.cpu().numpy()
    n = sc.n
    if group == O.COLOR:
        g, H = _colour_full(b, nv, 16, n)
        st = step[: 3 * 16 * n].reshape(3, 16, n)
    else:
        D = 3 if group in (O.POS, O.SCALE) else 1
        g = b[: D * n].reshape(D, n)
        H = b[D * n: (D + D * (D + 1) // 2) * n].reshape(-1, n)
        st = step.reshape(-1, n)
    os_ = O.solve(group, sc, primary, ob["g"], ob["H"], ocfg)
    keep = ~amb & (ob["npix"] > 0)
    gs = np.maximum(ob["gabs"], 1e-6 * ob["gabs"].max())
    hs = np.maximum(ob["Habs"], 1e-6 * ob["Habs"].max())
    eg = np.abs(g - ob["g"])[..., keep] / gs[..., keep]
    eh = np.abs(H - ob["H"])[..., keep] / hs[..., keep]
    ok = keep & ((os_["status"] == 0).all(0) if group == O.COLOR else (os_["status"] == 0))
    if group == O.COLOR:
        d = np.linalg.norm(st - os_["step"], axis=1)[:, ok]
        nr = np.maximum(np.linalg.norm(os_["step"], axis=1)[:, ok], 1e-12)
    else:
        d = np.linalg.norm(st - os_["step"], axis=0)[ok]
        nr = np.maximum(np.linalg.norm(os_["step"], axis=0)[ok], 1e-12)
    es = d / nr
    return dict(g_max=float(eg.max()), g_med=float(np.median(eg)), H_max=float(eh.max()),
                H_med=float(np.median(eh)), step_med=float(np.median(es)), step_p99=float(np.quantile(es, 0.99)))


def test_precision_error_report():
    from paper_2501_13975_b300 import gs2
    rows = []
    for group in O.GROUPS:
        plain = _case(gs2, group, 0)
        mixed = _case(gs2, group, 1)
        rows.append((NAMES[group], plain, mixed))
        assert plain["g_max"] <= 1e-4 and plain["H_max"] <= 1e-3
        assert mixed["g_max"] <= 1e-4 and mixed["H_max"] <= 1e-3
        # FP64 accumulation removes the summation error: not worse than FP32 (up to noise)
        assert mixed["g_med"] <= 1.05 * plain["g_med"] + 1e-9
        assert mixed["H_med"] <= 1.05 * plain["H_med"] + 1e-9
    print()
    print(f"{'block':10s} {'mode':6s} {'g max':>9s} {'g med':>9s} {'H max':>9s} {'H med':>9s} "
          f"{'step med':>9s} {'step p99':>9s}")
    for name, p, m in rows:
        for mode, r in (("fp32", p), ("mixed", m)):
            print(f"{name:10s} {mode:6s} {r['g_max']:9.2e} {r['g_med']:9.2e} {r['H_max']:9.2e} {r['H_med']:9.2e} "
                  f"{r['step_med']:9.2e} {r['step_p99']:9.2e}")


def _rot2(rng):
    a = rng.uniform(0, np.pi)
    return np.array([[np.cos(a), -np.sin(a)], [np.sin(a), np.cos(a)]])


def _ill_blocks(group, sc, primary, ocfg, rng):
    """Blocks whose damped reduced system has condition 4e6..4e7 (position:
    H = U D U^T in the plane of the reduction; scaling: H = P D P^T with
    P = Q (Q^T Q)^-1, so that Q^T H Q = D) and whose exact reduced step is a
    small random x_r (g_r = -A x_r), so no trust radius or bound binds."""
    n = sc.n
    B, bst, gap = O.reduced_basis(group, sc, primary, ocfg)
    g = np.zeros((3, n))
    Hp = np.zeros((6, n))
    ok = np.zeros(n, bool)
    iu = np.triu_indices(3)
    mu0 = ocfg["damping_mu0"]
    for k in range(n):
        if bst[k] != 0 or gap[k] < 1e-2:
            continue
        l1 = 10.0 ** rng.uniform(-1, 1)
        R2 = _rot2(rng)
        D = R2 @ np.diag([l1, l1 / 10.0 ** rng.uniform(6.6, 7.6)]) @ R2.T
        Bk = B[k]
        P = Bk @ np.linalg.inv(Bk.T @ Bk)
        H3 = P @ D @ P.T
        A = D + mu0 * np.abs(np.diag(D)).mean() * np.eye(2)
        xr = rng.standard_normal(2) * 1e-3 * float(sc.scale[:, k].max())
        g[:, k] = P @ (-A @ xr)
        Hp[:, k] = H3[iu]
        ok[k] = True
    return g.astype(np.float32), Hp.astype(np.float32), ok


@pytest.mark.parametrize("group", [0, 2, 4])
def test_fp64_resolve_fires_on_ill_conditioned_blocks(group):
    """precision = 1 on blocks constructed with a condition estimate > 1e6 (a
    tiny damping mu0 = 1e-9 keeps them so): the FP64 branch runs for most of
    them (gs2_fp64_resolves) and its steps agree with the FP64 oracle on the
    same FP32 blocks far better than the FP32 path's (which loses about
    cond x 1e-7 relative).  Rotation and opacity blocks are scalars
    (condition 1): the branch never runs for them."""
    from paper_2501_13975_b300 import gs2
    rng = np.random.default_rng(300 + group)
    n = 2000
    sh = 3 if group == O.COLOR else 0
    S = (sh + 1) ** 2
    sc = synth.tiny_scene(n=n, seed=21, sh_degree=sh)
    cams = synth.ring_cameras(4, 64)
    primary = cams[1]
    extra = dict(damping_mu0=1e-9, trust_pos=1e6, trust_color=1e6, scale_trust=1e3)
    ocfg = oracle_cfg(gs2.default_config(**extra))
    if group == O.COLOR:
        nv = 4
        slots = np.zeros((nv, 6 + S, n), np.float32)
        # nearly collinear view bases: the range-space system is ill-conditioned
        # in a way no diagonal scaling removes
        slots[:, 0:3] = rng.standard_normal((nv, 3, n)) * 1e-3
        slots[:, 3:6] = 10.0 ** rng.uniform(-1, 0, (nv, 3, n))
        b0 = rng.standard_normal((S, n))
        for v in range(nv):
            slots[v, 6:] = b0 + (v > 0) * 10.0 ** rng.uniform(-4, -3, n) * rng.standard_normal((S, n))
        g64, H64 = _colour_full(slots.reshape(-1), nv, S, n)
        blocks = slots.reshape(-1)
        ok = np.ones(n, bool)
    else:
        nv = 1
        g, Hp, ok = _ill_blocks(group, sc, primary, ocfg, rng)
        blocks = np.concatenate([g.reshape(-1), Hp.reshape(-1)])
        g64, H64 = g.astype(np.float64), Hp.astype(np.float64)
    ref = O.solve(group, sc, primary, g64, H64, ocfg)
    ds = gs2.DeviceScene.from_host(sc)
    errs, fired = {}, {}
    for prec in (0, 1):
        ctx = gs2.Context(n, 64, 64, sh, 0, dict(precision=prec, **extra))
        ctx.fp64_resolves(reset=True)
        got = ctx.solve(group, torch.tensor(blocks, device="cuda"), nv, ds, primary).cpu().numpy()
        fired[prec] = ctx.fp64_resolves()[group]
        if group == O.COLOR:
            st = got[:3 * S * n].reshape(3, S, n)
            good = (ref["status"] == 0)
            d = np.linalg.norm(st - ref["step"], axis=1)[good]
            nr = np.linalg.norm(ref["step"], axis=1)[good]
        else:
            st = got[:3 * n].reshape(3, n)
            good = ok & (ref["status"] == 0)
            d = np.linalg.norm(st - ref["step"], axis=0)[good]
            nr = np.linalg.norm(ref["step"], axis=0)[good]
        errs[prec] = d / np.maximum(nr, 1e-30)
    total = 3 * n if group == O.COLOR else int(ok.sum())
    med32, med64 = float(np.median(errs[0])), float(np.median(errs[1]))
    print(f"group {group}: FP64 re-solves {fired[1]} of {total}; median relative step error "
          f"fp32 {med32:.2e}, mixed {med64:.2e}")
    assert fired[0] == 0
    assert fired[1] >= 0.5 * total
    assert med64 <= 1e-3 and med64 <= 0.1 * med32


def test_fp64_resolve_never_runs_for_scalar_blocks():
    from paper_2501_13975_b300 import gs2
    rng = np.random.default_rng(9)
    n = 1000
    sc = synth.tiny_scene(n=n, seed=22)
    primary = synth.ring_cameras(4, 64)[0]
    ctx = gs2.Context(n, 64, 64, 0, 0, dict(precision=1, damping_mu0=1e-9))
    ds = gs2.DeviceScene.from_host(sc)
    for group in (O.ROT, O.OPACITY):
        g = rng.standard_normal(n).astype(np.float32)
        h = (10.0 ** rng.uniform(-8, 2, n)).astype(np.float32)
        ctx.solve(group, torch.tensor(np.concatenate([g, h]), device="cuda"), 1, ds, primary)
    assert ctx.fp64_resolves() == [0, 0, 0, 0, 0]


def test_precision_error_scene_crop():
    """Per-block-type error against the FP64 oracle on the scene-scale
    workload (all 1M Gaussians, SH degree 3; a 32x24 crop view of a scene
    camera, L2 loss), for the FP32 path and the mixed path (position,
    rotation, scaling, opacity; the oracle's 16-variable colour jets for 1M
    Gaussians would need ~11 GB).  Printed per group and mode: max and median
    block error relative to the absolute-term scale, median and 99th
    percentile of the step error."""
    from paper_2501_13975_b300 import gs2
    from tests.test_gpu_sweep import _crop
    gt = synth.spread_scene()
    cams = synth.trajectory_cameras()
    train = synth.perturbed(gt, seed=4, sd=0.02)
    cam = _crop(cams[5], 780, 500, 32, 24)
    n = train.n
    rows = []
    ocfg = None
    for group in (O.POS, O.ROT, O.SCALE, O.OPACITY):
        res = {}
        ob = None
        for prec in (0, 1):
            ctx = gs2.Context(n, 32, 24, 3, 8_000_000, dict(lambda_ssim=0.0, precision=prec))
            ocfg = oracle_cfg(ctx.config)
            if ob is None:
                target = O.render(gt, cam, ocfg)["image"].astype(np.float32)
                orc = O.render(train, cam, ocfg)
                L = O.loss(orc["image"], target, ocfg)
                ob = O.accum(group, train, cam, cam, L["e"], L["h"], ocfg)
                amb, _ = ambiguous_gaussians(O, train, cam, ocfg, orc["margin"], thresh=2e-5)
                os_ = O.solve(group, train, cam, ob["g"], ob["H"], ocfg)
            ds = gs2.DeviceScene.from_host(train)
            proj = ctx.project(ds, cam)
            img, rs = ctx.raster_fwd(ds, cam, proj)
            blocks = ctx.blocks_buffer(group, n, 3, 1)
            ctx.accum(group, ds, cam, cam, proj, rs, img, torch.tensor(target, device="cuda"), 0, blocks)
            step = ctx.solve(group, blocks, 1, ds, cam).cpu().numpy()
            torch.cuda.synchronize()
            ctx.check()
            b = blocks.cpu().numpy()
            D = 3 if group in (O.POS, O.SCALE) else 1
            g = b[:D * n].reshape(D, n)
            H = b[D * n:(D + D * (D + 1) // 2) * n].reshape(-1, n)
            keep = ~amb & (ob["npix"] > 0)
            gs = np.maximum(ob["gabs"], 1e-6 * ob["gabs"].max())
            hs = np.maximum(ob["Habs"], 1e-6 * ob["Habs"].max())
            eg = (np.abs(g - ob["g"]) / gs)[..., keep]
            eh = (np.abs(H - ob["H"]) / hs)[..., keep]
            ok = keep & (os_["status"] == 0)
            st = step[:D * n].reshape(D, n)
            es = np.linalg.norm(st - os_["step"], axis=0)[ok] / np.maximum(np.linalg.norm(os_["step"], axis=0)[ok],
                                                                           1e-30)
            res[prec] = (float(eg.max()), float(np.median(eg)), float(eh.max()), float(np.median(eh)),
                         float(np.median(es)), float(np.quantile(es, 0.99)), int(keep.sum()))
            assert eg.max() <= 1e-4 and eh.max() <= 1e-3, (group, prec, eg.max(), eh.max())
        rows.append((NAMES[group], res))
    print()
    print(f"{'block':10s} {'mode':6s} {'g max':>9s} {'g med':>9s} {'H max':>9s} {'H med':>9s} "
          f"{'step med':>9s} {'step p99':>9s} {'Gaussians':>9s}")
    for name, res in rows:
        for prec, mode in ((0, "fp32"), (1, "mixed")):
            r = res[prec]
            print(f"{name:10s} {mode:6s} " + " ".join(f"{v:9.2e}" for v in r[:6]) + f" {r[6]:9d}")

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

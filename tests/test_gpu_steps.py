"""Newton steps, GPU against the oracle (Eq. local_newton; Sec. 4.2 solves;
Sec. 4.3 secondary views), within the block tolerances propagated through
each group's damped reduced system (tests.gpu_common.step_bound_check):

- one view, GPU blocks -> GPU step against oracle blocks -> oracle step, for
  every group;
- a whole sweep in lockstep: every group's blocks from the primary and its
  three downsampled secondaries, started on both sides from the same FP32
  state (the oracle's state after the previous group, rounded to FP32), for
  the paper's configuration, a permuted group order and Gauss-Newton blocks.
  Every Gaussian that contributes and is not excluded by an ambiguous
  decision is checked, including the rotation (its step and the updated
  quaternion); the excluded count is reported and held to 5% of the
  contributors."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2501_13975_b300 import synth  # noqa: E402
from tests.gpu_common import ambiguous_gaussians, oracle_cfg, step_bound_check  # noqa: E402


def _views_oracle(cams, tg, t, knn, f=2):
    out = [(cams[t], tg[t])]
    for v in knn[t]:
        out.append((O.downsample_camera(cams[v], f), O.downsample_image(tg[v], f)))
    return out


def oracle_group(group, state, views, primary, ocfg):
    """The oracle's blocks (summed over views, Eq. tildel), its step and the
    Gaussians touched by an ambiguous compositing decision in any view
    (dilated by the SSIM windows' reach when lambda > 0)."""
    n = state.mean.shape[1]
    acc = None
    amb = np.zeros(n, bool)
    dil = 10 if ocfg["lambda_ssim"] else 0
    for vcam, tgt in views:
        orc = O.render(state, vcam, ocfg)
        L = O.loss(orc["image"], tgt, ocfg)
        acc = O.accum(group, state, vcam, primary, L["e"], L["h"], ocfg, out=acc)
        a, _ = ambiguous_gaussians(O, state, vcam, ocfg, orc["margin"], thresh=2e-5, dilate=dil)
        amb |= a
    os_ = O.solve(group, state, primary, acc["g"], acc["H"], ocfg)
    return acc, os_, amb


@pytest.fixture(scope="module")
def gs2():
    from paper_2501_13975_b300 import gs2 as m
    return m


@pytest.mark.parametrize("group", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("lam", [0.0, 0.2])
def test_newton_steps_end_to_end(gs2, group, lam):
    """One view of 1,000 Gaussians at 128x128 (SH degree 1 for colour)."""
    sh = 1 if group == O.COLOR else 0
    S = (sh + 1) ** 2
    sc = synth.tiny_scene(seed=1, n=1000, sh_degree=sh)
    if sh:
        rng = np.random.default_rng(51)
        sc.sh[:, 1:, :] = rng.normal(0, 0.1, sc.sh[:, 1:, :].shape).astype(np.float32)
    cams = synth.ring_cameras(4, 128)
    ctx = gs2.Context(sc.n, 128, 128, 3, 0, gs2.default_config(lambda_ssim=lam))
    ocfg = oracle_cfg(ctx.config)
    gt = synth.perturbed(sc, seed=2, sd=0.05)
    cam = cams[0]
    target = O.render(gt, cam, ocfg)["image"].astype(np.float32)
    ds = gs2.DeviceScene.from_host(sc)
    proj = ctx.project(ds, cam)
    img, rs = ctx.raster_fwd(ds, cam, proj)
    blocks = ctx.blocks_buffer(group, sc.n, sh, 1)
    ctx.accum(group, ds, cam, cam, proj, rs, img, torch.tensor(target, device="cuda"), 0, blocks)
    step = ctx.solve(group, blocks, 1, ds, cam).cpu().numpy()
    torch.cuda.synchronize()
    ctx.check()
    ob, os_, amb = oracle_group(group, sc, [(cam, target.astype(np.float64))], cam, ocfg)
    r = step_bound_check(O, group, sc, cam, ob, os_, step, ocfg, S, amb)
    print(f"group {group} lambda {lam}: checked {r['checked']}, excluded {r['excluded']} of "
          f"{r['contributors']} contributors, worst err/bound {r['worst']:.3f}")
    assert r["checked"] > 100
    assert r["excluded"] <= 0.05 * r["contributors"], r
    assert not r["fails"], r["fails"][:5]


def _apply_check(gs2, group, ds, step_gpu, state, os_, primary, ocfg, amb_or_excl, sh):
    """The GPU's update of the FP32 state by its own step against the
    oracle's update by the oracle's step: within the step difference
    (rotation: |q - q'| <= |dtheta| / 2) plus FP32 rounding."""
    new_o = O.apply(group, state, primary, os_["step"], ocfg)
    got = ds.to_host()
    n = state.mean.shape[1]
    name = {0: "mean", 1: "quat", 2: "scale", 3: "opacity", 4: "sh"}[group]
    a = getattr(got, name).astype(np.float64).reshape(-1, n)
    b = getattr(new_o, name).reshape(-1, n)
    d = np.linalg.norm(a - b, axis=0)
    if group == O.ROT:
        dstep = np.abs(step_gpu[:n] - os_["step"][0]) / 2
    elif group == O.COLOR:
        S = (sh + 1) ** 2
        dstep = np.linalg.norm(step_gpu[:3 * S * n].reshape(3 * S, n) - os_["step"].reshape(3 * S, n), axis=0)
    else:
        D = 3 if group in (O.POS, O.SCALE) else 1
        dstep = np.linalg.norm(step_gpu[:D * n].reshape(D, n) - os_["step"].reshape(D, n), axis=0)
    tol = dstep + 4e-6 * np.maximum(1.0, np.linalg.norm(b, axis=0))
    ok = d <= tol
    assert np.all(ok[~amb_or_excl]), (group, np.nonzero(~ok & ~amb_or_excl)[0][:5])
    return new_o


@pytest.mark.parametrize("variant", [{}, {"group_order": (4, 2, 0, 3, 1)}, {"gauss_newton": 1}],
                         ids=["paper", "order-42031", "gauss-newton"])
def test_sweep_steps_lockstep(gs2, variant):
    n, size = 400, 64
    sc = synth.tiny_scene(n=n, seed=1)
    gt = synth.perturbed(sc, seed=2, sd=0.05)
    cams = synth.ring_cameras(4, size)
    ctx = gs2.Context(n, size, size, 0, 0, gs2.default_config(**variant))
    ocfg = oracle_cfg(ctx.config)
    tg32 = np.stack([O.render(gt, c, ocfg)["image"] for c in cams]).astype(np.float32)
    tg = tg32.astype(np.float64)
    targets = [torch.tensor(x, device="cuda") for x in tg32]
    centres = np.stack([c.center() for c in cams])
    knn, _ = O.knn(centres, O.bounding_sphere(sc), 3)
    t = 2
    primary = cams[t]
    views_o = _views_oracle(cams, tg, t, knn)
    state = sc.copy()
    total_c = total_x = 0
    for group in ctx.config["group_order"]:
        ob, os_, amb = oracle_group(group, state, views_o, primary, ocfg)
        ds = gs2.DeviceScene.from_host(state)
        blocks = ctx.blocks_buffer(group, n, 0, 4)
        for slot, v in enumerate([t] + list(knn[t])):
            if slot == 0:
                cam, tgt = cams[v], targets[v]
            else:
                cam, tgt = gs2.camera_downsample(cams[v], 2), ctx.downsample(targets[v], 2)
            proj = ctx.project(ds, cam)
            img, rs = ctx.raster_fwd(ds, cam, proj)
            ctx.accum(group, ds, cam, primary, proj, rs, img, tgt, slot, blocks)
        step = ctx.solve(group, blocks, 4, ds, primary)
        ctx.apply(group, step, ds, primary)
        torch.cuda.synchronize()
        ctx.check()
        step = step.cpu().numpy()
        r = step_bound_check(O, group, state, primary, ob, os_, step, ocfg, 1, amb)
        print(f"{variant} group {group}: checked {r['checked']}, excluded {r['excluded']} of "
              f"{r['contributors']}, worst err/bound {r['worst']:.3f}")
        assert r["checked"] > 50, r
        assert not r["fails"], (group, r["fails"][:5])
        total_c += r["contributors"]
        total_x += r["excluded"]
        new_o = _apply_check(gs2, group, ds, step, state, os_, primary, ocfg, ~r["mask"], 0)
        state = O.to_fp32_scene(new_o, state)
    assert total_x <= 0.05 * total_c, (total_x, total_c)

"""Deterministic mode (config.deterministic = 1): no float atomics in the
block sums (Eq. local_hessian_gradient).  Every tile-list entry gets its own
partial (the tile's four warp sums added in warp order), each Gaussian's
entries are summed in emission order (compensated FP32; FP64 with mixed
precision), and a sweep's views run one after another.  So two runs give the
same bytes, for every group's blocks and for the parameters after whole
sweeps, and the blocks still match the oracle within the parity tolerances."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2501_13975_b300 import synth  # noqa: E402
from tests.gpu_common import oracle_cfg  # noqa: E402
from tests.test_gpu_parity import _blocks_case, _check_blocks  # noqa: E402


@pytest.fixture(scope="module")
def gs2():
    from paper_2501_13975_b300 import gs2 as m
    return m


@pytest.mark.parametrize("group", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("precision", [0, 1])
def test_deterministic_blocks_parity_and_identical_bytes(gs2, group, precision):
    r = _blocks_case(gs2, group, sh=(1 if group == O.COLOR else 0), lam=0.2,
                     extra=dict(deterministic=1, precision=precision))
    _check_blocks(r)
    ctx, ds, vcam, primary = r["ctx"], r["ds"], r["vcam"], r["primary"]
    tgt = torch.tensor(r["target"], device="cuda")
    sh = 1 if group == O.COLOR else 0
    again = []
    for _ in range(3):
        proj = ctx.project(ds, vcam)
        img, rs = ctx.raster_fwd(ds, vcam, proj)
        b = ctx.blocks_buffer(group, r["sc"].n, sh, 1)
        ctx.accum(group, ds, vcam, primary, proj, rs, img, tgt, 0, b)
        torch.cuda.synchronize()
        again.append(b.cpu().numpy().view(np.uint32))
    ref = r["blocks"].cpu().numpy().view(np.uint32)
    for a in again:
        assert np.array_equal(a, ref)


def _sweep_setup(gs2, cfg, n=800, size=96):
    sc = synth.tiny_scene(n=n, seed=6, sh_degree=1)
    sc.sh[:, 1:, :] = np.random.default_rng(8).normal(0, 0.1, sc.sh[:, 1:, :].shape).astype(np.float32)
    gt = synth.perturbed(sc, seed=7, sd=0.05)
    cams = synth.ring_cameras(6, size)
    ctx = gs2.Context(n, size, size, 1, 0, cfg)
    ocfg = oracle_cfg(ctx.config)
    targets = [torch.tensor(O.render(gt, c, ocfg)["image"].astype(np.float32), device="cuda") for c in cams]
    centres = np.stack([c.center() for c in cams]).astype(np.float32)
    sphere = ctx.bounding_sphere(gs2.DeviceScene.from_host(sc)).cpu().numpy()
    knn = gs2.camera_knn(centres, sphere, 3)
    return sc, cams, ctx, targets, knn


def _state_bytes(ds):
    return [getattr(ds, k).cpu().numpy().view(np.uint32).copy() for k in ("mean", "quat", "scale", "opacity", "sh")]


@pytest.mark.parametrize("precision", [0, 1])
def test_deterministic_sweeps_identical_bytes(gs2, precision):
    """Three sweeps (primaries 0, 2, 4) from the same start, twice, on two
    contexts: the parameters after every sweep are the same bytes.  The
    atomic path is run beside it for comparison (its bytes are not required to
    match)."""
    sc, cams, ctx, targets, knn = _sweep_setup(gs2, dict(deterministic=1, precision=precision))
    _, _, ctx2, _, _ = _sweep_setup(gs2, dict(deterministic=1, precision=precision))
    runs = []
    for c in (ctx, ctx2, ctx):
        ds = gs2.DeviceScene.from_host(sc)
        states = []
        for t in (0, 2, 4):
            c.sweep(ds, cams, targets, knn, t)
            torch.cuda.synchronize()
            c.check()
            states.append(_state_bytes(ds))
        runs.append(states)
    for other in runs[1:]:
        for sa, sb in zip(runs[0], other):
            for a, b in zip(sa, sb):
                assert np.array_equal(a, b)
    # the deterministic sweep moves the scene like the atomic one (same method)
    _, _, cat, _, _ = _sweep_setup(gs2, dict(precision=precision))
    ds = gs2.DeviceScene.from_host(sc)
    for t in (0, 2, 4):
        cat.sweep(ds, cams, targets, knn, t)
    torch.cuda.synchronize()
    got = [x.view(np.float32) for x in runs[0][-1]]
    want = [getattr(ds, k).cpu().numpy() for k in ("mean", "quat", "scale", "opacity", "sh")]
    differ = sum(int((a.view(np.uint32) != b.view(np.uint32)).sum()) for a, b in zip(got, want))
    for a, b in zip(got, want):
        assert np.abs(a.astype(np.float64) - b).max() <= 1e-3 * max(1.0, np.abs(b).max())
    print(f"precision {precision}: parameters differing in some bit from the atomic path: {differ}")


def test_deterministic_mode_is_the_path_taken(gs2):
    """The deterministic accumulation really replaces the atomics: its block
    sums of a view equal the atomic path's to rounding, and with the option
    off the context holds no partial buffers (gs2_set_config allocates them)."""
    r = _blocks_case(gs2, O.POS, lam=0.0)
    ctx = r["ctx"]
    ctx.set_config(deterministic=1)
    proj = ctx.project(r["ds"], r["vcam"])
    img, rs = ctx.raster_fwd(r["ds"], r["vcam"], proj)
    b = ctx.blocks_buffer(O.POS, r["sc"].n, 0, 1)
    ctx.accum(O.POS, r["ds"], r["vcam"], r["primary"], proj, rs, img, torch.tensor(r["target"], device="cuda"), 0, b)
    torch.cuda.synchronize()
    a, d = r["blocks"].cpu().numpy(), b.cpu().numpy()
    assert np.abs(a - d).max() <= 1e-5 * np.abs(a).max()

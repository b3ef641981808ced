"""Failure detection without a GPU fault: non-finite parameters or target
pixels and an overflowing pair list are reported through the device status
word (gs2_check) while the sweep completes and the other Gaussians stay
finite."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2501_13975_b300 import synth  # noqa: E402


def _setup(gs2, n=600, size=64):
    sc = synth.tiny_scene(n=n, seed=90)
    gt = synth.perturbed(sc, seed=91, sd=0.05)
    cams = synth.ring_cameras(4, size)
    ctx = gs2.Context(n, size, size, 0)
    dg = gs2.DeviceScene.from_host(gt)
    targets = []
    for c in cams:
        proj = ctx.project(dg, c)
        img, _ = ctx.raster_fwd(dg, c, proj)
        targets.append(img.clone())
    knn = np.array([[1, 2, 3], [0, 2, 3], [0, 1, 3], [0, 1, 2]], np.int32)
    torch.cuda.synchronize()
    ctx.check()
    return sc, cams, ctx, targets, knn


def _finite_except(ds, k):
    for name in ("mean", "quat", "scale", "opacity", "sh"):
        x = getattr(ds, name).reshape(-1, ds.n)
        keep = torch.ones(ds.n, dtype=torch.bool, device=x.device)
        if k is not None:
            keep[k] = False
        assert bool(torch.isfinite(x[:, keep]).all()), name


def test_clean_sweep_reports_ok():
    from paper_2501_13975_b300 import gs2
    sc, cams, ctx, targets, knn = _setup(gs2)
    ds = gs2.DeviceScene.from_host(sc)
    ctx.sweep(ds, cams, targets, knn, 0)
    ctx.check()
    _finite_except(ds, None)


def test_nonfinite_parameter_is_reported_and_contained():
    from paper_2501_13975_b300 import gs2
    sc, cams, ctx, targets, knn = _setup(gs2)
    bad = sc.copy()
    bad.mean[1, 17] = np.nan
    bad.scale[0, 40] = np.inf
    ds = gs2.DeviceScene.from_host(bad)
    ctx.sweep(ds, cams, targets, knn, 1)
    with pytest.raises(gs2.GS2Error, match="NONFINITE"):
        ctx.check()
    ctx.check()   # the status word was cleared by the first check
    mask = torch.ones(ds.n, dtype=torch.bool, device="cuda")
    mask[17] = False
    mask[40] = False
    for name in ("mean", "quat", "scale", "opacity", "sh"):
        x = getattr(ds, name).reshape(-1, ds.n)
        assert bool(torch.isfinite(x[:, mask]).all()), name


def test_nonfinite_target_pixel_is_reported():
    from paper_2501_13975_b300 import gs2
    sc, cams, ctx, targets, knn = _setup(gs2)
    targets[2][1, 10, 12] = float("nan")
    ds = gs2.DeviceScene.from_host(sc)
    ctx.sweep(ds, cams, targets, knn, 2)
    with pytest.raises(gs2.GS2Error, match="NONFINITE"):
        ctx.check()
    _finite_except(ds, None)


def test_pair_capacity_overflow_is_reported():
    from paper_2501_13975_b300 import gs2
    sc = synth.tiny_scene(n=2000, seed=92)
    cam = synth.ring_cameras(4, 128)[0]
    ctx = gs2.Context(sc.n, 128, 128, 0, max_pairs=64)
    ds = gs2.DeviceScene.from_host(sc)
    proj = ctx.project(ds, cam)
    img, _ = ctx.raster_fwd(ds, cam, proj)
    with pytest.raises(gs2.GS2Error, match="CAPACITY"):
        ctx.check()
    assert bool(torch.isfinite(img).all())


@pytest.mark.parametrize("chunk,limit", [(1, 64), (40, 4096)])
def test_bounded_wait_gives_up_and_is_reported(chunk, limit):
    """The scan's look-back wait, run over states that nothing publishes,
    gives up after its poll limit: gs2_check reports GS2_ERR_TIMEOUT (and
    clears it), and the context then sweeps and checks clean."""
    import time
    from paper_2501_13975_b300 import gs2
    sc, cams, ctx, targets, knn = _setup(gs2)
    t0 = time.perf_counter()
    ctx.debug_lookback_timeout(chunk, limit)
    torch.cuda.synchronize()
    assert time.perf_counter() - t0 < 5.0
    with pytest.raises(gs2.GS2Error, match="TIMEOUT"):
        ctx.check()
    ctx.check()   # read and cleared
    ds = gs2.DeviceScene.from_host(sc)
    ctx.sweep(ds, cams, targets, knn, 0)
    torch.cuda.synchronize()
    ctx.check()
    _finite_except(ds, None)
    for bad in ((0, 10), (256, 10), (3, 0), (3, (1 << 20) + 1)):
        with pytest.raises(gs2.GS2Error):
            ctx.debug_lookback_timeout(*bad)

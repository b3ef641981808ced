"""Host-resident targets (gs2.HostTargets): each sweep's views are uploaded on
a copy stream into one of two buffer sets while the previous sweep runs.
The buffers a sweep reads hold exactly its views' host images when the sweep
reads them, and a sweep on uploaded targets equals one on device-resident
targets."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2501_13975_b300 import synth  # noqa: E402


@pytest.fixture(scope="module")
def gs2():
    from paper_2501_13975_b300 import gs2 as m
    return m


def _setup(gs2, n=1500, size=64, ncam=6):
    gt = synth.tiny_scene(seed=91, n=n, sh_degree=3)
    cams = synth.ring_cameras(ncam, size)
    ctx = gs2.Context(n, size, size, 3, 64 * n)
    dgt = gs2.DeviceScene.from_host(gt)
    targets = []
    for c in cams:
        proj = ctx.project(dgt, c)
        img, _ = ctx.raster_fwd(dgt, c, proj)
        targets.append(img.clone())
    train = synth.perturbed(gt, seed=92, sd=0.02)
    sphere = ctx.bounding_sphere(gs2.DeviceScene.from_host(train)).cpu().numpy()
    knn = gs2.camera_knn(np.stack([c.center() for c in cams]).astype(np.float32), sphere, 3)
    torch.cuda.synchronize()
    return ctx, cams, targets, train, knn


def test_buffers_hold_the_views_when_read(gs2):
    """Long work on the compute stream between acquiring a sweep's targets and
    reading them gives a wrongly ordered upload time to overwrite them; the
    checksums taken on the compute stream must still equal the host images'."""
    ctx, cams, targets, train, knn = _setup(gs2)
    host = [t.cpu() for t in targets]
    ht = gs2.HostTargets(host, knn)
    ref = [float(h.double().sum()) for h in host]
    a = torch.randn(2048, 2048, device="cuda")
    order = [0, 3, 1, 4, 2, 5, 0, 1]
    sums = []
    for i, t in enumerate(order):
        tg = ht.targets(t)
        assert [v for v in range(len(host)) if tg[v] is not None] == sorted(ht.views(t))
        for _ in range(20):   # keep the compute stream busy before the read
            a = torch.tanh(a @ a * 1e-3)
        sums.append({v: tg[v].double().sum() for v in ht.views(t)})
        ht.release(t)
        if i + 1 < len(order):
            ht.prefetch(order[i + 1])
    torch.cuda.synchronize()
    for i, t in enumerate(order):
        for v, s in sums[i].items():
            assert float(s) == ref[v], (i, t, v)


def test_sweep_on_uploaded_targets_equals_device_targets(gs2):
    ctx, cams, targets, train, knn = _setup(gs2)
    ht = gs2.HostTargets([t.cpu() for t in targets], knn)
    out = []
    for use_host in (False, True):
        scene = gs2.DeviceScene.from_host(train)
        losses = torch.zeros(10, dtype=torch.float64, device="cuda")
        tg = ht.targets(2) if use_host else targets
        ctx.sweep(scene, cams, tg, knn, 2, losses)
        if use_host:
            ht.release(2)
        torch.cuda.synchronize()
        ctx.check()
        out.append((losses.cpu().numpy(), scene.mean.cpu().numpy()))
    (l0, m0), (l1, m1) = out
    # the primary view's first-group loss is formed before any step: equal
    # up to the order of its double-precision block sums
    np.testing.assert_allclose(l1[:2], l0[:2], rtol=1e-12)
    # the position step, up to the order of atomic additions
    assert np.abs(m1 - m0).max() <= 1e-4 * max(1.0, np.abs(m0).max())


def test_bytes_for_counts_the_views(gs2):
    ctx, cams, targets, train, knn = _setup(gs2)
    ht = gs2.HostTargets([t.cpu() for t in targets], knn)
    per = targets[0].numel() * 4
    assert ht.bytes_for(0) == per * len(ht.views(0))
    assert ht.views(0)[0] == 0 and len(ht.views(0)) == 1 + knn.shape[1]

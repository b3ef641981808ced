"""Split accumulation: every tile's back-to-front walk cut into work items of
`accum_split` list entries, each started from the compositing's checkpoint
(T and the colour in front) at its back end, taken by a persistent grid.

- Blocks against the FP64 oracle at the block tolerances, on scenes whose
  walks span several items (faint Gaussians: no pixel stops early).
- Blocks against the whole-walk accumulation on the same inputs, where many
  pixels stop at t_min (the same FP32 stop decisions on both sides), for
  every group, both pixel-per-thread shapes, primary and downsampled views
  and both accumulation precisions.
- A native sweep with split walks against one with whole walks, and a
  batched sweep under a CUDA graph against the eager per-scene sweep.
- The tuning field's validation and the autotuner's candidates."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2501_13975_b300 import synth  # noqa: E402
from tests.gpu_common import rel_err  # noqa: E402
from tests.test_gpu_parity import _blocks_case, _check_blocks  # noqa: E402
from tests.test_gpu_batch import _close  # noqa: E402


@pytest.fixture(scope="module")
def gs2():
    from paper_2501_13975_b300 import gs2 as m
    return m


def _walk_max(r):
    """Largest list position after a last contributor (the longest walk) of the case's view."""
    v = r["vcam"]
    _, last = r["ctx"].raster_state(r["rs"], int(v.width), int(v.height))
    return int(last.max())


DENSE = dict(n=6000, size=64)


@pytest.mark.parametrize("group,px", [(0, 2), (0, 4), (1, 2), (2, 2), (3, 2), (4, 2), (4, 4)])
def test_split_blocks_parity(gs2, group, px):
    """Faint Gaussians (opacity x 0.1): walks up to about 1600 entries, cut
    into items of 256; the blocks equal the oracle's."""
    r = _blocks_case(gs2, group, sh=(1 if group == O.COLOR else 0), lam=0.2, opacity_scale=0.1,
                     tuning=dict(accum_split=256, accum_px=px), **DENSE)
    assert r["ctx"].tuning()["accum_split"] == 256
    assert _walk_max(r) > 3 * 256   # several items per tile, so checkpoints are used
    _check_blocks(r)


@pytest.mark.parametrize("group", [0, 4])
def test_split_blocks_parity_secondary(gs2, group):
    """Downsampled secondary view (32x32: two tiles a side, walks up to about
    2000 entries) with SH degree 3.  Against the oracle at 3e-4 of the
    absolute-term scale for g: the largest deviation (2.1e-4, position row 0)
    is in a Gaussian that covers a single pixel, the same with whole walks
    and with FP64 accumulation, so it comes from that pixel's FP32 term, not
    from the walk.  The split blocks equal the whole-walk blocks to the same
    tolerance: the split compositing sums a pixel's colour per segment, and
    the loss derivative magnifies that rounding where render and target
    nearly agree."""
    kw = dict(sh=3, lam=0.2, secondary=True, opacity_scale=0.1, **DENSE)
    whole = _blocks_case(gs2, group, tuning=dict(accum_split=0), **kw)
    part = _blocks_case(gs2, group, tuning=dict(accum_split=256), **kw)
    assert _walk_max(part) > 3 * 256
    ob = whole["ob"]
    gs = np.maximum(ob["gabs"], 1e-6 * ob["gabs"].max())
    hs = np.maximum(ob["Habs"], 1e-6 * ob["Habs"].max())
    assert rel_err(part["g"], whole["g"], gs) <= 3e-4 and rel_err(part["H"], whole["H"], hs) <= 1e-3
    _check_blocks(part, gtol=3e-4)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("case", [dict(group=0, px=4), dict(group=0, px=2), dict(group=1, px=2),
                                  dict(group=2, px=2), dict(group=3, px=2), dict(group=4, px=4),
                                  dict(group=0, px=4, secondary=True), dict(group=4, px=2, secondary=True)],
                         ids=["pos4", "pos2", "rot", "scale", "opacity", "colour4", "pos4-secondary",
                              "colour2-secondary"])
@pytest.mark.parametrize("split", [256, 1024])
def test_split_equals_whole_walks(gs2, case, precision, split):
    """Opacity x 0.6: part of the pixels stop at t_min inside the walk.  The
    split and the whole-walk accumulation take the same stop decisions (one
    compositing), so their blocks agree to rounding: the checkpointed T
    against T recovered by division, the image summed per segment against the
    image summed along the walk, the checkpointed colour against the colour
    summed from behind (the checkpoint keeps the colour of the entries behind
    it, not C_final - C, whose cancellation at a deep T near t_min lost three
    digits), and the order of the atomic additions.  Scaled by the
    oracle's sums of absolute per-pixel terms, as the oracle parity is."""
    group, px, secondary = case["group"], case["px"], case.get("secondary", False)
    sh = 1 if group == O.COLOR else 0
    kw = dict(sh=sh, lam=0.2, secondary=secondary, opacity_scale=0.6, extra=dict(precision=precision), **DENSE)
    whole = _blocks_case(gs2, group, tuning=dict(accum_split=0, accum_px=px), **kw)
    part = _blocks_case(gs2, group, tuning=dict(accum_split=split, accum_px=px), **kw)
    assert _walk_max(part) > split   # more than one item in some tile
    tf, _ = part["ctx"].raster_state(part["rs"], int(part["vcam"].width), int(part["vcam"].height))
    assert float((tf < 2e-4).float().mean()) > 0.02   # pixels that stopped inside their walk
    ob = whole["ob"]
    gs = np.maximum(ob["gabs"], 1e-6 * ob["gabs"].max())
    hs = np.maximum(ob["Habs"], 1e-6 * ob["Habs"].max())
    eg = rel_err(part["g"], whole["g"], gs)
    eh = rel_err(part["H"], whole["H"], hs)
    print(f"split {split} vs whole: g {eg:.2e} H {eh:.2e}")
    assert eg <= 1e-4 and eh <= 1e-3, (eg, eh)
    # a Gaussian with no contribution has none in either
    assert np.array_equal(part["g"] == 0, whole["g"] == 0)


def _dense_sweep_setup(gs2, n=6000, size=64, f=0.5):
    gt = synth.tiny_scene(seed=31, n=n, sh_degree=1)
    gt.opacity = (gt.opacity * f).astype(np.float32)
    train = synth.perturbed(gt, seed=32, sd=0.02)
    cams = synth.ring_cameras(6, size)
    tmp = gs2.Context(n, size, size, 1, 0)
    g = gs2.DeviceScene.from_host(gt)
    targets = []
    for c in cams:
        proj = tmp.project(g, c)
        img, _ = tmp.raster_fwd(g, c, proj)
        targets.append(img.clone())
    sphere = tmp.bounding_sphere(gs2.DeviceScene.from_host(train)).cpu().numpy()
    knn = gs2.camera_knn(np.stack([c.center() for c in cams]).astype(np.float32), sphere, 3)
    torch.cuda.synchronize()
    return train, cams, targets, knn


@pytest.mark.parametrize("lanes", [0, 1])
def test_split_sweep_equals_whole_walk_sweep(gs2, lanes):
    """One native sweep (4 views x 5 groups, views concurrent or in series)
    with split walks against the same sweep with whole walks, from the same
    snapshot: equal up to the rounding of atomic order."""
    train, cams, targets, knn = _dense_sweep_setup(gs2)
    out = []
    for split in (0, 256):
        ctx = gs2.Context(train.n, 64, 64, 1, 0)
        ctx.set_tuning(view_lanes=lanes, accum_split=split)
        s = gs2.DeviceScene.from_host(train)
        ctx.sweep(s, cams, targets, knn, 2)
        torch.cuda.synchronize()
        ctx.check()
        out.append(s)
    _close(out[1], out[0], gs2.DeviceScene.from_host(train))


@pytest.mark.parametrize("variant", ["jacobi", "gauss-newton", "networks"])
def test_split_sweep_variants_equal_whole_walks(gs2, variant):
    """The split walks under the other sweep forms: the single-render sweep
    (every group accumulated from one compositing per view), Gauss-Newton
    blocks, and the learned damping and step-scale networks (the view lanes
    then accumulate into their own blocks) equal the same sweep with whole
    walks, from the same snapshot, up to the rounding of atomic order."""
    train, cams, targets, knn = _dense_sweep_setup(gs2)
    cfg = dict(group_jacobi=1) if variant == "jacobi" else dict(gauss_newton=1) if variant == "gauss-newton" else {}
    out = []
    for split in (0, 256):
        ctx = gs2.Context(train.n, 64, 64, 1, 0, cfg)
        ctx.set_tuning(accum_split=split)
        if variant == "networks":
            _, dbits = synth.mlp_init(67, out_scale=2.0)
            _, sbits = synth.mlp_init(68, out_scale=1.0)
            ctx.set_damping_model(torch.tensor(dbits.astype(np.int16), device="cuda"))
            ctx.set_step_model(torch.tensor(sbits.astype(np.int16), device="cuda"))
        s = gs2.DeviceScene.from_host(train)
        ctx.sweep(s, cams, targets, knn, 1)
        torch.cuda.synchronize()
        ctx.check()
        out.append(s)
    _close(out[1], out[0], gs2.DeviceScene.from_host(train))


@pytest.mark.parametrize("use_graph", [0, 1])
def test_split_batched_graph_equals_eager(gs2, use_graph):
    """A one-scene batch with split walks (eager fork/join, or captured as a
    CUDA graph: the item builder, the persistent grid and its fetch counter
    replay inside the graph) against gs2_sweep of the same context settings."""
    train, cams, targets, knn = _dense_sweep_setup(gs2)
    size = dict(max_gaussians=train.n, max_width=64, max_height=64, max_sh_degree=1, max_pairs=0)
    batch = gs2.Batch([size])
    tun = batch.tuning(0)
    batch.set_tuning(0, tun["sort_blocks"], tun["sort_rows"], tun["view_lanes"], tun["accum_px"], 256)
    assert batch.tuning(0)["accum_split"] == 256
    ref_ctx = gs2.Context(train.n, 64, 64, 1, 0)
    ref_ctx.set_tuning(accum_split=256)
    s = gs2.DeviceScene.from_host(train)
    prep = batch.prepare([s], [cams], [targets], [knn])
    losses = torch.zeros((1, 10), dtype=torch.float64, device="cuda")
    for t in (0, 3, 0):
        snap = s.clone()
        ref = s.clone()
        batch.sweep(prep, [t], losses=losses, use_graph=use_graph)
        ref_ctx.sweep(ref, cams, targets, knn, t)
        torch.cuda.synchronize()
        batch.check()
        ref_ctx.check()
        _close(s, ref, snap)
    assert bool((losses[:, 0] > 0).all())


def test_kept_graphs_follow_split_buffer_changes(gs2):
    """Kept graphs (use_graph = 2) across tuning changes that reallocate the
    split walks' checkpoints (1024 -> 256 -> 1024 entries per item): every
    batched sweep equals gs2_sweep with the same settings from the same
    snapshot (a graph captured with the freed buffers is not replayed: the
    graph key holds the buffers' addresses)."""
    train, cams, targets, knn = _dense_sweep_setup(gs2)
    size = dict(max_gaussians=train.n, max_width=64, max_height=64, max_sh_degree=1, max_pairs=0)
    batch = gs2.Batch([size])
    tun = batch.tuning(0)
    s = gs2.DeviceScene.from_host(train)
    prep = batch.prepare([s], [cams], [targets], [knn])
    for split in (1024, 256, 1024):
        batch.set_tuning(0, tun["sort_blocks"], tun["sort_rows"], tun["view_lanes"], tun["accum_px"], split)
        ref_ctx = gs2.Context(train.n, 64, 64, 1, 0)
        ref_ctx.set_tuning(accum_split=split)
        for t in (0, 3):
            snap = s.clone()
            ref = s.clone()
            batch.sweep(prep, [t], use_graph=2)
            ref_ctx.sweep(ref, cams, targets, knn, t)
            torch.cuda.synchronize()
            batch.check()
            ref_ctx.check()
            _close(s, ref, snap)


def test_split_tuning_validation(gs2):
    ctx = gs2.Context(100, 32, 32, 0)
    assert ctx.tuning()["accum_split"] == 0
    for bad in (-256, 100, 255, 3 << 20):
        with pytest.raises(gs2.GS2Error):
            ctx.set_tuning(accum_split=bad)
    assert ctx.tuning()["accum_split"] == 0
    for ok in (256, 1024, 0, 512):
        ctx.set_tuning(accum_split=ok)
        assert ctx.tuning()["accum_split"] == ok


def test_autotune_tries_split_walks(gs2):
    """The autotuner times the split candidates and keeps one of them or none;
    the caller's scene is not moved."""
    train, cams, targets, knn = _dense_sweep_setup(gs2)
    ctx = gs2.Context(train.n, 64, 64, 1, 0)
    s = gs2.DeviceScene.from_host(train)
    before = s.clone()
    best = ctx.autotune(s, cams, targets, knn, 0, reps=1)
    assert best["accum_split"] in (0, 256, 1024)
    assert ctx.tuning() == {k: v for k, v in best.items() if k != "ms"}
    for name in ("mean", "quat", "scale", "opacity", "sh"):
        assert torch.equal(getattr(s, name), getattr(before, name))

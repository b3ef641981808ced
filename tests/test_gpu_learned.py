"""Learned step scale on the GPU against the FP64 oracle (oracle/learned.py):
network forward, loss gradient and Adam; step records and labels; the logged
sweep; inference inside gs2_solve_step with its fallback; and what a network
trained on logged records gains over the plain step."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import learned as Lr  # noqa: E402
from oracle import oracle as O  # noqa: E402
from paper_2501_13975_b300 import synth  # noqa: E402
from tests.gpu_common import ambiguous_gaussians, oracle_cfg  # noqa: E402


def _random_records(seed, chunks=3, chunk_n=1000):
    rng = np.random.default_rng(seed)
    rec = np.zeros((chunks, Lr.REC_ROWS, chunk_n), np.float32)
    rec[:, :Lr.NF] = rng.normal(0.0, 1.0, (chunks, Lr.NF, chunk_n))
    rec[:, Lr.NF] = -np.abs(rng.normal(1.0, 0.5, (chunks, chunk_n)))
    rec[:, Lr.NF, ::23] *= -0.3                      # some rejected steps (phi0 > 0)
    rec[:, Lr.NF + 2] = rec[:, Lr.NF] + rng.uniform(-0.5, 2.0, (chunks, chunk_n))
    rec[:, Lr.NF + 1] = rng.uniform(0.0, 2.0, (chunks, chunk_n))
    rec[:, Lr.NF + 1, ::17] = -1.0          # unusable labels
    rec[0, 3, 5::29] = np.nan               # unusable features
    return rec


def _oracle_xy(rec, idx):
    r = np.moveaxis(rec.astype(np.float64), 1, 2).reshape(-1, Lr.REC_ROWS)[idx]
    return r[:, :Lr.NF], r[:, Lr.NF + 1]


def test_mlp_forward_and_gradient_match_oracle():
    from paper_2501_13975_b300 import gs2
    master, bits = synth.mlp_init(30, out_scale=1.0)
    p = Lr.bf16_to_f64(bits)
    rec = _random_records(31)
    chunk_n = rec.shape[2]
    perm = np.random.default_rng(32).permutation(rec.shape[0] * chunk_n)[:2500]
    w = torch.tensor(bits.astype(np.int16), device="cuda")
    recd = torch.tensor(rec, device="cuda").reshape(-1)
    idx = torch.tensor(perm, dtype=torch.int64, device="cuda")
    alpha = gs2.mlp_forward(w, recd, chunk_n, len(perm), idx=idx).cpu().numpy()
    partial = torch.empty((gs2.MLP_GRID, gs2.MLP_NPARAM), dtype=torch.float32, device="cuda")
    stats = torch.empty((gs2.MLP_GRID, 2), dtype=torch.float64, device="cuda")
    gs2.mlp_grad(w, recd, chunk_n, len(perm), partial, stats, idx=idx)
    g = partial.double().sum(0).cpu().numpy()
    st = stats.sum(0).cpu().numpy()
    X, Y = _oracle_xy(rec, perm)
    ok = Lr.usable(X, Y)
    a_ref, _ = Lr.mlp_forward(p, np.where(ok[:, None], X, 0.0))
    assert np.abs(alpha[ok] - a_ref[ok]).max() <= 2e-6
    loss, cnt, g_ref = Lr.mlp_loss_grad(p, X, Y)
    assert int(st[1]) == cnt
    assert st[0] == pytest.approx(loss, rel=1e-5)
    err = np.abs(g - g_ref).max() / np.abs(g_ref).max()
    assert err <= 1e-4, err


def test_line_objective_and_chunk_scale_match_oracle():
    """The line-model loss (per-chunk scales from the device kernel) and its
    gradient equal the oracle's."""
    from paper_2501_13975_b300 import gs2
    _, bits = synth.mlp_init(35, out_scale=1.0)
    p = Lr.bf16_to_f64(bits)
    rec = _random_records(36)
    chunk_n = rec.shape[2]
    recd = torch.tensor(rec, device="cuda").reshape(-1)
    sc = gs2.records_chunk_scale(recd, chunk_n, rec.shape[0]).cpu().numpy()
    sc_ref = Lr.chunk_scale(rec)
    assert np.allclose(sc, sc_ref, rtol=1e-6)
    perm = np.random.default_rng(37).permutation(rec.shape[0] * chunk_n)[:2000]
    w = torch.tensor(bits.astype(np.int16), device="cuda")
    idx = torch.tensor(perm, dtype=torch.int64, device="cuda")
    partial = torch.empty((gs2.MLP_GRID, gs2.MLP_NPARAM), dtype=torch.float32, device="cuda")
    stats = torch.empty((gs2.MLP_GRID, 2), dtype=torch.float64, device="cuda")
    gs2.mlp_grad(w, recd, chunk_n, len(perm), partial, stats, idx=idx,
                 chunk_scale=torch.tensor(sc, device="cuda"))
    g = partial.double().sum(0).cpu().numpy()
    st = stats.sum(0).cpu().numpy()
    X, Y = _oracle_xy(rec, perm)
    flat = np.moveaxis(rec.astype(np.float64), 1, 2).reshape(-1, Lr.REC_ROWS)[perm]
    chunk = perm // chunk_n
    line = Lr.line_terms(flat[:, Lr.NF], flat[:, Lr.NF + 2], sc_ref[chunk])
    loss, cnt, g_ref = Lr.mlp_loss_grad(p, X, Y, line)
    assert int(st[1]) == cnt
    assert st[0] == pytest.approx(loss, rel=1e-4, abs=1e-9)
    assert np.abs(g - g_ref).max() / np.abs(g_ref).max() <= 1e-4


def test_adam_step_matches_oracle():
    """One Adam step from zero moments on the batch mean gradient; the BF16
    copy is the round-to-nearest-even of the FP32 master."""
    from paper_2501_13975_b300 import gs2
    from paper_2501_13975_b300.learned import RecordSet, StepModel
    master, bits = synth.mlp_init(33, out_scale=1.0)
    rec = _random_records(34, chunks=2)
    chunk_n = rec.shape[2]
    recs = RecordSet(torch.tensor(rec, device="cuda").reshape(-1), chunk_n)
    model = StepModel(master=master, bits=bits)
    lr = 1e-3
    model.step(recs, None, recs.n, lr)
    X, Y = _oracle_xy(rec, np.arange(recs.n))
    _, cnt, g = Lr.mlp_loss_grad(Lr.bf16_to_f64(bits), X, Y)
    q, _, _ = Lr.adam_step(master.astype(np.float64), g / cnt, np.zeros_like(g), np.zeros_like(g), 1, lr)
    got = model.master.cpu().numpy().astype(np.float64)
    # the first step is lr g / (|g| + eps): its size depends on g only where |g| ~ eps
    assert np.abs(got - q).max() <= 1e-3 * lr + 1e-7
    wb = model.w.cpu().numpy().view(np.uint16)
    m32 = model.master.cpu().numpy()
    u = m32.view(np.uint32).astype(np.uint64)
    rne = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16).astype(np.uint16)
    assert np.array_equal(wb, rne)
    assert gs2.MLP_NPARAM == Lr.NPARAM


def _blocks_and_steps(gs2, group, model_bits=None, seed=40):
    """GPU and oracle blocks and plain steps for one group, 4 views (primary
    plus 3 downsampled secondaries) of a 1500-Gaussian tiny scene."""
    sh = 3 if group == O.COLOR else 0
    sc = synth.tiny_scene(n=1500, seed=seed, sh_degree=sh)
    if sh:
        sc.sh[:, 1:, :] = np.random.default_rng(seed + 1).normal(0, 0.1, sc.sh[:, 1:, :].shape).astype(np.float32)
    cams = synth.ring_cameras(4, 128)
    gt = synth.perturbed(sc, seed=seed + 2, sd=0.05)
    ctx = gs2.Context(sc.n, 128, 128, 3)
    ocfg = oracle_cfg(ctx.config)
    primary = cams[0]
    ds = gs2.DeviceScene.from_host(sc)
    nv = 4
    blocks = ctx.blocks_buffer(group, sc.n, sh, nv)
    ob = None
    gp = None
    amb = None
    for slot in range(4):
        cam = primary if slot == 0 else O.downsample_camera(cams[slot], 2)
        cam = synth.Camera(cam.width, cam.height, cam.fx, cam.fy, cam.cx, cam.cy,
                           np.asarray(cam.viewmat, np.float32))
        tgt = O.render(gt, cam, ocfg)["image"].astype(np.float32)
        proj = ctx.project(ds, cam)
        img, rs = ctx.raster_fwd(ds, cam, proj)
        ctx.accum(group, ds, cam, primary, proj, rs, img, torch.tensor(tgt, device="cuda"), slot, blocks)
        r = O.render(sc, cam, ocfg)
        L = O.loss(r["image"], tgt, ocfg)
        ob = O.accum(group, sc, cam, primary, L["e"], L["h"], ocfg, out=ob)
        if slot == 0:
            gp = np.array(ob["g"], copy=True)
        a, _ = ambiguous_gaussians(O, sc, cam, ocfg, r["margin"], thresh=2e-5, dilate=10)
        amb = a if amb is None else (amb | a)
    plain = ctx.solve(group, blocks, nv, ds, primary)
    rec = ctx.step_records(group, blocks, nv, ds, plain)
    learned = None
    if model_bits is not None:
        w = torch.tensor(model_bits.astype(np.int16), device="cuda")
        ctx.set_step_model(w)
        learned = ctx.solve(group, blocks, nv, ds, primary)
        ctx.set_step_model(None)
    torch.cuda.synchronize()
    ctx.check()
    os_ = O.solve(group, sc, primary, ob["g"], ob["H"], ocfg)
    st_ok = (os_["status"] == 0).all(0) if group == O.COLOR else (os_["status"] == 0)
    keep = ~amb & (ob["npix"] > 0) & st_ok
    return dict(sc=sc, ocfg=ocfg, ob=ob, gp=gp, os=os_, keep=keep, plain=plain.cpu().numpy(), rec=rec.cpu().numpy(),
                learned=None if learned is None else learned.cpu().numpy(), n=sc.n, S=(sh + 1) ** 2)


@pytest.mark.parametrize("group", [0, 1, 2, 3, 4])
def test_step_records_match_oracle(group):
    from paper_2501_13975_b300 import gs2
    c = _blocks_and_steps(gs2, group)
    orec = Lr.step_records(group, c["ob"]["g"], c["ob"]["H"], c["os"]["step"], c["sc"], c["ocfg"], c["gp"])
    grec = c["rec"]
    both = c["keep"] & (orec[Lr.NF + 1] >= 0) & (grec[Lr.NF + 1] >= 0)
    # usability agrees wherever the oracle's g.d is clearly negative
    gn = np.linalg.norm(np.asarray(c["ob"]["g"]).reshape(-1, c["n"]), axis=0)
    dn = np.linalg.norm(np.asarray(c["os"]["step"]).reshape(-1, c["n"]), axis=0)
    clear = c["keep"] & (orec[Lr.NF] < -1e-3 * gn * dn)
    assert np.array_equal(grec[Lr.NF + 1][clear] >= 0, orec[Lr.NF + 1][clear] >= 0)
    assert both.sum() >= 50, both.sum()
    # f4 divides by g.d: compared where the step clearly descends
    firm = both & (orec[Lr.NF] < -0.05 * gn * dn)
    for j, tol in ((0, 2e-3), (1, 2e-3), (2, 2e-3), (3, 1e-6), (4, 2e-3), (6, 2e-3)):
        m = firm if j == 4 else both
        d = np.abs(grec[j][m] - orec[j][m])
        assert np.quantile(d, 0.99) <= tol and d.max() <= 50 * tol, (j, d.max(), np.quantile(d, 0.99))
    assert np.all(grec[7] == np.float32(group / 4.0))
    # the clip flag: equal except within 1e-4 of the threshold
    flag_diff = grec[5][both] != orec[5][both]
    assert flag_diff.mean() <= 0.01, flag_diff.mean()
    sc = np.maximum(gn * dn, 1e-30)[both]
    assert np.quantile(np.abs(grec[Lr.NF][both] - orec[Lr.NF][both]) / sc, 0.99) <= 2e-3


def test_logged_sweep_matches_plain_sweep_and_oracle():
    """The logged sweep ends where gs2_sweep ends; its records (features from
    the solve's blocks, labels from the loss over all 4 views) match the
    oracle's logged sweep."""
    from paper_2501_13975_b300 import gs2
    sc = synth.tiny_scene(n=300, seed=41)
    gt = synth.perturbed(sc, seed=42, sd=0.05)
    cams = synth.ring_cameras(4, 64)
    ctx = gs2.Context(sc.n, 64, 64, 0)
    ocfg = oracle_cfg(ctx.config)
    tg_np = np.stack([O.render(gt, c, ocfg)["image"] for c in cams]).astype(np.float32)
    targets = [torch.tensor(x, device="cuda") for x in tg_np]
    sphere = O.bounding_sphere(sc)
    centres = np.stack([c.center() for c in cams])
    knn, _ = O.knn(centres, sphere, 3)
    t = 2
    a = gs2.DeviceScene.from_host(sc)
    rec = ctx.sweep_logged(a, cams, targets, knn, t)
    b = gs2.DeviceScene.from_host(sc)
    ctx.sweep(b, cams, targets, knn, t)
    torch.cuda.synchronize()
    ctx.check()
    for name in ("mean", "quat", "scale", "opacity", "sh"):
        x, y = getattr(a, name), getattr(b, name)
        assert float((x - y).abs().max()) <= 1e-4 * max(1.0, float(y.abs().max())), name
    _, orec = Lr.sweep_logged(sc, cams, tg_np.astype(np.float64), knn, t, ocfg)
    grec = rec.cpu().numpy()
    for group in range(5):
        g, o = grec[group], orec[group]
        both = (g[Lr.NF + 1] >= 0) & (o[Lr.NF + 1] >= 0)
        assert both.sum() >= 30, (group, both.sum())
        agree = (g[Lr.NF + 1] >= 0) == (o[Lr.NF + 1] >= 0)
        assert agree.mean() >= 0.97, (group, agree.mean())
        # labels: well-conditioned where |phi0 - phi1| is not small against |phi0|
        phi0 = o[Lr.NF][both]
        lab_o = o[Lr.NF + 1][both]
        cond = (lab_o > 0.05) & (lab_o < 1.95)
        d = np.abs(g[Lr.NF + 1][both] - lab_o)[cond]
        if d.size:
            assert np.quantile(d, 0.95) <= 2e-2, (group, np.quantile(d, 0.95))
        del phi0


@pytest.mark.parametrize("group", [0, 2, 3, 4])
def test_learned_scale_inside_solve_matches_oracle(group):
    """gs2_solve_step with a network installed = the oracle's learned step
    (alpha from its FP64 forward of the BF16 weights on its own record)."""
    from paper_2501_13975_b300 import gs2
    _, bits = synth.mlp_init(43, out_scale=2.0)
    c = _blocks_and_steps(gs2, group, model_bits=bits)
    p = Lr.bf16_to_f64(bits)
    ref = Lr.learned_step(group, c["ob"]["g"], c["ob"]["H"], c["os"]["step"], c["sc"], c["ocfg"], p, c["gp"])
    n = c["n"]
    got = c["learned"][: ref.size].reshape(ref.shape)
    ref2 = ref.reshape(-1, n)
    got2 = got.reshape(-1, n)
    plain2 = c["plain"][: ref.size].reshape(-1, n)
    keep = c["keep"]
    nr = np.maximum(np.linalg.norm(ref2, axis=0), 1e-12)
    err = np.linalg.norm(got2 - ref2, axis=0) / nr
    assert np.quantile(err[keep], 0.99) <= 5e-3, np.quantile(err[keep], 0.99)
    # the network changed the steps (scales away from 1)
    ratio = np.linalg.norm(got2, axis=0)[keep] / np.maximum(np.linalg.norm(plain2, axis=0)[keep], 1e-30)
    assert np.std(ratio) > 0.01


def test_non_finite_network_falls_back_to_plain_step():
    from paper_2501_13975_b300 import gs2
    bits = np.full(gs2.MLP_NPARAM, 0x7FC0, np.uint16)     # NaN everywhere
    c = _blocks_and_steps(gs2, O.POS, model_bits=bits)
    assert np.array_equal(c["learned"], c["plain"])


def test_trained_network_gains_over_plain_step():
    """Records from 150 logged tiny-scene runs (seeds 100..249), trained on
    the first 80% of the runs: on the held-out runs the network's error
    against the labels is well below the plain step's (alpha = 1)."""
    from paper_2501_13975_b300 import learned
    recs = learned.collect_records(range(100, 250))
    train, held = recs.split(0.2)
    base, cnt = learned.plain_loss(held)
    model = learned.StepModel(seed=20)
    l0, _ = model.loss(held)
    model.fit(train, epochs=4, batch=8192)
    l1, cnt1 = model.loss(held)
    print(f"\nheld-out records {cnt}: plain {base:.4g}, initial {l0:.4g}, trained {l1:.4g}")
    assert cnt1 == cnt and cnt > 100_000
    assert l1 < 0.8 * base
    # line-model objective: the predicted change of the loss over all views
    # (about -1 per chunk for the plain step) falls further with the network
    lbase, _ = learned.plain_loss(held, objective="line")
    line_model = learned.StepModel(seed=20).fit(train, epochs=4, batch=8192, objective="line")
    l2, _ = line_model.loss(held, objective="line")
    print(f"line objective: plain {lbase:.4g}, trained {l2:.4g}")
    assert l2 < lbase

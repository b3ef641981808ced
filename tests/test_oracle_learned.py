"""Pins of the learned-step-scale oracle (oracle/learned.py) against
mathematics it does not itself use: central finite differences and torch
autograd for the network gradient, closed forms for the output layer, Adam's
first step and the quadratic line model, and finite differences of the
rendered loss along the step for phi0 and phi1."""
import numpy as np
import pytest

from oracle import learned as Lr
from oracle import oracle as O
from paper_2501_13975_b300 import synth


def _params(seed=0, scale=0.3):
    rng = np.random.default_rng(seed)
    p = rng.normal(0.0, scale, Lr.NPARAM)
    p[Lr.OFF_B1:Lr.OFF_W2] = rng.uniform(0.05, 0.3, Lr.NH)   # keep most units active
    p[Lr.OFF_B2:Lr.OFF_W3] = rng.uniform(0.05, 0.3, Lr.NH)
    return p


def _batch(seed=1, m=16):
    rng = np.random.default_rng(seed)
    X = rng.normal(0.0, 1.0, (m, Lr.NF))
    Y = rng.uniform(0.0, 2.0, m)
    Y[3] = -1.0            # unusable label
    X[5, 2] = np.nan       # unusable feature
    return X, Y


def test_bf16_decoding():
    bits = np.array([0x3F80, 0xC000, 0x7F80, 0x0001, 0x3E80, 0x4049], np.uint16)
    v = Lr.bf16_to_f64(bits)
    assert v[0] == 1.0 and v[1] == -2.0 and np.isinf(v[2]) and v[4] == 0.25
    assert v[3] == 2.0 ** -133
    assert v[5] == 3.140625


def test_mlp_gradient_central_differences():
    p = _params()
    X, Y = _batch()
    loss, cnt, g = Lr.mlp_loss_grad(p, X, Y)
    assert cnt == 14
    assert loss == pytest.approx(Lr.mlp_loss(p, X, Y)[0], rel=1e-14)
    h = 1e-6
    fd = np.zeros(Lr.NPARAM)
    for i in range(Lr.NPARAM):
        e = np.zeros(Lr.NPARAM)
        e[i] = h
        fd[i] = (Lr.mlp_loss(p + e, X, Y)[0] - Lr.mlp_loss(p - e, X, Y)[0]) / (2 * h)
    err = np.abs(fd - g).max() / np.abs(g).max()
    assert err < 1e-6, err


def test_mlp_gradient_matches_torch_autograd():
    torch = pytest.importorskip("torch")
    p = _params(seed=3)
    X, Y = _batch(seed=4, m=40)
    _, _, g = Lr.mlp_loss_grad(p, X, Y)
    m = Lr.usable(X, Y)
    Xt = torch.tensor(X[m], dtype=torch.float64)
    Yt = torch.tensor(Y[m], dtype=torch.float64)
    pt = torch.tensor(p, dtype=torch.float64, requires_grad=True)
    W1 = pt[Lr.OFF_W1:Lr.OFF_B1].view(Lr.NH, Lr.NF)
    b1 = pt[Lr.OFF_B1:Lr.OFF_W2]
    W2 = pt[Lr.OFF_W2:Lr.OFF_B2].view(Lr.NH, Lr.NH)
    b2 = pt[Lr.OFF_B2:Lr.OFF_W3]
    W3 = pt[Lr.OFF_W3:Lr.OFF_B3]
    b3 = pt[Lr.OFF_B3]
    y = torch.relu(torch.relu(Xt @ W1.T + b1) @ W2.T + b2) @ W3 + b3
    a = 2 * torch.sigmoid(y)
    (0.5 * ((a - Yt) ** 2).sum()).backward()
    assert np.allclose(pt.grad.numpy(), g, rtol=1e-10, atol=1e-12)


def test_mlp_closed_form_with_zero_output_weights():
    """W3 = 0: alpha = 2 sigmoid(b3) for every input; dL/db3 = sum (a - y) a (1 - a/2),
    dL/dW3 = sum (a - y) a (1 - a/2) h2, all other gradients vanish."""
    p = _params(seed=5)
    p[Lr.OFF_W3:Lr.OFF_B3] = 0.0
    p[Lr.OFF_B3] = 0.4
    X, Y = _batch(seed=6)
    a0 = 2.0 / (1.0 + np.exp(-0.4))
    alpha, _ = Lr.mlp_forward(p, np.nan_to_num(X))
    assert np.allclose(alpha, a0, rtol=0, atol=1e-15)
    _, _, g = Lr.mlp_loss_grad(p, X, Y)
    m = Lr.usable(X, Y)
    r = (a0 - Y[m]) * a0 * (1 - a0 / 2)
    assert g[Lr.OFF_B3] == pytest.approx(r.sum(), rel=1e-12)
    h2 = np.maximum(np.maximum(X[m] @ p[:Lr.OFF_B1].reshape(Lr.NH, Lr.NF).T + p[Lr.OFF_B1:Lr.OFF_W2], 0)
                    @ p[Lr.OFF_W2:Lr.OFF_B2].reshape(Lr.NH, Lr.NH).T + p[Lr.OFF_B2:Lr.OFF_W3], 0)
    assert np.allclose(g[Lr.OFF_W3:Lr.OFF_B3], r @ h2, rtol=1e-12, atol=1e-14)
    assert np.all(g[:Lr.OFF_W3] == 0.0)


def test_adam_first_step_and_bias_correction():
    """From zero moments the first step is lr g / (|g| + eps) (bias-corrected
    moments equal g and g^2); a constant gradient keeps that step size."""
    rng = np.random.default_rng(7)
    p = rng.normal(size=50)
    g = rng.normal(size=50)
    q, m, v = Lr.adam_step(p, g, np.zeros(50), np.zeros(50), 1, 1e-2)
    assert np.allclose(q, p - 1e-2 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    for t in range(2, 6):
        q2, m, v = Lr.adam_step(q, g, m, v, t, 1e-2)
        assert np.allclose(q2 - q, -1e-2 * g / (np.abs(g) + 1e-8), rtol=1e-9, atol=1e-14)
        q = q2


# ---------------------------------------------------------------- records
def _scene_for(n, seed=8):
    return synth.tiny_scene(n=n, seed=seed)


def _spd(rng, D, cond=20.0):
    Q, _ = np.linalg.qr(rng.normal(size=(D, D)))
    return Q @ np.diag(np.geomspace(1.0, cond, D)) @ Q.T


def _pos_blocks(rng, n, mu=0.0):
    """Random 3x3 SPD blocks and gradients; d = -(H + mu I)^-1 g."""
    g = rng.normal(size=(3, n))
    Hs = [_spd(rng, 3) for _ in range(n)]
    Hu = np.stack([[H[0, 0], H[0, 1], H[0, 2], H[1, 1], H[1, 2], H[2, 2]] for H in Hs], axis=1)
    d = np.stack([-np.linalg.solve(H + mu * np.eye(3), g[:, k]) for k, H in enumerate(Hs)], axis=1)
    return g, Hu, d, Hs


def test_record_of_undamped_newton_step_and_its_label():
    """d = -H^-1 g: d^T H d = -g.d, so f0 = 0; on the quadratic model g_after
    = g + H d = 0, so alpha* = 1."""
    rng = np.random.default_rng(9)
    sc = _scene_for(6)
    g, Hu, d, Hs = _pos_blocks(rng, 6)
    cfg = dict(trust_pos=1e9)                       # no trust radius in the way
    rec = Lr.step_records(O.POS, g, Hu, d, sc, cfg)
    assert np.all(rec[Lr.NF + 1] == 0.0)
    assert np.allclose(rec[0], 0.0, atol=1e-12)
    cos = -np.sum(g * d, 0) / (np.linalg.norm(g, axis=0) * np.linalg.norm(d, axis=0))
    assert np.allclose(rec[1], cos, rtol=1e-12)
    assert np.all(rec[5] == 0.0) and np.all(rec[7] == 0.0)
    g_after = g + np.stack([H @ d[:, k] for k, H in enumerate(Hs)], axis=1)
    lab = Lr.step_labels(O.POS, g_after, d, rec)
    assert np.allclose(lab[Lr.NF + 1], 1.0, atol=1e-12)


def test_label_is_the_line_minimum_of_the_quadratic():
    """Damped d: on q(a) = a g.d + a^2/2 d^T H d the label equals argmin q
    (found by golden-section search, not by the formula); a concave line
    model gives 2; an ascent direction is unusable."""
    from scipy.optimize import minimize_scalar
    rng = np.random.default_rng(10)
    sc = _scene_for(5)
    g, Hu, d, Hs = _pos_blocks(rng, 5, mu=3.0)
    cfg = dict(trust_pos=1e9)
    rec = Lr.step_records(O.POS, g, Hu, d, sc, cfg)
    g_after = g + np.stack([H @ d[:, k] for k, H in enumerate(Hs)], axis=1)
    lab = Lr.step_labels(O.POS, g_after, d, rec)[Lr.NF + 1]
    for k, H in enumerate(Hs):
        gd, q = g[:, k] @ d[:, k], d[:, k] @ H @ d[:, k]
        best = minimize_scalar(lambda a: a * gd + 0.5 * a * a * q, bracket=(0.0, 1.0), tol=1e-12).x
        assert lab[k] == pytest.approx(min(max(best, 0.0), 2.0), abs=1e-7)
        assert lab[k] > 1.0          # damping shortens the step: the minimum lies beyond it
    # concave: g_after.d below g.d
    lab2 = Lr.step_labels(O.POS, g - 0.5 * np.abs(g) * np.sign(d), d, rec)[Lr.NF + 1]
    assert np.all(lab2 == 2.0)
    # ascent direction
    rec_up = Lr.step_records(O.POS, g, Hu, -d, sc, cfg)
    assert np.all(rec_up[Lr.NF + 1] == -1.0)


def test_features_invariant_to_loss_normalisation():
    """Scaling g and H by c > 0 (a differently normalised loss) leaves d and
    every feature unchanged."""
    rng = np.random.default_rng(11)
    sc = _scene_for(8)
    g, Hu, d, _ = _pos_blocks(rng, 8, mu=0.5)
    a = Lr.step_records(O.POS, g, Hu, d, sc, None)
    b = Lr.step_records(O.POS, 37.0 * g, 37.0 * Hu, d, sc, None)
    assert np.allclose(a[:Lr.NF], b[:Lr.NF], rtol=1e-12, atol=1e-12)


def test_colour_record_matches_dense_form():
    """Colour: d^T H d with the per-channel blocks equals the dense
    block-diagonal quadratic form; f7 = 1."""
    rng = np.random.default_rng(12)
    n, S = 4, 16
    sc = synth.tiny_scene(n=n, seed=12, sh_degree=3)
    g = rng.normal(size=(3, S, n))
    iu = np.triu_indices(S)
    Hs = [[_spd(rng, S, 50.0) for _ in range(3)] for _ in range(n)]
    Hu = np.stack([np.stack([Hs[k][c][iu] for k in range(n)], axis=1) for c in range(3)])
    d = np.stack([np.stack([-np.linalg.solve(Hs[k][c] + np.eye(S), g[c, :, k]) for k in range(n)], axis=1)
                  for c in range(3)])
    rec = Lr.step_records(O.COLOR, g, Hu, d, sc, dict(trust_color=1e9))
    for k in range(n):
        q = sum(d[c, :, k] @ Hs[k][c] @ d[c, :, k] for c in range(3))
        gd = float(np.sum(g[:, :, k] * d[:, :, k]))
        assert rec[0, k] == pytest.approx(np.log10(q / -gd), abs=1e-12)
        hd = np.mean([Hs[k][c][i, i] for c in range(3) for i in range(S)])
        assert rec[6, k] == pytest.approx(np.log10(np.linalg.norm(g[:, :, k]) / (hd * np.linalg.norm(d[:, :, k]))),
                                          abs=1e-12)
    assert np.all(rec[7] == 1.0)


def _group_loss(scene, views, cfg):
    tot = 0.0
    for cam, tgt in views:
        r = O.render(scene, cam, cfg)
        tot += O.loss(r["image"], tgt, cfg, derivs=False)["loss"]
    return tot


@pytest.mark.parametrize("group", [O.POS, O.OPACITY, O.COLOR])
def test_phi0_phi1_are_directional_derivatives(group):
    """phi0 = g.d and phi1 = g_after.d are the derivatives of the group's loss
    (primary plus downsampled secondaries) along d at steps 0 and 1 (central
    differences of the rendered loss; 3 Gaussians, 4 views)."""
    sc = synth.tiny_scene(n=3, seed=13, sh_degree=1)
    gt = synth.perturbed(sc, seed=14, sd=0.05)
    cams = synth.ring_cameras(4, 32)
    cfg = O.default_config()
    targets = [O.render(gt, c, cfg)["image"] for c in cams]
    knn = np.array([[1, 2, 3], [0, 2, 3], [0, 1, 3], [0, 1, 2]], np.int32)
    views = Lr._views(cams, targets, knn, 0, cfg)
    cur = O.scene_handle(sc)
    ob = Lr._blocks(group, cur, views, cams[0], cfg)
    st = O.solve(group, cur, cams[0], ob["g"], ob["H"], cfg)
    d = st["step"]
    gp = Lr._blocks(group, cur, views[:1], cams[0], cfg)["g"]
    rec = Lr.step_records(group, ob["g"], ob["H"], d, cur, cfg, gp)
    S = O.sh_count(sc.sh_degree)
    checked = 0
    for k in range(sc.n):
        if rec[Lr.NF + 1, k] < 0:
            continue
        dk = np.zeros_like(d)
        dk[..., k] = d[..., k]
        h = 1e-4

        def L(a):
            return _group_loss(O.apply(group, cur, cams[0], a * dk, cfg), views, cfg)

        phi0_fd = (L(h) - L(-h)) / (2 * h)
        phi1_fd = (L(1 + h) - L(1 - h)) / (2 * h)
        assert rec[Lr.NF, k] == pytest.approx(phi0_fd, rel=1e-4, abs=1e-12)
        # f4: the primary view's share of that derivative
        Lp = lambda a: _group_loss(O.apply(group, cur, cams[0], a * dk, cfg), views[:1], cfg)  # noqa: E731
        share = ((Lp(h) - Lp(-h)) / (2 * h)) / phi0_fd
        assert rec[4, k] == pytest.approx(min(max(share, -4.0), 4.0), rel=1e-3, abs=1e-6)
        # Gaussian k stepped alone: its after-step gradient along d
        oa = Lr._blocks(group, O.apply(group, cur, cams[0], dk, cfg), views, cams[0], cfg)
        phi1 = float(np.sum(np.asarray(oa["g"])[..., k] * d[..., k]))
        assert phi1 == pytest.approx(phi1_fd, rel=1e-3, abs=1e-6 * abs(phi0_fd))
        lab = Lr.step_labels(group, oa["g"], d, rec, S)[Lr.NF + 1, k]
        den = rec[Lr.NF, k] - phi1_fd
        expect = 2.0 if den >= 0 else min(max(rec[Lr.NF, k] / den, 0.0), 2.0)
        assert lab == pytest.approx(expect, rel=5e-3, abs=1e-6)
        checked += 1
    assert checked >= 2


@pytest.mark.parametrize("group", [O.POS, O.ROT, O.OPACITY, O.COLOR])
def test_global_phi_sums_are_derivatives_of_the_total_loss(group):
    """Every Gaussian steps together: the sums over Gaussians of phi0 and
    phi1 taken over all training views are the derivatives of the total loss
    along the whole step at 0 and 1 (chain rule; central differences).  The
    alpha_min skip is made negligible (1e-9): with every Gaussian moving, a
    pixel crossing it would put a jump inside the difference quotient."""
    sc = synth.tiny_scene(n=40, seed=18, sh_degree=1)
    gt = synth.perturbed(sc, seed=19, sd=0.05)
    cams = synth.ring_cameras(6, 32)
    cfg = O.default_config(alpha_min=1e-9)
    targets = [O.render(gt, c, cfg)["image"] for c in cams]
    every = [(c, targets[v]) for v, c in enumerate(cams)]
    knn = np.array([[1, 5, 2]] + [[0, 0, 0]] * 5, np.int32)
    views = Lr._views(cams, targets, knn, 0, cfg)
    cur = O.scene_handle(sc)
    ob = Lr._blocks(group, cur, views, cams[0], cfg)
    d = O.solve(group, cur, cams[0], ob["g"], ob["H"], cfg)["step"]
    phi0 = Lr.phi(group, Lr._blocks(group, cur, every, cams[0], cfg)["g"], d)
    phi1 = Lr.phi(group, Lr._blocks(group, O.apply(group, cur, cams[0], d, cfg), every, cams[0], cfg)["g"], d)
    h = 1e-5

    def L(a):
        return _group_loss(O.apply(group, cur, cams[0], a * d, cfg), every, cfg)

    assert phi0.sum() == pytest.approx((L(h) - L(-h)) / (2 * h), rel=2e-4)
    assert phi1.sum() == pytest.approx((L(1 + h) - L(1 - h)) / (2 * h), rel=2e-4)


def test_rejected_step_has_label_zero():
    """A usable record whose step does not descend the label loss (phi0 >= 0)
    gets label 0; a descending one the line-model minimum."""
    rec = np.zeros((Lr.REC_ROWS, 3))
    rec[Lr.NF] = -1.0
    rec[Lr.NF + 1] = [0.0, 0.0, -1.0]
    d = np.ones((1, 3))
    out = Lr.step_labels(O.OPACITY, np.array([[0.5, 0.5, 0.5]]), d, rec, phi0=np.array([0.2, -1.0, -1.0]))
    assert out[Lr.NF + 1, 0] == 0.0
    assert out[Lr.NF + 1, 1] == pytest.approx(1.0 / 1.5)
    assert out[Lr.NF + 1, 2] == -1.0
    assert np.array_equal(out[Lr.NF], [0.2, -1.0, -1.0])


def test_learned_step_bounds_and_fallback():
    """alpha -> 2 (large output bias): the step doubles inside learned_trust
    times the trust radius and is cut back to it outside (learned_trust 2 and
    1); a non-finite network leaves the plain step."""
    rng = np.random.default_rng(15)
    sc = _scene_for(10)
    g, Hu, d, _ = _pos_blocks(rng, 10, mu=1.0)
    sh = O.scene_handle(sc)
    smax = sh.scale.max(0)
    d *= (smax * 2.0) / np.linalg.norm(d, axis=0)             # |d| = 2 max(s)
    d[:, :5] *= 0.5                                            # |d| = max(s) for half
    p = np.zeros(Lr.NPARAM)
    p[Lr.OFF_B3] = 40.0                                        # alpha = 2 to double precision
    for cfg in (O.default_config(trust_pos=1.5, learned_trust=2.0),    # 2 x 1.5 max(s)
                O.default_config(trust_pos=3.0, learned_trust=1.0)):       # the plain radius, 3 max(s)
        # the cap, 3 max(s), lies between 2|d| of the two halves
        assert cfg["learned_trust"] * cfg["trust_pos"] == 3.0
        out = Lr.learned_step(O.POS, g, Hu, d, sc, cfg, p)
        n_out = np.linalg.norm(out, axis=0)
        assert np.allclose(n_out[:5], 2.0 * smax[:5], rtol=1e-12)
        assert np.allclose(n_out[5:], 3.0 * smax[5:], rtol=1e-12)
        assert np.allclose(out / n_out, d / np.linalg.norm(d, axis=0), rtol=1e-12)
    p_nan = p.copy()
    p_nan[Lr.OFF_B3] = np.nan
    assert np.array_equal(Lr.learned_step(O.POS, g, Hu, d, sc, cfg, p_nan), d)
    # opacity: bounded by the fraction-to-boundary rule
    go = rng.normal(size=(1, 10))
    ho = np.abs(rng.normal(size=(1, 10))) + 0.1
    do = -go / ho
    out_o = Lr.learned_step(O.OPACITY, go, ho, do, sc, cfg, p)
    sg = sh.opacity
    assert np.all(out_o >= -0.99 * sg - 1e-15) and np.all(out_o <= 0.99 * (1 - sg) + 1e-15)


def test_logged_sweep_equals_oracle_sweep():
    """The logged sweep (Python, oracle calls) ends in the same scene as the
    oracle's own sweep; its records have labels for the usable ones."""
    sc = synth.tiny_scene(n=60, seed=16)
    gt = synth.perturbed(sc, seed=17, sd=0.05)
    cams = synth.ring_cameras(4, 32)
    cfg = O.default_config()
    targets = np.stack([O.render(gt, c, cfg)["image"] for c in cams])
    knn = np.array([[1, 2, 3], [0, 2, 3], [0, 1, 3], [0, 1, 2]], np.int32)
    a, rec = Lr.sweep_logged(sc, cams, targets, knn, 1, cfg)
    b, _, _ = O.sweep(sc, cams, targets, knn, 1, cfg)
    for name in ("mean", "quat", "scale", "opacity", "sh"):
        assert np.allclose(getattr(a, name), getattr(b, name), rtol=0, atol=1e-12), name
    assert rec.shape == (5, Lr.REC_ROWS, sc.n)
    lab = rec[:, Lr.NF + 1]
    assert np.all((lab == -1.0) | ((lab >= 0.0) & (lab <= 2.0)))
    assert (lab >= 0).sum() >= 100


def _line_batch(seed=20, m=24):
    rng = np.random.default_rng(seed)
    X = rng.normal(0.0, 1.0, (m, Lr.NF))
    Y = rng.uniform(0.0, 2.0, m)
    Y[2] = -1.0
    phi0 = -np.abs(rng.normal(1.0, 0.5, m))
    phi0[4] = 0.3                      # a rejected step (ascent of the label loss)
    phi1 = phi0 + rng.uniform(-0.5, 2.0, m)
    return X, Y, Lr.line_terms(phi0, phi1, 0.7)


def test_line_objective_gradient_central_differences():
    p = _params(seed=21)
    X, Y, line = _line_batch()
    loss, cnt, g = Lr.mlp_loss_grad(p, X, Y, line)
    assert cnt == 23
    assert loss == pytest.approx(Lr.mlp_loss(p, X, Y, line)[0], rel=1e-13)
    h = 1e-6
    idx = np.random.default_rng(22).choice(Lr.NPARAM, 400, replace=False)
    for i in idx:
        e = np.zeros(Lr.NPARAM)
        e[i] = h
        fd = (Lr.mlp_loss(p + e, X, Y, line)[0] - Lr.mlp_loss(p - e, X, Y, line)[0]) / (2 * h)
        assert fd == pytest.approx(g[i], abs=1e-7 * np.abs(g).max())


def test_line_objective_closed_form_and_minimiser():
    """W3 = 0: every alpha = 2 sigmoid(b3) and dL/db3 = sum (s phi0 + s (phi1 - phi0) alpha)
    alpha (1 - alpha/2); a single convex descent record's loss is smallest at its label."""
    p = _params(seed=23)
    p[Lr.OFF_W3:Lr.OFF_B3] = 0.0
    p[Lr.OFF_B3] = -0.3
    X, Y, line = _line_batch(seed=24)
    a0 = 2.0 / (1.0 + np.exp(0.3))
    m = Lr.usable(X, Y)
    _, _, g = Lr.mlp_loss_grad(p, X, Y, line)
    assert g[Lr.OFF_B3] == pytest.approx(np.sum(((line[0] + line[1] * a0) * a0 * (1 - a0 / 2))[m]), rel=1e-12)
    # minimiser of s (phi0 a + 1/2 (phi1 - phi0) a^2) = the label of step_labels
    rec = np.zeros((Lr.REC_ROWS, 1))
    rec[Lr.NF] = -0.8
    lab = Lr.step_labels(O.POS, np.array([[0.4]]), np.array([[1.0]]), rec)   # phi1 = 0.4
    a = np.linspace(0, 2, 200001)
    q = -0.8 * a + 0.5 * (0.4 + 0.8) * a * a
    assert lab[Lr.NF + 1, 0] == pytest.approx(a[np.argmin(q)], abs=1e-4)
    assert lab[Lr.NF + 2, 0] == pytest.approx(0.4)


def test_chunk_scale():
    rec = np.zeros((2, Lr.REC_ROWS, 3))
    rec[0, Lr.NF] = [-1.0, -3.0, 2.0]
    rec[0, Lr.NF + 1] = [0.0, 1.0, -1.0]          # the third record is unusable
    rec[1, Lr.NF + 1] = -1.0                       # no usable record
    s = Lr.chunk_scale(rec)
    assert s[0] == pytest.approx(0.25) and s[1] == 0.0


# ---------------------------------------------------------------- learned damping
def _iso_blocks(rng, n, h):
    """Position blocks with H = h I (so the reduced 2x2 block is h I for any
    basis of the plane) and random gradients."""
    g = rng.normal(size=(3, n))
    Hu = np.zeros((6, n))
    Hu[0] = Hu[3] = Hu[5] = h
    return g, Hu


@pytest.mark.parametrize("mu0, c, want", [(1.0, 2.0, 0.0), (0.01, 2.0, 4.0 / 3.0),
                                          (1.0, 1.0, 0.0), (0.1, 11.0, 4.0 / 3.0),
                                          (0.1, 1.0 + 0.1 * 10.0 ** 2.5, 5.0 / 3.0)])
def test_damping_label_closed_form(mu0, c, want):
    """H = h I, g_all = g, H_all = c h I: the damped step (h + mu h) d = -g
    in the plane has Q = |g_v|^2 / h (c t^2 / 2 - t), t = 1 / (1 + mu),
    minimal at t = 1 / c, i.e. mu = c - 1.  With mu = mu0 rho on the grid
    10^0, 10^0.5, .., 10^3: rho* = (c - 1) / mu0 (label 2 log10(rho*) / 3),
    and where that is below the grid (c = 1: the exact Newton step is best;
    mu0 = c - 1) the smallest rho, 1 (label 0)."""
    rng = np.random.default_rng(21)
    n, h = 8, 2.5
    sc = _scene_for(n)
    g, Hu = _iso_blocks(rng, n, h)
    cfg = O.default_config(damping_mu0=mu0, trust_pos=1e9)
    cams = synth.ring_cameras(4, 32)
    d = O.solve(O.POS, sc, cams[0], g, Hu, cfg)["step"]
    rec = Lr.step_records(O.POS, g, Hu, d, sc, cfg)
    out = Lr.damping_records(O.POS, g, Hu, rec, sc, cams[0], g, c * Hu, cfg)
    assert np.array_equal(out[:Lr.NF], rec[:Lr.NF])
    assert np.allclose(out[Lr.NF + 1], want, atol=1e-12), out[Lr.NF + 1]
    # Q of the candidates, from the plane's closed form (not the oracle's Q),
    # and the weight w = max Q - min Q of rows 8 and 10
    sh = O.scene_handle(sc)
    for k in range(n):
        r = np.asarray(sh.mean, np.float64).reshape(3, n)[:, k] - cams[0].center()
        r /= np.linalg.norm(r)
        gv2 = np.sum(g[:, k] ** 2) - np.dot(g[:, k], r) ** 2       # |g_v|^2: g without its ray component
        qs = []
        for rho in Lr.RHO_GRID:
            t = 1.0 / (1.0 + mu0 * rho)
            dk = O.solve(O.POS, sc, cams[0], g, Hu, dict(cfg, damping_mu0=mu0 * rho))["step"][:, k]
            q = np.dot(g[:, k], dk) + 0.5 * c * h * np.dot(dk, dk)
            assert q == pytest.approx(gv2 / h * (0.5 * c * t * t - t), rel=1e-9, abs=1e-14)
            qs.append(gv2 / h * (0.5 * c * t * t - t))
        w = max(qs) - min(qs)
        assert out[Lr.NF, k] == pytest.approx(-w * want, rel=1e-9, abs=1e-15)
        assert out[Lr.NF + 2, k] - out[Lr.NF, k] == pytest.approx(w, rel=1e-9)


def test_damping_records_unusable_and_other_groups():
    """Rotation and opacity get no damping label (1 x 1 blocks: damping and
    step scale coincide); an unusable step record stays unusable; a model
    that no candidate lowers (Q >= 0) gives no label."""
    rng = np.random.default_rng(22)
    n = 6
    sc = _scene_for(n)
    cams = synth.ring_cameras(4, 32)
    cfg = O.default_config(trust_pos=1e9)
    g, Hu = _iso_blocks(rng, n, 1.0)
    d = O.solve(O.POS, sc, cams[0], g, Hu, cfg)["step"]
    rec = Lr.step_records(O.POS, g, Hu, d, sc, cfg)
    rec[Lr.NF + 1, 0] = -1.0
    out = Lr.damping_records(O.POS, g, Hu, rec, sc, cams[0], g, Hu, cfg)
    assert out[Lr.NF + 1, 0] == -1.0 and np.all(out[Lr.NF + 1, 1:] == 0.0)
    assert out[Lr.NF, 0] == 0.0 and out[Lr.NF + 2, 0] == 0.0      # no label: no weight
    up = Lr.damping_records(O.POS, g, Hu, rec, sc, cams[0], -g, Hu, cfg)   # every candidate ascends Q
    assert np.all(up[Lr.NF + 1] == -1.0)
    go = rng.normal(size=(1, n))
    ho = np.abs(rng.normal(size=(1, n))) + 0.1
    for grp in (O.ROT, O.OPACITY):
        do = O.solve(grp, sc, cams[0], go, ho, cfg)["step"]
        r1 = Lr.step_records(grp, go, ho, do, sc, cfg)
        assert np.all(Lr.damping_records(grp, go, ho, r1, sc, cams[0], go, ho, cfg)[Lr.NF + 1] == -1.0)


def test_damped_step_constant_network():
    """A network with zero weights and output bias b gives alpha = 2 sigmoid(b)
    for every usable record, so rho is one value and the damped step equals
    O.solve with damping_mu0 rho; unusable records keep rho = 1."""
    rng = np.random.default_rng(23)
    n = 10
    sc = _scene_for(n)
    cams = synth.ring_cameras(4, 32)
    cfg = O.default_config(trust_pos=1e9)
    g, Hu, d, _ = _pos_blocks(rng, n, mu=0.3)
    d = O.solve(O.POS, sc, cams[0], g, Hu, cfg)["step"]
    p = np.zeros(Lr.NPARAM)
    p[Lr.OFF_B3] = np.log(1.5 / 0.5)              # alpha = 1.5: rho = 10^2.25
    out, rho = Lr.damped_step(O.POS, g, Hu, d, sc, cams[0], cfg, p)
    assert np.allclose(rho, 10.0 ** 2.25, rtol=1e-12)
    want = O.solve(O.POS, sc, cams[0], g, Hu, dict(cfg, damping_mu0=10.0 ** 2.25))["step"]
    assert np.allclose(out, want, rtol=1e-12, atol=0)
    assert np.linalg.norm(out) < np.linalg.norm(d)   # more damping, shorter steps

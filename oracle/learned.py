"""FP64 oracle of the learned step scale (an extension of the local Newton
step of Sec. 4.2, whose step size is 1): step records of the plain method,
their labels, the 8-64-64-1 step-scale MLP, its loss gradient and Adam.

TEST INFRASTRUCTURE ONLY: imported by tests/ and the CPU legs of bench.py.
It uses the FP64 oracle (oracle.py) for blocks and steps and plain numpy for
everything else; it never imports the CUDA package.

Definitions (g, H: a Gaussian's group block; d: its plain damped step):
  record  f0 = log10 clamp(d^T H d / (-g.d), 1e-6, 1e6)
          f1 = cos(-g, d)
          f2 = log10 max(|d| / u, 1e-12), u = max(s) for position/scaling, else 1
          f3 = sigma
          f4 = clamp(g_p.d / g.d, -4, 4): the share of the predicted decrease
               that the primary view's own gradient g_p gives (1 without g_p)
          f5 = 1 if a trust radius or bound is within 1e-3 of limiting d
          f6 = log10 clamp(|g| / (mean|diag H| |d|), 1e-6, 1e6)
          f7 = group / 4
          phi0 = g.d; usable iff |d| > 0, phi0 < 0 and all features finite
  label   of a loss L_lab along d: phi0 = grad L_lab . d before the step,
          phi1 = grad L_lab . d once every Gaussian of the group took its
          step; alpha* = 0 if phi0 >= 0 (d does not descend L_lab: the step
          is rejected), else the minimum of the quadratic through phi0 and
          phi1, phi0 / (phi0 - phi1) (2 when phi1 <= phi0, the model then
          being concave), clipped to [0, 2].  With L_lab the local loss (the
          views the step was solved from) phi0 is the record's own g.d; the
          logged sweep takes L_lab = the loss summed over every training view
          at full resolution, whose increase is what the paper calls
          overshoot (Sec. overshoot).
  rows    0-7 features, 8 phi0, 9 label (-1 unusable, 0 pending), 10 phi1
  network y = W3 relu(W2 relu(W1 x + b1) + b2) + b3, alpha = 2 sigmoid(y)
  loss    over usable records: 1/2 sum (alpha - alpha*)^2 (labels), or the
          line model's predicted change of the label loss,
          sum s_c (phi0 alpha + 1/2 (phi1 - phi0) alpha^2) (line), with
          s_c = 1 / sum |phi0| over the usable records of the record's chunk
  Adam    m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
          p -= lr (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps)
  damping a second network of the same shape gives rho = 10^(1.5 alpha) in
          (1, 1e3), the multiplier of damping_mu0 in a second solve (position,
          scaling, colour); its label is 2 log10(rho*) / 3, rho* in 10^0 .. 10^3
          minimising Q(d) = g_all . d + 1/2 d^T H_all d over the candidate
          steps, g_all, H_all the blocks over every training view
"""
from __future__ import annotations

import numpy as np

from oracle import oracle as O

NF, NH = 8, 64
OFF_W1 = 0
OFF_B1 = OFF_W1 + NH * NF
OFF_W2 = OFF_B1 + NH
OFF_B2 = OFF_W2 + NH * NH
OFF_W3 = OFF_B2 + NH
OFF_B3 = OFF_W3 + NH
NPARAM = OFF_B3 + 1
REC_ROWS = NF + 3


# ---------------------------------------------------------------- parameters
def bf16_to_f64(bits) -> np.ndarray:
    """BF16 bit patterns (uint16) -> float64: the upper half of an FP32 word."""
    b = np.asarray(bits).astype(np.uint16).astype(np.uint32) << np.uint32(16)
    return b.view(np.float32).astype(np.float64)


def unpack(p):
    p = np.asarray(p, np.float64)
    return dict(W1=p[OFF_W1:OFF_B1].reshape(NH, NF), b1=p[OFF_B1:OFF_W2], W2=p[OFF_W2:OFF_B2].reshape(NH, NH),
                b2=p[OFF_B2:OFF_W3], W3=p[OFF_W3:OFF_B3], b3=p[OFF_B3])


def pack(W1, b1, W2, b2, W3, b3) -> np.ndarray:
    return np.concatenate([np.ravel(W1), np.ravel(b1), np.ravel(W2), np.ravel(b2), np.ravel(W3),
                           np.atleast_1d(b3)]).astype(np.float64)


# ---------------------------------------------------------------- network
def mlp_forward(p, X):
    """alpha for the rows of X (m, 8); also returns the activations."""
    w = unpack(p)
    X = np.asarray(X, np.float64)
    z1 = X @ w["W1"].T + w["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ w["W2"].T + w["b2"]
    h2 = np.maximum(z2, 0.0)
    y = h2 @ w["W3"] + w["b3"]
    alpha = 2.0 / (1.0 + np.exp(-y))
    return alpha, dict(z1=z1, h1=h1, z2=z2, h2=h2, y=y)


def usable(X, Y):
    X = np.asarray(X, np.float64)
    Y = np.asarray(Y, np.float64)
    return (Y >= 0) & np.all(np.isfinite(X), axis=1)


def _per_record_loss(a, Y, m, line):
    """Loss and dL/d alpha per record (zero where unusable)."""
    if line is None:
        e = (a - np.where(m, Y, 0.0)) * m
        return 0.5 * e * e, e
    p0, cv = line            # s phi0, s (phi1 - phi0)
    p0 = np.where(m, p0, 0.0)
    cv = np.where(m, cv, 0.0)
    return (p0 * a + 0.5 * cv * a * a) * m, (p0 + cv * a) * m


def line_terms(phi0, phi1, scale):
    """(s phi0, s (phi1 - phi0)) per record for the line-model loss."""
    phi0 = np.asarray(phi0, np.float64)
    return scale * phi0, scale * (np.asarray(phi1, np.float64) - phi0)


def chunk_scale(rec_chunks):
    """s_c = 1 / sum |phi0| over the usable records of each chunk [..., REC_ROWS, n]."""
    r = np.asarray(rec_chunks, np.float64).reshape(-1, REC_ROWS, np.asarray(rec_chunks).shape[-1])
    ok = (r[:, NF + 1] >= 0) & np.isfinite(r[:, NF])
    tot = np.sum(np.where(ok, np.abs(r[:, NF]), 0.0), axis=1)
    return np.where(tot > 0, 1.0 / np.where(tot > 0, tot, 1.0), 0.0)


def mlp_loss(p, X, Y, line=None):
    m = usable(X, Y)
    if line is not None:
        m = m & np.isfinite(line[0]) & np.isfinite(line[1])
    a, _ = mlp_forward(p, np.where(m[:, None], X, 0.0))
    lr, _ = _per_record_loss(a, Y, m, line)
    return float(np.sum(lr)), int(m.sum())


def mlp_loss_grad(p, X, Y, line=None):
    """(loss sum, usable count, gradient of the loss sum w.r.t. p) by reverse-mode chain rule."""
    m = usable(X, Y)
    if line is not None:
        m = m & np.isfinite(line[0]) & np.isfinite(line[1])
    X = np.where(m[:, None], np.asarray(X, np.float64), 0.0)
    w = unpack(p)
    a, act = mlp_forward(p, X)
    lr, e = _per_record_loss(a, np.asarray(Y, np.float64), m, line)
    loss = float(np.sum(lr))
    dy = e * a * (1.0 - 0.5 * a)                       # dL/dy; d alpha/dy = alpha (1 - alpha/2)
    gW3 = act["h2"].T @ dy
    gb3 = dy.sum()
    d2 = np.outer(dy, w["W3"]) * (act["z2"] > 0)       # dL/dz2
    gW2 = d2.T @ act["h1"]
    gb2 = d2.sum(0)
    d1 = (d2 @ w["W2"]) * (act["z1"] > 0)              # dL/dz1
    gW1 = d1.T @ X
    gb1 = d1.sum(0)
    return loss, int(m.sum()), pack(gW1, gb1, gW2, gb2, gW3, gb3)


def adam_step(master, grad, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (returns new master, m, v)."""
    m = b1 * m + (1.0 - b1) * grad
    v = b2 * v + (1.0 - b2) * grad * grad
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return master - lr * mh / (np.sqrt(vh) + eps), m, v


def records_to_xy(rec):
    """Records [REC_ROWS][n] (or [..., REC_ROWS, n]) -> X (m, 8), Y (m,)."""
    r = np.asarray(rec, np.float64)
    r = np.moveaxis(r.reshape(-1, REC_ROWS, r.shape[-1]), 1, 2).reshape(-1, REC_ROWS)
    return r[:, :NF], r[:, NF + 1]


# ---------------------------------------------------------------- records
def _full_sym3(Hu):
    """(6, n) upper triangle 00 01 02 11 12 22 -> (n, 3, 3)."""
    H = np.zeros((Hu.shape[1], 3, 3))
    iu = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
    for r, (i, j) in enumerate(iu):
        H[:, i, j] = Hu[r]
        H[:, j, i] = Hu[r]
    return H


def _full_colour(Hu, S):
    """(3, S(S+1)/2, n) upper triangles -> (n, 3, S, S)."""
    n = Hu.shape[2]
    H = np.zeros((n, 3, S, S))
    iu = np.triu_indices(S)
    for c in range(3):
        H[:, c, iu[0], iu[1]] = Hu[c].T
        H[:, c, iu[1], iu[0]] = Hu[c].T
    return H


def _near_or_past(v, lim):
    return v >= (1.0 - 1e-3) * lim


def _as_vectors(group, g, H, d, S):
    """Per Gaussian: g, d as (n, D) and H as (n, D, D) (colour block-diagonal)."""
    n = np.asarray(d).shape[-1]
    if group in (O.POS, O.SCALE):
        return np.asarray(g, np.float64).T, _full_sym3(np.asarray(H, np.float64)), np.asarray(d, np.float64).T
    if group in (O.ROT, O.OPACITY):
        return (np.asarray(g, np.float64).reshape(1, n).T, np.asarray(H, np.float64).reshape(1, 1, n).transpose(2, 0, 1),
                np.asarray(d, np.float64).reshape(1, n).T)
    Hc = _full_colour(np.asarray(H, np.float64), S)
    Hf = np.zeros((n, 3 * S, 3 * S))
    for c in range(3):
        Hf[:, c * S:(c + 1) * S, c * S:(c + 1) * S] = Hc[:, c]
    return (np.asarray(g, np.float64).reshape(3 * S, n).T, Hf, np.asarray(d, np.float64).reshape(3 * S, n).T)


def step_records(group, g, H, d, scene, cfg, g_primary=None):
    """Records [REC_ROWS][n] (label row 0 = pending, -1 = unusable) of the
    plain step d (oracle layouts: g, H, d as O.accum / O.solve give them) at
    the scene's current parameters; g_primary: the primary view's own
    gradient (same layout as g), None for f4 = 1."""
    cfg = O.default_config(**(cfg or {}))
    sc = O.scene_handle(scene)
    n, S = sc.n, O.sh_count(sc.sh_degree)
    scale = np.asarray(sc.scale, np.float64).reshape(3, n)
    sigma = np.asarray(sc.opacity, np.float64).reshape(n)
    gv, Hm, dv = _as_vectors(group, g, H, d, S)
    gd = np.einsum("ni,ni->n", gv, dv)
    q = np.einsum("ni,nij,nj->n", dv, Hm, dv)
    gn = np.linalg.norm(gv, axis=1)
    dn = np.linalg.norm(dv, axis=1)
    hd = np.mean(np.abs(np.diagonal(Hm, axis1=1, axis2=2)), axis=1)
    smax = scale.max(0)
    if group == O.POS:
        clipped = _near_or_past(dn, cfg["trust_pos"] * smax)
    elif group == O.SCALE:
        k = cfg["scale_trust"]
        clipped = np.any(_near_or_past(-dv.T, scale - scale / k) | _near_or_past(dv.T, k * scale - scale), axis=0)
    elif group == O.ROT:
        clipped = _near_or_past(np.abs(dv[:, 0]), cfg["trust_rot"])
    elif group == O.OPACITY:
        tau = cfg["frac_to_boundary"]
        clipped = _near_or_past(-dv[:, 0], tau * sigma) | _near_or_past(dv[:, 0], tau * (1.0 - sigma))
    else:
        cn = np.linalg.norm(dv.reshape(n, 3, S), axis=2)
        clipped = np.any(_near_or_past(cn, cfg["trust_color"]), axis=1)
    u = smax if group in (O.POS, O.SCALE) else np.ones(n)
    with np.errstate(divide="ignore", invalid="ignore"):
        ratio = np.where(-gd > 0, q / np.where(-gd > 0, -gd, 1.0), 1e6)
        f = np.zeros((NF, n))
        f[0] = np.log10(np.clip(ratio, 1e-6, 1e6))
        f[1] = np.where(gn * dn > 0, -gd / np.where(gn * dn > 0, gn * dn, 1.0), 0.0)
        f[2] = np.log10(np.maximum(dn / u, 1e-12))
        f[3] = sigma
        if g_primary is None:
            f[4] = 1.0
        else:
            gpd = np.sum(np.asarray(g_primary, np.float64).reshape(-1, n) * dv.T, axis=0)
            f[4] = np.where(gd < 0, np.clip(gpd / np.where(gd < 0, gd, -1.0), -4.0, 4.0), 0.0)
        f[5] = clipped.astype(np.float64)
        den = hd * dn
        f[6] = np.log10(np.clip(np.where(den > 0, gn / np.where(den > 0, den, 1.0), 1e6), 1e-6, 1e6))
        f[7] = group / 4.0
    ok = (dn > 0) & (gd < 0) & np.all(np.isfinite(f), axis=0)
    rec = np.zeros((REC_ROWS, n))
    rec[:NF] = f
    rec[NF] = gd
    rec[NF + 1] = np.where(ok, 0.0, -1.0)
    return rec


def step_labels(group, g_after, d, rec, S=1, phi0=None):
    """Fills the label row of pending records: phi1 = g_after . d and phi0 =
    the record's row 8, or the given phi0 (then also written to row 8)."""
    n = rec.shape[1]
    gv = np.asarray(g_after, np.float64).reshape(-1, n)
    dv = np.asarray(d, np.float64).reshape(-1, n)
    out = rec.copy()
    if phi0 is not None:
        out[NF] = phi0
    phi0 = out[NF]
    phi1 = np.sum(gv * dv, axis=0)
    den = phi0 - phi1
    with np.errstate(divide="ignore", invalid="ignore"):
        a = np.where(den < 0, phi0 / np.where(den < 0, den, -1.0), 2.0)
    a = np.where(phi0 >= 0, 0.0, a)
    pend = rec[NF + 1] >= 0
    out[NF + 1] = np.where(pend, np.where(np.isfinite(a), np.clip(a, 0.0, 2.0), -1.0), rec[NF + 1])
    out[NF + 2] = np.where(pend, phi1, 0.0)
    return out


def phi(group, g, d):
    """g . d per Gaussian (any layout of g and d with n last)."""
    n = np.asarray(d).shape[-1]
    return np.sum(np.asarray(g, np.float64).reshape(-1, n) * np.asarray(d, np.float64).reshape(-1, n), axis=0)


def learned_step(group, g, H, d, scene, cfg, p, g_primary=None):
    """alpha d (alpha from the network on the step's record) inside
    learned_trust times the plain step's trust radii (scale bounds with
    k^learned_trust) and the opacity fraction-to-boundary; d where the record
    is unusable."""
    cfg = O.default_config(**(cfg or {}))
    sc = O.scene_handle(scene)
    n, S = sc.n, O.sh_count(sc.sh_degree)
    rec = step_records(group, g, H, d, scene, cfg, g_primary)
    ok = rec[NF + 1] >= 0
    a, _ = mlp_forward(p, np.where(ok[:, None], rec[:NF].T, 0.0))
    ok &= np.isfinite(a)
    a = np.where(ok, a, 1.0)
    scale = np.asarray(sc.scale, np.float64).reshape(3, n)
    sigma = np.asarray(sc.opacity, np.float64).reshape(n)
    d = np.asarray(d, np.float64)
    lt = cfg["learned_trust"]
    if group == O.POS:
        lim = lt * cfg["trust_pos"] * scale.max(0)
        dn = a * np.linalg.norm(d, axis=0)
        m = np.where(dn > lim, a * lim / np.where(dn > 0, dn, 1.0), a)
        out = d * m
    elif group == O.SCALE:
        k = cfg["scale_trust"] ** lt
        out = np.clip(a * d, scale / k - scale, k * scale - scale)
    elif group == O.ROT:
        out = np.clip(a * d, -lt * cfg["trust_rot"], lt * cfg["trust_rot"])
    elif group == O.OPACITY:
        tau = cfg["frac_to_boundary"]
        out = np.clip(a * d.reshape(1, n), -tau * sigma, tau * (1.0 - sigma))
    else:
        dc = d.reshape(3, S, n)
        cn = a * np.linalg.norm(dc, axis=1)                     # (3, n)
        m = np.where(cn > lt * cfg["trust_color"], a * lt * cfg["trust_color"] / np.where(cn > 0, cn, 1.0), a)
        out = dc * m[:, None, :]
    return np.where(ok, out.reshape(d.shape), d)


# ---------------------------------------------------------------- learned damping
DAMP_GROUPS = (O.POS, O.SCALE, O.COLOR)   # damping turns these steps, not only shortens them
RHO_GRID = tuple(10.0 ** (0.5 * j) for j in range(7))   # the damping can only grow


def quad_model(group, g, H, d, S):
    """Q(d) = g . d + 1/2 d^T H d per Gaussian (oracle block layouts)."""
    gv, Hm, dv = _as_vectors(group, g, H, d, S)
    return np.einsum("ni,ni->n", gv, dv) + 0.5 * np.einsum("ni,nij,nj->n", dv, Hm, dv)


def damping_records(group, g, H, rec, scene, primary, g_all, H_all, cfg, return_q=False):
    """The damping network's records: the step records' features (rows 0-7
    of rec), the label 2 log10(rho*) / 3 (row 9), rho* the multiplier of
    damping_mu0 among 10^0, 10^0.5, .., 10^3 (ascending; the first of equal values)
    whose step -- O.solve of the local blocks g, H with mu0 rho -- has the
    smallest Q over the all-view blocks g_all, H_all; -1 where the step record
    is unusable, no candidate has Q < 0, or the group is not in DAMP_GROUPS;
    rows 8 and 10 = -w a*, -w a* + w (w = the largest minus the smallest
    finite Q of the candidates, 0 without a label): the line objective's
    quadratic with its minimum at the label.
    return_q: also the candidates' Q [len(RHO_GRID)][n] (None if no label)."""
    cfg = O.default_config(**(cfg or {}))
    sc = O.scene_handle(scene)
    n, S = sc.n, O.sh_count(sc.sh_degree)
    out = np.zeros((REC_ROWS, n))
    out[:NF] = rec[:NF]
    out[NF + 1] = -1.0
    if group not in DAMP_GROUPS or cfg["gd_lr"][group] > 0:
        return (out, None) if return_q else out
    best_q = np.full(n, np.inf)
    best_rho = np.ones(n)
    qs = []
    for rho in RHO_GRID:
        cj = dict(cfg, damping_mu0=cfg["damping_mu0"] * rho)
        d = O.solve(group, sc, primary, g, H, cj)["step"]
        q = quad_model(group, g_all, H_all, d, S)
        q = np.where(np.isfinite(q), q, np.inf)
        qs.append(q)
        better = q < best_q
        best_q = np.where(better, q, best_q)
        best_rho = np.where(better, rho, best_rho)
    ok = (rec[NF + 1] >= 0) & (best_q < 0)
    lab = np.clip(np.log10(best_rho) * (2.0 / 3.0), 0.0, 2.0)
    out[NF + 1] = np.where(ok, lab, -1.0)
    # rows 8 and 10: the label as the line objective's quadratic, weighted by
    # the spread w of the candidates' finite Q
    Q = np.stack(qs)
    worst = np.max(np.where(np.isfinite(Q), Q, -np.inf), axis=0)
    w = np.where(ok, np.maximum(worst - best_q, 0.0), 0.0)
    out[NF] = -w * np.where(ok, lab, 0.0)
    out[NF + 2] = out[NF] + w
    return (out, Q) if return_q else out


def damped_step(group, g, H, d, scene, primary, cfg, p_damp, g_primary=None):
    """The learned-damping step: rho = 10^(1.5 alpha) from the network
    p_damp on the plain step d's record (1 where the record is unusable or
    the group is not in DAMP_GROUPS), then O.solve with damping_mu0 rho per
    Gaussian (one solve per Gaussian's own multiplier)."""
    cfg = O.default_config(**(cfg or {}))
    sc = O.scene_handle(scene)
    n = sc.n
    d = np.asarray(d, np.float64)
    if group not in DAMP_GROUPS:
        return d.copy(), np.ones(n)
    rec = step_records(group, g, H, d, sc, cfg, g_primary)
    ok = rec[NF + 1] >= 0
    a, _ = mlp_forward(p_damp, np.where(ok[:, None], rec[:NF].T, 0.0))
    rho = np.where(ok & np.isfinite(a), 10.0 ** (1.5 * a), 1.0)
    out = np.zeros_like(d)
    for r in np.unique(rho):
        cj = dict(cfg, damping_mu0=cfg["damping_mu0"] * r)
        st = O.solve(group, sc, primary, g, H, cj)["step"]
        sel = rho == r
        out[..., sel] = st[..., sel]
    return out, rho


# ---------------------------------------------------------------- logged sweep
def _views(cams, targets, knn_table, t, cfg):
    K, f = cfg["knn_k"], cfg["downsample"]
    out = [(cams[t], np.asarray(targets[t], np.float64))]
    for q in range(K):
        v = int(knn_table[t][q])
        if v < 0:
            continue
        cam, tgt = cams[v], np.asarray(targets[v], np.float64)
        if f > 1:
            cam, tgt = O.downsample_camera(cam, f), O.downsample_image(tgt, f)
        out.append((cam, tgt))
    return out


def _blocks(group, scene, views, primary, cfg):
    ob = None
    for cam, tgt in views:
        r = O.render(scene, cam, cfg)
        L = O.loss(r["image"], tgt, cfg)
        ob = O.accum(group, scene, cam, primary, L["e"], L["h"], cfg, out=ob)
    return ob


def sweep_logged(scene, cams, targets, knn_table, t, cfg, damping=False):
    """The oracle's sweep (same order as O.sweep) logging every group's
    records; labels from the loss over every training view at full
    resolution.  Returns (scene handle, records [5][REC_ROWS][n]) and, with
    damping, the damping records [5][REC_ROWS][n] third (damping == "q": a
    list of damping_records(..., return_q=True) pairs instead)."""
    cfg = O.default_config(**(cfg or {}))
    cur = O.scene_handle(scene)
    views = _views(cams, targets, knn_table, t, cfg)
    every = [(c, np.asarray(targets[v], np.float64)) for v, c in enumerate(cams)]
    primary = cams[t]
    S = O.sh_count(cur.sh_degree)
    recs, drecs = [], []
    for group in O.GROUPS:
        ob = _blocks(group, cur, views, primary, cfg)
        gp = _blocks(group, cur, views[:1], primary, cfg)["g"]
        st = O.solve(group, cur, primary, ob["g"], ob["H"], cfg)
        d = st["step"]
        rec = step_records(group, ob["g"], ob["H"], d, cur, cfg, gp)
        ball = _blocks(group, cur, every, primary, cfg)
        phi0 = phi(group, ball["g"], d)
        if damping:
            drecs.append(damping_records(group, ob["g"], ob["H"], rec, cur, primary, ball["g"], ball["H"], cfg,
                                         return_q=damping == "q"))
        nxt = O.apply(group, cur, primary, d, cfg)
        g_after = _blocks(group, nxt, every, primary, cfg)["g"]
        recs.append(step_labels(group, g_after, d, rec, S, phi0=phi0))
        cur = nxt
    if damping:
        return cur, np.stack(recs), (drecs if damping == "q" else np.stack(drecs))
    return cur, np.stack(recs)

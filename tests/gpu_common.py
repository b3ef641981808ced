"""Shared helpers of the GPU parity tests: one configuration given to both the
CUDA path and the oracle (the oracle receives the FP32-rounded values, so
every threshold is the same number on both sides), and comparison helpers."""
import numpy as np

GPU_CFG_KEYS = ("lambda_ssim", "alpha_min", "alpha_max", "t_min", "lowpass", "near_z", "barrier_alpha",
                "frac_to_boundary", "damping_mu0", "damping_tries", "scale_min", "scale_trust", "trust_pos",
                "trust_rot", "trust_color", "ssim_c1",
                "ssim_c2", "ssim_sigma", "ssim_radius", "knn_k", "downsample", "gauss_newton", "group_order",
                "group_jacobi", "gd_lr", "learned_trust")


def oracle_cfg(gpu_cfg: dict) -> dict:
    out = {}
    for k in GPU_CFG_KEYS:
        v = gpu_cfg[k]
        if k == "group_order":
            out[k] = [int(x) for x in v]
        elif k == "gd_lr":
            out[k] = [float(np.float32(x)) for x in v]
        else:
            out[k] = int(v) if isinstance(v, (int, np.integer)) and not isinstance(v, bool) else float(np.float32(v))
    return out


def rel_err(got, want, scale):
    """max |got - want| / scale (scale: array broadcastable to the entries or a scalar)."""
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    return float(np.max(np.abs(got - want) / scale)) if got.size else 0.0


def ambiguous_gaussians(O, scene, cam, cfg, margin, thresh=1e-4, dilate=0):
    """Gaussians that contribute (alpha >= alpha_min) to a pixel whose compositing
    decisions are within `thresh` (relative) of a threshold in the oracle. Such
    decisions may go either way between FP32 and FP64; what depends on them is
    excluded from element-wise comparison and counted."""
    bad = margin < thresh
    if dilate:
        from scipy.ndimage import binary_dilation
        bad = binary_dilation(bad, iterations=dilate)
    if not bad.any():
        return np.zeros(scene.n, bool), bad
    pr = O.project(scene, cam, cfg)
    ys, xs = np.nonzero(bad)
    amb = np.zeros(scene.n, bool)
    vis = ~pr["culled"]
    for y, x in zip(ys, xs):
        dx = x - pr["pix"][0]
        dy = y - pr["pix"][1]
        q = pr["conic"][0] * dx * dx + 2 * pr["conic"][1] * dx * dy + pr["conic"][2] * dy * dy
        a = pr["opacity"] * np.exp(-0.5 * q)
        amb |= vis & (a >= 0.5 * cfg["alpha_min"])
    return amb, bad


def _sym_full(Hp, D):
    H = np.zeros((D, D))
    iu = np.triu_indices(D)
    H[iu] = Hp
    H[(iu[1], iu[0])] = Hp
    return H


def _ladder_ambiguous(Hr, mu0, tries, mu_acc, eps_of):
    """True if a damping decision up to the accepted one could go the other
    way under the block perturbation: at attempt i the damped block is
    A_i = H_r + mu_i m I (mu_i = mu0 10^i, m = mean |diag H_r|) and Weyl's
    inequality moves its smallest eigenvalue by at most eps_of(mu_i).  A 1x1
    block is the exception: h + mu |h| is exactly 0 for h < 0 at mu = 1 in any
    arithmetic, so only the sign of h (|h| <= eps_of(0)) is in doubt."""
    D = Hr.shape[0]
    if D == 1:
        return abs(Hr[0, 0]) <= eps_of(0.0)
    m = np.abs(np.diag(Hr)).mean()
    mu = mu0
    for _ in range(tries + 1):
        A = Hr + mu * m * np.eye(D)
        lam = np.linalg.eigvalsh(A)
        if abs(lam[0]) <= eps_of(mu) + 1e-5 * np.abs(lam).max():
            return True
        if mu >= mu_acc * (1 - 1e-12):
            return False
        mu *= 10
    return False


def step_bound_check(O, group, scene, primary, ob, os_, got, cfg, S, amb, gtol=1e-4, htol=1e-3):
    """Compares a GPU step with the oracle's step of the same blocks' problem.

    The GPU's blocks are within gtol / htol of the oracle's, entry by entry,
    relative to the oracle's sum of absolute per-pixel terms (floored at 1e-6 of
    the largest): |dg| <= gtol gs, |dH| <= htol Hs.  For the damped reduced
    system A x = -g_r (A = B^T H B + mu m I, m = mean |diag B^T H B|, B the
    group's basis: U for position, Q for scaling, the identity otherwise) the
    first-order perturbation is
        |dx| <= |A^-1| |B| (|dg| + (1 + mu) |B| |dH| |x_u|),
    x_u the unclipped step; trust radii, the scale box and the opacity
    fraction-to-boundary are projections (1-Lipschitz), so the bound holds for
    the clipped steps too.  FP32 solve rounding adds 1e-3 |x| (scaling also
    1e-6 cond(Q^T Q) |Q| |x_u| for FP32 rounding of its basis).
    Excluded and counted: Gaussians touched by an ambiguous compositing
    decision (amb); blocks whose damping decision could flip under the same
    perturbation (_ladder_ambiguous); blocks the oracle could not solve (no
    contribution, failed ladder, undefined scaling reduction) and scaling
    reductions within 1e-3 of degenerate (the basis itself is then not
    determined by FP32 inputs).

    got: the GPU step in the library's layout.  Returns dict(checked,
    excluded, contributors, worst = max err / bound, fails, mask = the checked
    Gaussians)."""
    n = scene.mean.shape[1]
    contrib = ob["npix"] > 0
    gs_all = np.maximum(ob["gabs"], 1e-6 * ob["gabs"].max())
    hs_all = np.maximum(ob["Habs"], 1e-6 * ob["Habs"].max())
    if group in (O.POS, O.SCALE):
        Bas, bst, gap = O.reduced_basis(group, scene, primary, cfg)
    mu0, tries = cfg["damping_mu0"], cfg["damping_tries"]
    checked, excluded, worst = 0, 0, 0.0
    fails = []
    mask = np.zeros(n, bool)
    for k in np.nonzero(contrib)[0]:
        if amb[k] or (group == O.SCALE and (bst[k] != 0 or gap[k] < 1e-3)):
            excluded += 1
            continue
        chans = range(3) if group == O.COLOR else [None]
        skip = False
        items = []
        for ch in chans:
            if group == O.COLOR:
                st, mu = os_["status"][ch, k], os_["info"][ch, 0, k]
            else:
                st, mu = os_["status"][k], os_["info"][0, k]
            if st != 0:
                skip = True
                break
            if group == O.COLOR:
                Hf = _sym_full(ob["H"][ch, :, k], S)
                gv = ob["g"][ch, :, k]
                dg = gtol * np.linalg.norm(gs_all[ch, :, k])
                dH = htol * np.linalg.norm(_sym_full(hs_all[ch, :, k], S))
                B = np.eye(S)
                x = os_["step"][ch, :, k]
                y = got[ch * S * n + k: (ch * S + S) * n + k: n]
            elif group in (O.POS, O.SCALE):
                Hf = _sym_full(ob["H"][:, k], 3)
                gv = ob["g"][:, k]
                dg = gtol * np.linalg.norm(gs_all[:, k])
                dH = htol * np.linalg.norm(_sym_full(hs_all[:, k], 3))
                B = Bas[k]
                x = os_["step"][:, k]
                y = got[k::n][:3]
            else:
                Hf = ob["H"][:, k].reshape(1, 1).copy()
                gv = ob["g"][:, k].copy()
                if group == O.OPACITY:
                    sg = float(scene.opacity[k])
                    a = cfg["barrier_alpha"]
                    gv = gv + a * (-1 / sg + 1 / (1 - sg))
                    Hf = Hf + a * (1 / sg ** 2 + 1 / (1 - sg) ** 2)
                dg = gtol * gs_all[0, k]
                dH = htol * hs_all[0, k]
                B = np.eye(1)
                x = os_["step"][:, k]
                y = got[k:k + 1]
            Hr = B.T @ Hf @ B
            gr = B.T @ gv
            nB = np.linalg.norm(B, 2)
            if _ladder_ambiguous(Hr, mu0, tries, mu, lambda m_: (1 + m_) * nB * nB * dH):
                skip = True
                break
            m = np.abs(np.diag(Hr)).mean()
            A = Hr + mu * m * np.eye(Hr.shape[0])
            xu = -np.linalg.solve(A, gr)
            inv = np.linalg.norm(np.linalg.inv(A), 2)
            bound = nB * inv * nB * (dg + (1 + mu) * nB * dH * np.linalg.norm(xu))
            bound += 1e-3 * np.linalg.norm(x)
            if group == O.SCALE:
                bound += 1e-6 * np.linalg.cond(B.T @ B) * nB * np.linalg.norm(xu)
            if group == O.OPACITY:
                bound += 1e-6
            items.append((np.linalg.norm(y - x), bound, ch))
        if skip:
            excluded += 1
            continue
        for err, bound, ch in items:
            worst = max(worst, err / bound if bound > 0 else (np.inf if err > 0 else 0.0))
            if err > bound:
                fails.append((int(k), ch, float(err), float(bound)))
        checked += 1
        mask[k] = True
    return dict(checked=checked, excluded=excluded, contributors=int(contrib.sum()), worst=worst, fails=fails,
                mask=mask)

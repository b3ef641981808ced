"""Shared helpers of the GPU parity tests: one configuration given to both the
CUDA path and the oracle (the oracle receives the FP32-rounded values, so
every threshold is the same number on both sides), and comparison helpers."""
import numpy as np

GPU_CFG_KEYS = ("lambda_ssim", "alpha_min", "alpha_max", "t_min", "lowpass", "near_z", "barrier_alpha",
                "frac_to_boundary", "damping_mu0", "damping_tries", "scale_min", "scale_trust", "trust_pos",
                "trust_rot", "trust_color", "ssim_c1",
                "ssim_c2", "ssim_sigma", "ssim_radius", "knn_k", "downsample", "gauss_newton", "group_order",
                "group_jacobi", "gd_lr")


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

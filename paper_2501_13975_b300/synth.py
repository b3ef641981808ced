"""Seeded synthetic inputs: Gaussian scenes and camera poses.

This module is shared by the oracle tests, the GPU tests and bench.py. It
holds none of the method's arithmetic: it only draws random parameters with
numpy's PCG64 and builds camera poses. Everything is FP32 (the GPU path's
storage precision); the oracle converts exactly to FP64.

Workloads (shapes follow the paper's experiments, whose datasets are not
available; see the scene functions for the recipes):
  tiny    1,000 Gaussians in [-1,1]^3, SH degree 0, 4 cameras 128x128 on a ring
  object  100k Gaussians on a unit-sphere shell, SH degree 3, 100 cameras
          800x800 on a Fibonacci hemisphere of radius 4
  scene   1M Gaussians spread log-uniformly to radius 50, SH degree 3, 200
          cameras 1600x1040 along a smooth closed trajectory
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# DC coefficients are drawn uniform on [0, 2*sqrt(pi)] so that the rendered
# DC colour (basis value 1/(2*sqrt(pi))) is uniform on [0, 1].
DC_RANGE = 2.0 * math.sqrt(math.pi)


@dataclasses.dataclass
class Scene:
    mean: np.ndarray      # (3, n) float32
    quat: np.ndarray      # (4, n) float32, unit, (w, x, y, z)
    scale: np.ndarray     # (3, n) float32, linear
    opacity: np.ndarray   # (n,) float32 in (0, 1)
    sh: np.ndarray        # (3, S, n) float32
    sh_degree: int

    @property
    def n(self) -> int:
        return int(self.mean.shape[1])

    def copy(self) -> "Scene":
        return Scene(self.mean.copy(), self.quat.copy(), self.scale.copy(), self.opacity.copy(),
                     self.sh.copy(), self.sh_degree)


@dataclasses.dataclass
class Camera:
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    viewmat: np.ndarray   # (3, 4) float32 row-major [R | t], world -> camera, +z forward, y down
    clip_x: float = 0.0   # frustum clamp limits (0: derived from this image's size)
    clip_y: float = 0.0

    def center(self) -> np.ndarray:
        R = self.viewmat[:, :3].astype(np.float64)
        t = self.viewmat[:, 3].astype(np.float64)
        return -R.T @ t


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def _unit_quats(rng, n):
    q = rng.standard_normal((4, n))
    q /= np.linalg.norm(q, axis=0, keepdims=True)
    return q.astype(np.float32)


def _sh_coeffs(rng, n, degree, higher_std=0.1):
    S = (degree + 1) ** 2
    sh = np.zeros((3, S, n), np.float32)
    sh[:, 0, :] = rng.uniform(0.0, DC_RANGE, (3, n))
    if S > 1:
        sh[:, 1:, :] = rng.normal(0.0, higher_std, (3, S - 1, n))
    return sh


def look_at(eye, target, up=(0.0, 1.0, 0.0)) -> np.ndarray:
    """World->camera [R|t] (3x4, float32) for a camera at eye looking at target,
    +z forward, y down, x right (right-handed)."""
    eye = np.asarray(eye, np.float64)
    z = np.asarray(target, np.float64) - eye
    z /= np.linalg.norm(z)
    up = np.asarray(up, np.float64)
    if abs(float(np.dot(z, up / np.linalg.norm(up)))) > 0.99:
        up = np.array([0.0, 0.0, 1.0])
    down = -up / np.linalg.norm(up)
    x = np.cross(down, z)
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    R = np.stack([x, y, z])
    t = -R @ eye
    return np.concatenate([R, t[:, None]], axis=1).astype(np.float32)


def pinhole(width, height, fov_x_deg, viewmat) -> Camera:
    fx = 0.5 * width / math.tan(math.radians(fov_x_deg) / 2.0)
    return Camera(int(width), int(height), float(np.float32(fx)), float(np.float32(fx)),
                  float((width - 1) / 2.0), float((height - 1) / 2.0), viewmat)


# ----------------------------------------------------------------------------- tiny

def tiny_scene(seed: int = 1, n: int = 1000, sh_degree: int = 0, log_scale=(-3.0, 0.3)) -> Scene:
    """Means U[-1,1]^3, log-scales N(mu, sd), random unit quaternions,
    opacity sigmoid(N(0,1)), DC colour uniform."""
    rng = _rng(seed)
    mean = rng.uniform(-1.0, 1.0, (3, n)).astype(np.float32)
    scale = np.exp(rng.normal(log_scale[0], log_scale[1], (3, n))).astype(np.float32)
    quat = _unit_quats(rng, n)
    opacity = _sigmoid(rng.standard_normal(n)).astype(np.float32)
    sh = _sh_coeffs(rng, n, sh_degree)
    return Scene(mean, quat, scale, opacity, sh, sh_degree)


def ring_cameras(count: int = 4, size: int = 128, radius: float = 3.0, fov: float = 60.0, height=None):
    h = size if height is None else height
    cams = []
    for i in range(count):
        phi = 2.0 * math.pi * i / count
        eye = (radius * math.cos(phi), 0.0, radius * math.sin(phi))
        cams.append(pinhole(size, h, fov, look_at(eye, (0.0, 0.0, 0.0))))
    return cams


def perturbed(scene: Scene, seed: int = 2, sd: float = 0.02) -> Scene:
    """Copy with means + N(0, sd^2) (the scene the targets are rendered from)."""
    rng = _rng(seed)
    s = scene.copy()
    s.mean = (s.mean + rng.normal(0.0, sd, s.mean.shape)).astype(np.float32)
    return s


def initialised(scene: Scene, seed: int = 9, opacity: float = 0.1, scale_sd: float = 0.3) -> Scene:
    """Copy in the state a 3DGS training run starts from: grey DC colour
    (rendered 0.5), higher SH bands 0, every opacity `opacity`, scales
    multiplied by exp(N(0, scale_sd^2)); means and rotations kept."""
    rng = _rng(seed)
    s = scene.copy()
    sh = np.zeros_like(s.sh)
    sh[:, 0, :] = 0.5 * DC_RANGE
    s.sh = sh.astype(np.float32)
    s.opacity = np.full_like(s.opacity, opacity)
    s.scale = (s.scale * np.exp(rng.normal(0.0, scale_sd, s.scale.shape))).astype(np.float32)
    return s


# ----------------------------------------------------------------------------- object

def object_scene(seed: int = 3, n: int = 100_000, sh_degree: int = 3) -> Scene:
    """Shell of radius U[0.9, 1.0] with uniform directions; log-scales N(-3, 0.3);
    SH degree 3: DC uniform, higher bands N(0, 0.1)."""
    rng = _rng(seed)
    d = rng.standard_normal((3, n))
    d /= np.linalg.norm(d, axis=0, keepdims=True)
    r = rng.uniform(0.9, 1.0, n)
    mean = (d * r).astype(np.float32)
    scale = np.exp(rng.normal(-3.0, 0.3, (3, n))).astype(np.float32)
    quat = _unit_quats(rng, n)
    opacity = _sigmoid(rng.standard_normal(n)).astype(np.float32)
    sh = _sh_coeffs(rng, n, sh_degree)
    return Scene(mean, quat, scale, opacity, sh, sh_degree)


def hemisphere_cameras(count: int = 100, size: int = 800, radius: float = 4.0, fov: float = 60.0,
                       height: int | None = None):
    """Fibonacci points on the upper hemisphere, looking at the origin; images
    size x size (size x height when height is given, fov horizontal)."""
    golden = math.pi * (3.0 - math.sqrt(5.0))
    cams = []
    for i in range(count):
        y = (i + 0.5) / count
        rr = math.sqrt(max(0.0, 1.0 - y * y))
        phi = golden * i
        eye = (radius * rr * math.cos(phi), radius * y, radius * rr * math.sin(phi))
        cams.append(pinhole(size, height or size, fov, look_at(eye, (0.0, 0.0, 0.0))))
    return cams


# ----------------------------------------------------------------------------- scene

def spread_scene(seed: int = 6, n: int = 1_000_000, sh_degree: int = 3, r_min: float = 0.5,
                 r_max: float = 50.0) -> Scene:
    """Uniform directions, radius log-uniform in [r_min, r_max]; log-scales
    N(-2.5, 0.5); SH degree 3."""
    rng = _rng(seed)
    d = rng.standard_normal((3, n))
    d /= np.linalg.norm(d, axis=0, keepdims=True)
    r = np.exp(rng.uniform(math.log(r_min), math.log(r_max), n))
    mean = (d * r).astype(np.float32)
    scale = np.exp(rng.normal(-2.5, 0.5, (3, n))).astype(np.float32)
    quat = _unit_quats(rng, n)
    opacity = _sigmoid(rng.standard_normal(n)).astype(np.float32)
    sh = _sh_coeffs(rng, n, sh_degree)
    return Scene(mean, quat, scale, opacity, sh, sh_degree)


def trajectory_cameras(count: int = 200, width: int = 1600, height: int = 1040, fov: float = 60.0,
                       seed: int = 7):
    """centre(t) = (20 + 5 sin(2 pi t + p1)) (cos 2 pi t, 0.2 sin(4 pi t + p2), sin 2 pi t),
    looking at 0.3 centre(t + 0.05)."""
    rng = _rng(seed)
    p1, p2 = rng.uniform(0.0, 2.0 * math.pi, 2)

    def centre(t):
        a = 20.0 + 5.0 * math.sin(2.0 * math.pi * t + p1)
        return np.array([a * math.cos(2 * math.pi * t), a * 0.2 * math.sin(4 * math.pi * t + p2),
                         a * math.sin(2 * math.pi * t)])

    cams = []
    for i in range(count):
        t = i / count
        cams.append(pinhole(width, height, fov, look_at(centre(t), 0.3 * centre(t + 0.05))))
    return cams


BATCH_RESOLUTIONS = ((512, 512), (640, 480), (800, 600), (1024, 768))


def batched_workload(seed: int = 8, count: int = 16, n_min: int = 20_000, n_max: int = 500_000,
                     views_min: int = 16, views_max: int = 128):
    """Independent scenes for the batched form: Gaussian counts log-uniform in
    [n_min, n_max], view counts uniform in [views_min, views_max], resolution
    uniform from BATCH_RESOLUTIONS, SH degree 3; even entries are shells
    (object_scene, hemisphere cameras), odd ones spread scenes
    (spread_scene, trajectory cameras).  Returns a list of dicts with the
    ground-truth scene, the training start (means + N(0, 0.02^2)) and the
    cameras."""
    rng = _rng(seed)
    out = []
    for i in range(count):
        n = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        views = int(rng.integers(views_min, views_max + 1))
        w, h = BATCH_RESOLUTIONS[int(rng.integers(len(BATCH_RESOLUTIONS)))]
        s = int(rng.integers(1 << 30))
        if i % 2 == 0:
            gt = object_scene(seed=s, n=n)
            cams = hemisphere_cameras(views, w, height=h)
            kind = "shell"
        else:
            gt = spread_scene(seed=s, n=n)
            cams = trajectory_cameras(views, w, h, seed=s + 1)
            kind = "spread"
        out.append(dict(kind=kind, n=n, views=views, width=w, height=h, gt=gt,
                        train=perturbed(gt, seed=s + 2, sd=0.02), cams=cams))
    return out


def procedural_targets(count: int, width: int, height: int, seed: int = 11) -> np.ndarray:
    """Smooth random images in [0, 1], (count, 3, H, W) float32: a sum of a few
    random low-frequency cosines per channel (used where no reference render
    is wanted, e.g. timing inputs)."""
    rng = _rng(seed)
    yy, xx = np.meshgrid(np.arange(height, dtype=np.float32), np.arange(width, dtype=np.float32),
                         indexing="ij")
    out = np.empty((count, 3, height, width), np.float32)
    for i in range(count):
        for c in range(3):
            acc = np.full((height, width), 0.5, np.float32)
            for _ in range(4):
                kx, ky = rng.uniform(-0.05, 0.05, 2)
                ph = rng.uniform(0, 2 * math.pi)
                acc += np.float32(0.12) * np.cos(kx * xx + ky * yy + ph).astype(np.float32)
            out[i, c] = np.clip(acc, 0.0, 1.0)
    return out


def mlp_init(seed: int = 20, nfeat: int = 8, hidden: int = 64, out_scale: float = 0.1):
    """Initial parameters of the 8-64-64-1 step-scale network, packed as
    W1 [64][8], b1 [64], W2 [64][64], b2 [64], W3 [64], b3: W1, W2 normal with
    variance 2 / fan-in, W3 the same times out_scale, biases 0 (the output
    then starts near y = 0, alpha = 1: the plain step).  Values are truncated
    to BF16-representable FP32 numbers, so the FP32 master copy and the BF16
    copy hold the same values.  Returns (master float32 [P], bits uint16 [P])."""
    rng = _rng(seed)
    w1 = rng.normal(0.0, math.sqrt(2.0 / nfeat), hidden * nfeat)
    w2 = rng.normal(0.0, math.sqrt(2.0 / hidden), hidden * hidden)
    w3 = rng.normal(0.0, out_scale * math.sqrt(2.0 / hidden), hidden)
    p = np.concatenate([w1, np.zeros(hidden), w2, np.zeros(hidden), w3, np.zeros(1)]).astype(np.float32)
    bits = (p.view(np.uint32) >> np.uint32(16)).astype(np.uint16)
    master = (bits.astype(np.uint32) << np.uint32(16)).view(np.float32)
    return master, bits

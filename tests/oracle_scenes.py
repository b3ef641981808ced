"""Small hand-made scenes for the oracle pins (inputs only, no method arithmetic)."""
import numpy as np

from paper_2501_13975_b300 import synth

# every threshold of the rasteriser switched off: the rendered image is then a
# smooth function of all parameters, so finite differences are meaningful
NOTHRESH = dict(alpha_min=0.0, alpha_max=1.0, t_min=0.0)


def micro_scene(n, seed, sh_degree=0, z=(3.0, 5.0)):
    rng = np.random.default_rng(seed)
    mean = np.stack([rng.uniform(-0.4, 0.4, n), rng.uniform(-0.3, 0.3, n), rng.uniform(z[0], z[1], n)])
    scale = rng.uniform(0.08, 0.25, (3, n))
    q = rng.standard_normal((4, n))
    q /= np.linalg.norm(q, axis=0)
    op = rng.uniform(0.3, 0.8, n)
    S = (sh_degree + 1) ** 2
    sh = np.zeros((3, S, n))
    sh[:, 0] = rng.uniform(0.5, 3.0, (3, n))
    if S > 1:
        sh[:, 1:] = rng.normal(0.0, 0.3, (3, S - 1, n))
    f = np.float32
    return synth.Scene(mean.astype(f), q.astype(f), scale.astype(f), op.astype(f), sh.astype(f), sh_degree)


def micro_camera(eye=(0.0, 0.0, 0.0), target=(0.0, 0.0, 4.0), W=48, H=40, f=40.0):
    return synth.Camera(W, H, f, f, (W - 1) / 2.0, (H - 1) / 2.0, synth.look_at(eye, target))

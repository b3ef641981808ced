"""Learned step scale: logging, training and installation (host driver).

The arithmetic runs in the library's kernels (gs2_sweep_logged,
gs2_mlp_grad, gs2_mlp_adam, gs2_mlp_forward and the inference kernel inside
gs2_solve_step); this module only chooses scenes, batches and the order of
the calls.  See include/gs2.h for the record format and the features.

    recs = collect_records(range(100, 2100))       # tiny-scene runs, one sweep each
    model = StepModel(seed=20)
    model.fit(recs, epochs=3)
    ctx.set_step_model(model.w)                    # every later solve uses it

The damping network is a StepModel trained on the damping records (labels
objective) and installed with ctx.set_damping_model.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import gs2, synth


class RecordSet:
    """Records on the device: chunks [REC_ROWS][chunk_n] back to back."""

    def __init__(self, data: torch.Tensor, chunk_n: int):
        assert data.is_cuda and data.dtype == torch.float32
        self.data = data.contiguous()
        self.chunk_n = int(chunk_n)
        self.n = self.data.numel() // gs2.REC_ROWS
        self._scale = None

    def chunk_scale(self) -> torch.Tensor:
        """Per-chunk scale of the line-model loss (computed once, on the device)."""
        if self._scale is None:
            self._scale = gs2.records_chunk_scale(self.data, self.chunk_n, self.n // self.chunk_n)
        return self._scale

    def labels(self) -> torch.Tensor:
        return self.data.view(-1, gs2.REC_ROWS, self.chunk_n)[:, gs2.MLP_NFEAT + 1, :].reshape(-1)

    def split(self, frac: float):
        """First (1 - frac) of the chunks and the rest (held-out runs)."""
        chunks = self.data.view(-1, gs2.REC_ROWS * self.chunk_n)
        k = max(1, int(round(chunks.shape[0] * (1.0 - frac))))
        return (RecordSet(chunks[:k].reshape(-1), self.chunk_n),
                RecordSet(chunks[k:].reshape(-1), self.chunk_n))


def collect_records(seeds, kind: str = "tiny", sweeps: int = 1, n: int | None = None, size: int | None = None,
                    ncam: int | None = None, sd: float = 0.02, ctx=None, stream=None, damping: bool = False):
    """Records of the plain method, `sweeps` logged sweeps per seed.

    kind "tiny": n (1000) Gaussians in [-1,1]^3, SH degree 0, 4 ring cameras
      size x size (128); training starts from the scene, targets come from a
      copy whose means moved by N(0, sd^2).
    kind "shell": n (20k) Gaussians on a unit-sphere shell, SH degree 3, ncam
      (32) hemisphere cameras size x size (256); targets from the scene,
      training starts from a copy with means moved by N(0, sd^2), every second
      seed in the initialised state (grey colour, opacity 0.1, jittered
      scales).
    Primaries: a seeded permutation of the cameras per seed.
    damping: also the damping network's records; returns (steps, damping)
    RecordSets."""
    seeds = list(seeds)
    if kind == "tiny":
        n, size, ncam, sh = n or 1000, size or 128, 4, 0
    elif kind == "shell":
        n, size, ncam, sh = n or 20_000, size or 256, ncam or 32, 3
    else:
        raise ValueError(kind)
    cams = synth.ring_cameras(4, size) if kind == "tiny" else synth.hemisphere_cameras(ncam, size)
    own = ctx is None
    if own:
        ctx = gs2.Context(n, size, size, sh, 64 * n)
    out = torch.empty((len(seeds), sweeps, 5, gs2.REC_ROWS, n), dtype=torch.float32, device="cuda")
    outd = torch.empty_like(out) if damping else None
    centres = np.stack([c.center() for c in cams]).astype(np.float32)
    proj = ctx.proj_buffer(n)
    for i, s in enumerate(seeds):
        s = int(s)
        if kind == "tiny":
            start = synth.tiny_scene(seed=s, n=n)
            gt = synth.perturbed(start, seed=s + 100_000, sd=sd)
        else:
            gt = synth.object_scene(seed=s, n=n)
            start = synth.perturbed(gt, seed=s + 100_000, sd=sd)
            if i % 2 == 1:
                start = synth.initialised(start, seed=s + 200_000)
        dg = gs2.DeviceScene.from_host(gt)
        targets = []
        for c in cams:
            ctx.project(dg, c, proj, stream=stream)
            img, _ = ctx.raster_fwd(dg, c, proj, stream=stream)
            targets.append(img)
        ds = gs2.DeviceScene.from_host(start)
        sphere = ctx.bounding_sphere(ds, stream=stream).cpu().numpy()
        knn = gs2.camera_knn(centres, sphere, 3)
        order = np.random.Generator(np.random.PCG64(s)).permutation(ncam)
        for j in range(sweeps):
            ctx.sweep_logged(ds, cams, targets, knn, int(order[j % ncam]), records=out[i, j], stream=stream,
                             records_damping=None if outd is None else outd[i, j])
    if own:
        torch.cuda.synchronize()
        ctx.check()
    if damping:
        return RecordSet(out.reshape(-1), n), RecordSet(outd.reshape(-1), n)
    return RecordSet(out.reshape(-1), n)


class StepModel:
    """FP32 master weights, Adam moments and the BF16 copy, on the device."""

    def __init__(self, seed: int = 20, master: np.ndarray | None = None, bits: np.ndarray | None = None):
        if master is None:
            master, bits = synth.mlp_init(seed)
        self.master = torch.tensor(master, dtype=torch.float32, device="cuda")
        self.w = torch.tensor(bits.astype(np.int16), dtype=torch.int16, device="cuda")
        self.m = torch.zeros(gs2.MLP_NPARAM, dtype=torch.float32, device="cuda")
        self.v = torch.zeros_like(self.m)
        self.t = 0
        self.partial = torch.empty((gs2.MLP_GRID, gs2.MLP_NPARAM), dtype=torch.float32, device="cuda")
        self.stats = torch.empty((gs2.MLP_GRID, 2), dtype=torch.float64, device="cuda")

    def loss(self, recs, idx: torch.Tensor | None = None, nrec: int | None = None, objective: str = "labels"):
        """Mean loss over the usable records (of one RecordSet or a list of
        them), and their count.  objective "labels": 1/2 (alpha - alpha*)^2;
        "line": the line model's predicted change of the label loss, scaled
        per chunk (a descent of the plain step scores about -1 per chunk)."""
        sets = [recs] if isinstance(recs, RecordSet) else list(recs)
        tot = np.zeros(2)
        for r in sets:
            m = r.n if nrec is None else nrec
            sc = r.chunk_scale() if objective == "line" else None
            gs2.mlp_grad(self.w, r.data, r.chunk_n, m, self.partial, self.stats, idx=idx, chunk_scale=sc)
            tot += self.stats.sum(0).cpu().numpy()
        return float(tot[0] / max(tot[1], 1.0)), int(tot[1])

    def step(self, recs: RecordSet, idx: torch.Tensor, nrec: int, lr: float, objective: str = "labels"):
        sc = recs.chunk_scale() if objective == "line" else None
        gs2.mlp_grad(self.w, recs.data, recs.chunk_n, nrec, self.partial, self.stats, idx=idx, chunk_scale=sc)
        self.t += 1
        gs2.mlp_adam(self.master, self.w, self.partial, self.stats, self.m, self.v, self.t, lr)

    def fit(self, recs, epochs: int = 3, batch: int = 16384, lr: float = 2e-3, seed: int = 21,
            lr_final: float = 2e-4, objective: str = "labels"):
        """Adam over shuffled mini-batches of one RecordSet or a list of them
        (each batch from one set; per epoch a seeded permutation of every
        set's records and a seeded order of all batches), learning rate
        decayed geometrically from lr to lr_final."""
        sets = [recs] if isinstance(recs, RecordSet) else list(recs)
        rng = np.random.Generator(np.random.PCG64(seed))
        nb = [max(1, math.ceil(r.n / batch)) for r in sets]
        steps = epochs * sum(nb)
        k = 0
        for _ in range(epochs):
            perms = [torch.tensor(rng.permutation(r.n), dtype=torch.int64, device="cuda") for r in sets]
            plan = np.concatenate([np.stack([np.full(m, i), np.arange(m)], 1) for i, m in enumerate(nb)])
            for i, b in plan[rng.permutation(len(plan))]:
                r = sets[i]
                b0 = int(b) * batch
                m = min(batch, r.n - b0)
                self.step(r, perms[i][b0:b0 + m], m, lr * (lr_final / lr) ** (k / max(steps - 1, 1)), objective)
                k += 1
        return self

    def predict(self, recs: RecordSet) -> torch.Tensor:
        return gs2.mlp_forward(self.w, recs.data, recs.chunk_n, recs.n)


def plain_loss(recs, objective: str = "labels"):
    """The plain step's (alpha = 1) loss against the records: the reference a
    trained network must beat; computed by the same loss kernel with the
    all-zero network (y = 0, alpha = 1)."""
    zero = np.zeros(gs2.MLP_NPARAM, np.float32)
    return StepModel(master=zero, bits=np.zeros(gs2.MLP_NPARAM, np.uint16)).loss(recs, objective=objective)

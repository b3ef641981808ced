"""Learned step scale: logging, training and installation (host driver).

The arithmetic runs in the library's kernels (gs2_sweep_logged,
gs2_mlp_grad, gs2_mlp_adam, gs2_mlp_forward and the inference kernel inside
gs2_solve_step); this module only chooses scenes, batches and the order of
the calls.  See include/gs2.h for the record format and the features.

    recs = collect_records(range(100, 2100))       # tiny-scene runs, one sweep each
    model = StepModel(seed=20)
    model.fit(recs, epochs=3)
    ctx.set_step_model(model.w)                    # every later solve uses it
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

    def labels(self) -> torch.Tensor:
        return self.data.view(-1, gs2.REC_ROWS, self.chunk_n)[:, gs2.MLP_NFEAT + 1, :].reshape(-1)

    def split(self, frac: float):
        """First (1 - frac) of the chunks and the rest (held-out runs)."""
        chunks = self.data.view(-1, gs2.REC_ROWS * self.chunk_n)
        k = max(1, int(round(chunks.shape[0] * (1.0 - frac))))
        return (RecordSet(chunks[:k].reshape(-1), self.chunk_n),
                RecordSet(chunks[k:].reshape(-1), self.chunk_n))


def collect_records(seeds, n: int = 1000, size: int = 128, sd: float = 0.02, ctx=None,
                    stream=None) -> RecordSet:
    """One logged sweep per seed on a tiny scene (n Gaussians in [-1,1]^3,
    SH degree 0, 4 ring cameras size x size; targets rendered from a copy
    whose means moved by N(0, sd^2)); primary view seed mod 4."""
    seeds = list(seeds)
    cams = synth.ring_cameras(4, size)
    own = ctx is None
    if own:
        ctx = gs2.Context(n, size, size, 0)
    out = torch.empty((len(seeds), 5, gs2.REC_ROWS, n), dtype=torch.float32, device="cuda")
    centres = np.stack([c.center() for c in cams]).astype(np.float32)
    for i, s in enumerate(seeds):
        sc = synth.tiny_scene(seed=int(s), n=n)
        gt = synth.perturbed(sc, seed=int(s) + 100_000, sd=sd)
        dg = gs2.DeviceScene.from_host(gt)
        targets = []
        for c in cams:
            proj = ctx.project(dg, c, stream=stream)
            img, _ = ctx.raster_fwd(dg, c, proj, stream=stream)
            targets.append(img)
        ds = gs2.DeviceScene.from_host(sc)
        sphere = ctx.bounding_sphere(ds, stream=stream).cpu().numpy()
        knn = gs2.camera_knn(centres, sphere, 3)
        ctx.sweep_logged(ds, cams, targets, knn, int(s) % 4, records=out[i], stream=stream)
    if own:
        torch.cuda.synchronize()
        ctx.check()
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

    def loss(self, recs: RecordSet, idx: torch.Tensor | None = None, nrec: int | None = None):
        """Mean of 1/2 (alpha - alpha*)^2 over the usable records, and their count."""
        nrec = recs.n if nrec is None else nrec
        gs2.mlp_grad(self.w, recs.data, recs.chunk_n, nrec, self.partial, self.stats, idx=idx)
        s = self.stats.sum(0).cpu().numpy()
        return float(s[0] / max(s[1], 1.0)), int(s[1])

    def step(self, recs: RecordSet, idx: torch.Tensor, nrec: int, lr: float):
        gs2.mlp_grad(self.w, recs.data, recs.chunk_n, nrec, self.partial, self.stats, idx=idx)
        self.t += 1
        gs2.mlp_adam(self.master, self.w, self.partial, self.stats, self.m, self.v, self.t, lr)

    def fit(self, recs: RecordSet, epochs: int = 3, batch: int = 16384, lr: float = 2e-3, seed: int = 21,
            lr_final: float = 2e-4):
        """Adam over shuffled mini-batches (seeded permutation per epoch),
        learning rate decayed geometrically from lr to lr_final."""
        rng = np.random.Generator(np.random.PCG64(seed))
        steps = epochs * max(1, math.ceil(recs.n / batch))
        k = 0
        for _ in range(epochs):
            perm = torch.tensor(rng.permutation(recs.n), dtype=torch.int64, device="cuda")
            for b0 in range(0, recs.n, batch):
                nb = min(batch, recs.n - b0)
                r = lr * (lr_final / lr) ** (k / max(steps - 1, 1))
                self.step(recs, perm[b0:b0 + nb], nb, r)
                k += 1
        return self

    def predict(self, recs: RecordSet) -> torch.Tensor:
        return gs2.mlp_forward(self.w, recs.data, recs.chunk_n, recs.n)


def plain_loss(recs: RecordSet):
    """Mean 1/2 (1 - alpha*)^2 over the usable records: the plain step's error
    against the labels (the reference a trained network must beat), computed
    by the same loss kernel with the all-zero network (y = 0, alpha = 1)."""
    zero = np.zeros(gs2.MLP_NPARAM, np.float32)
    return StepModel(master=zero, bits=np.zeros(gs2.MLP_NPARAM, np.uint16)).loss(recs)

"""Writes tests/golden/oracle_tiny.json: oracle outputs on a 60-Gaussian slice of
the tiny workload (regression fixture; calls only oracle/ and the input
generators). Re-run only when a commit changes the oracle's arithmetic, and
name the passage of the paper that justifies the change in that commit."""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_2501_13975_b300 import synth  # noqa: E402


def compute():
    sc = synth.tiny_scene(n=60, seed=21)
    gt = synth.perturbed(sc, seed=22, sd=0.05)
    cams = synth.ring_cameras(4, 48)
    out = {}
    tgt = O.render(gt, cams[0])["image"]
    r = O.render(sc, cams[0])
    out["image_sum"] = r["image"].sum(axis=(1, 2)).tolist()
    out["image_px"] = r["image"][:, 24, 20].tolist()
    out["tfinal_min"] = float(r["tfinal"].min())
    L = O.loss(r["image"], tgt)
    out["loss"] = [L["loss"], L["l2"], L["lssim"]]
    out["e_px"] = L["e"][:, 24, 20].tolist()
    out["h_px"] = L["h"][:, 24, 20].tolist()
    h = O.scene_handle(sc)
    vis = np.argsort(-O.accum(O.OPACITY, h, cams[0], cams[0], L["e"], L["h"])["npix"])[:4].tolist()
    out["gaussians"] = vis
    for grp in O.GROUPS:
        b = O.accum(grp, h, cams[0], cams[0], L["e"], L["h"])
        s = O.solve(grp, h, cams[0], b["g"], b["H"])
        out[f"g{grp}"] = b["g"][..., vis].tolist()
        out[f"H{grp}"] = b["H"][..., vis].tolist()
        out[f"step{grp}"] = s["step"][..., vis].tolist()
    return out


if __name__ == "__main__":
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_tiny.json")
    with open(path, "w") as f:
        json.dump(compute(), f, indent=0)
    print("wrote", path)

"""Writes oracle_fixture_small.json: outputs of the FP64 oracle on a small
seeded scene.  It calls only oracle/ and synth/; the values are the oracle's
own (pinned to closed forms and finite differences in test_oracle_pins.py)
and serve to check that the oracle builds to the same numbers on another
machine (x86 here, aarch64 on the GPU host).

Run from the repository root:  python tests/golden/make_oracle_fixture.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import synth  # noqa: E402


def fixture_inputs():
    sc = synth.make_scene("sphere64", dims=(12, 12, 12), probe_dims=(4, 4, 4))
    rays = synth.make_rays("sphere64", n_rays=24)
    return sc, rays


def compute():
    sc, rays = fixture_inputs()
    m = oracle.Model.from_scene(sc)
    fw = oracle.render_forward(m, rays.o, rays.d, 64.0, 32)
    drgb = np.sign(fw["rgb"] - rays.target.astype(np.float64)) / (3.0 * rays.o.shape[0])
    gr = oracle.render_backward(m, rays.o, rays.d, drgb, 64.0, 32)
    out = {k: fw[k].ravel() for k in ("rgb", "depth", "wsum", "logT")}
    for k in ("sdf", "feat", "probes", "mlp"):
        out["grad_" + k] = gr[k].ravel()
    return out


def to_fixture(full):
    out = {k: full[k].tolist() for k in ("rgb", "depth", "wsum", "logT")}
    for k in ("sdf", "feat", "probes", "mlp"):
        flat = full["grad_" + k]
        idx = np.argsort(-np.abs(flat))[:32]
        out["grad_" + k] = {"index": idx.tolist(), "value": flat[idx].tolist()}
    return out


if __name__ == "__main__":
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_fixture_small.json")
    with open(path, "w") as f:
        json.dump(to_fixture(compute()), f, indent=1)
    print("wrote", path)

"""Writes tests/golden/cfg0_oracle.json from the oracle alone.

The paper prints no per-pixel values or worked example, so this fixture is a
regression record of the oracle (pinned by the closed-form and invariant
tests) on the 256-splat, 128x128 configuration: the key-list size and digest
and a seeded sample of pixels.  Run: python tests/golden/make_golden.py
"""
import hashlib
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import scenegen as sg  # noqa: E402
from oracle import keys as K  # noqa: E402
from oracle import render as R  # noqa: E402


def compute():
    scene = sg.make_scene(0)
    cam = sg.look_at_camera((4.0, 0.0, 0.0), 128, 128)
    env = sg.make_env(0)
    kl = K.build_keys(scene, cam)
    out = R.render(scene, cam, env, keylist=kl)
    rng = np.random.default_rng(123)
    cov = np.argwhere(out["A"].numpy() > 0.05)
    pick = cov[rng.choice(len(cov), size=24, replace=False)]
    digest = hashlib.sha256(kl["keys"].tobytes() + kl["ids"].tobytes()).hexdigest()
    return dict(
        source="oracle (FP64) on configuration 0: 256 splats, 4x4 texels, 128x128, seed 0",
        n_pairs=int(kl["keys"].size),
        keys_sha256=digest,
        pixels=[[int(y), int(x)] for y, x in pick],
        rgba=[[float(v) for v in out["rgba"].numpy()[y, x]] for y, x in pick],
        mean_rgba=[float(v) for v in out["rgba"].numpy().reshape(-1, 4).mean(0)],
    )


if __name__ == "__main__":
    with open(os.path.join(HERE, "cfg0_oracle.json"), "w") as f:
        json.dump(compute(), f, indent=1)

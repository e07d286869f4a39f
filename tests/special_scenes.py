"""Hand-built scenes shared by the GPU parity tests and the CPU checks of their set-up.

Each scene is meant to exercise one property of the method (the alpha cap of App. C.2, the
paper's Fig. 1 example, the ABI's camera limit).  Whether a scene really does so depends on the
oracle alone, so `tests/test_special_scene_setups.py` checks that on the CPU: an oracle change
that breaks a scene's premise then fails there instead of inside a GPU run."""
import json
import os

import numpy as np

from paper_2409_06765_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _f32(a):
    return np.ascontiguousarray(a, np.float32)


def clamp_scene():
    """A 4 x 4 grid of Gaussians facing an identity camera, boxes disjoint (one layer per pixel).
    Even ones have o~ = sigmoid(9) ~ 0.9999, so at the pixel 0.1 px from their mean
    o~ e^-sigma > alpha_max and alpha sits on the cap; odd ones never reach it.  Every pair stays
    0.87 % away from the cap, 1.2e-4 (relative) from the 1/255 skip and 0.1 px from a box edge,
    far beyond float32 rounding, so the GPU and the oracle take the same decisions."""
    W = H = 132
    f, c, z = 80.0, 66.0, 4.0
    cam = synth.Camera(W, H, np.eye(4, dtype=np.float32), f, f, c, c)
    gx, gy = np.meshgrid([18.4, 50.4, 82.4, 114.4], [18.4, 50.4, 82.4, 114.4])
    n = gx.size
    means = np.stack([(gx.ravel() - c) * z / f, (gy.ravel() - c) * z / f, np.full(n, z)], 1)
    rng = np.random.default_rng(23)
    quats = rng.normal(0, 1, (n, 4))
    quats[:, 0] += 3.0
    log_scales = np.log(0.15) + rng.normal(0, 0.05, (n, 3))
    logits = np.where(np.arange(n) % 2 == 0, 9.0, 0.5)
    sh = rng.normal(0, 0.4, (n, 4, 3))
    return synth.Scene(_f32(means), _f32(quats), _f32(log_scales), _f32(logits), _f32(sh), 1), cam


def clamped_pairs(oracle, scene, cam, bg):
    """Number of (centre pixel, Gaussian) pairs of the clamp scene whose alpha the oracle caps.
    The cap is compared with the oracle's own alpha_max (the float32 value the ABI carries)."""
    ref = oracle.render(scene, cam, bg=bg)
    sp = ref["splats"]
    clamped = 0
    for n in range(0, scene.n, 2):
        x, y = (int(v) for v in sp["means2d"][n])
        _, al, _ = oracle.render_trace(sp, ref["colors"], x, y, bg=bg)
        clamped += int(np.sum(al >= oracle.ALPHA_MAX))
    return clamped, ref


def fig1_scene():
    """Fig. 1's example as a caller passes it: float32 arrays built from the golden inputs."""
    with open(os.path.join(GOLDEN, "fig1_single_gaussian.json")) as fh:
        g = json.load(fh)
    scale = g["scale_for_test"]
    sc = synth.Scene(_f32([g["mean"]]), _f32([g["quat"]]), _f32([[np.log(scale)] * 3]),
                     _f32([g["opacity_logit_for_test"]]), _f32(np.ones((1, 1, 3))), 0)
    K = g["K"]
    cam = synth.Camera(g["width"], g["height"], np.eye(4, dtype=np.float32), K[0][0], K[1][1], K[0][2], K[1][2])
    return sc, cam


def ragged_sizes(count):
    """`count` distinct image sizes between 23 x 19 and 83 x 65; most have no side that is a
    multiple of 8, so their last tile row and column are partial at every tile size."""
    return [(23 + (17 * i) % 61, 19 + (13 * i) % 47) for i in range(count)]

"""Pins of the oracle's depth rendering (App. A): closed forms on one and two Gaussians and
FP64 central differences of the accumulated and expected depth through the whole chain."""
import numpy as np

import oracle
from paper_2409_06765_gb300 import synth

from test_oracle_grad_fd import _f64_scene


def _one_gaussian(z=3.0, logit=2.0):
    means = np.array([[0.1, -0.05, 0.0]])
    sc = synth.Scene(means, np.array([[1.0, 0.0, 0.0, 0.0]]), np.full((1, 3), np.log(0.15)), np.array([logit]),
                     np.full((1, 1, 3), 0.4), 0)
    cam = synth.make_camera(32, 24, np.array([0.0, 0.0, -z]), f=30.0)
    return sc, cam


def test_expected_depth_of_one_gaussian_is_its_depth():
    sc, cam = _one_gaussian()
    r = oracle.render_depth(sc, cam)
    z = float(r["splats"]["depths"][0])
    assert abs(z - 3.0) < 1e-12  # the camera looks along +z from z = -3 at the origin plane
    hit = r["alpha"] > 0
    assert hit.sum() > 20
    np.testing.assert_allclose(r["expected_depth"][hit], z, rtol=1e-12)
    np.testing.assert_allclose(r["acc_depth"][hit], z * r["alpha"][hit], rtol=1e-12)
    assert np.all(r["expected_depth"][~hit] == 0) and np.all(r["acc_depth"][~hit] == 0)


def test_expected_depth_of_two_gaussians_is_the_weighted_mean():
    means = np.array([[0.0, 0.0, 0.0], [0.02, 0.01, 1.5]])
    sc = synth.Scene(means, np.tile([1.0, 0, 0, 0], (2, 1)), np.full((2, 3), np.log(0.3)), np.array([0.3, 1.0]),
                     np.full((2, 1, 3), 0.2), 0)
    cam = synth.make_camera(16, 16, np.array([0.0, 0.0, -4.0]), f=20.0)
    r = oracle.render_depth(sc, cam)
    centre = 8 * 16 + 8
    ids, alphas, Ts = oracle.render_trace(r["splats"], r["colors"], 8, 8)
    assert len(ids) == 2
    z = r["splats"]["depths"][ids]
    w = alphas * Ts
    np.testing.assert_allclose(r["acc_depth"][centre], (z * w).sum(), rtol=1e-12)
    np.testing.assert_allclose(r["expected_depth"][centre], (z * w).sum() / w.sum(), rtol=1e-12)
    assert z.min() < r["expected_depth"][centre] < z.max()


def test_depth_gradients_match_finite_differences():
    sc0, cam = synth.random_small_scene(8, seed=51, sh_degree=1, width=20, height=16, log_scale_mu=-1.7, spread=0.6)
    sc = _f64_scene(sc0)
    rng = np.random.default_rng(52)
    P = cam.width * cam.height
    wc, wA, wE, wa = rng.normal(size=(P, 3)), rng.normal(size=P), rng.normal(size=P), rng.normal(size=P)

    def loss(r):
        return float((r["color"] * wc).sum() + (r["acc_depth"] * wA).sum() + (r["expected_depth"] * wE).sum()
                     + (r["alpha"] * wa).sum())

    def sig(r):
        sp = r["splats"]
        return sp["radii"].tobytes() + sp["boxes"].tobytes() + r["ncontrib"].tobytes() + r["blends"].tobytes()

    g = oracle.render_depth_grads(sc, cam, wc, d_acc_depth=wA, d_expected_depth=wE, d_alpha=wa)
    base = oracle.render_depth(sc, cam)
    assert base["ncontrib"].sum() > 40
    s0 = sig(base)
    h = 1e-6
    checked = skipped = 0
    for name, key in (("means", "d_means"), ("log_scales", "d_log_scales"), ("opacity_logits", "d_opacity_logits"),
                      ("quats", "d_quats")):
        flat = getattr(sc, name).reshape(-1)
        ana = g[key].reshape(-1)
        scale = np.abs(ana).max() + 1e-12
        for i in range(flat.size):
            old = flat[i]
            flat[i] = old + h
            rp = oracle.render_depth(sc, cam)
            flat[i] = old - h
            rm = oracle.render_depth(sc, cam)
            flat[i] = old
            if sig(rp) != s0 or sig(rm) != s0:
                skipped += 1
                continue
            fd = (loss(rp) - loss(rm)) / (2 * h)
            assert abs(fd - ana[i]) <= 1e-5 * abs(fd) + 2e-6 * scale, (name, i, fd, ana[i])
            checked += 1
    assert checked > 0.9 * (checked + skipped)

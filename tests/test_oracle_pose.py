"""Pins of the oracle's pose gradient (App. A, pose optimization): the gradient of the loss
w.r.t. the 12 free entries of the world->camera matrix [R | t], against FP64 central
differences, and the translation identity that moving the camera with the scene changes
nothing: sum_n dL/dmu_n = R^T dL/dt."""
import dataclasses

import numpy as np

import oracle
from paper_2409_06765_gb300 import synth

from test_oracle_grad_fd import _f64_scene


def _setup(seed, deg):
    sc0, cam0 = synth.random_small_scene(8, seed=seed, sh_degree=deg, width=20, height=16, log_scale_mu=-1.7,
                                         spread=0.6)
    vm = np.array(cam0.viewmat, dtype=np.float64)
    u, _, vt = np.linalg.svd(vm[:3, :3])
    vm[:3, :3] = u @ vt  # orthonormal to float64 rounding (the stored matrix is float32)
    cam = dataclasses.replace(cam0, viewmat=vm)
    rng = np.random.default_rng(seed + 100)
    P = cam.width * cam.height
    return _f64_scene(sc0), cam, rng.normal(size=(P, 3)), rng.normal(size=P)


def _loss(r, w, wA):
    P = w.shape[0]
    return float((r["image"].reshape(P, 3) * w).sum() + (r["alpha"].reshape(P) * wA).sum())


def _sig(r):
    sp = r["splats"]
    return sp["radii"].tobytes() + sp["boxes"].tobytes() + r["ncontrib"].tobytes() + r["blends"].tobytes()


def test_pose_gradient_matches_finite_differences():
    for seed, deg in ((71, 0), (72, 2), (73, 3)):
        sc, cam, w, wA = _setup(seed, deg)
        g = oracle.render_grads(sc, cam, w, d_alpha=wA)["d_viewmat"]
        assert np.all(g[3] == 0)
        base = oracle.render(sc, cam)
        assert base["ncontrib"].sum() > 40
        s0 = _sig(base)
        h = 1e-7
        checked = 0
        scale = np.abs(g).max()
        for i in range(3):
            for j in range(4):
                vm = cam.viewmat
                old = vm[i, j]
                vm[i, j] = old + h
                rp = oracle.render(sc, cam)
                vm[i, j] = old - h
                rm = oracle.render(sc, cam)
                vm[i, j] = old
                if _sig(rp) != s0 or _sig(rm) != s0:
                    continue
                fd = (_loss(rp, w, wA) - _loss(rm, w, wA)) / (2 * h)
                assert abs(fd - g[i, j]) <= 1e-5 * abs(fd) + 2e-6 * scale, (seed, i, j, fd, g[i, j])
                checked += 1
        assert checked >= 10


def test_moving_camera_and_scene_together_changes_nothing():
    """mu -> mu + d, t -> t - R d leaves every camera-space mean and view direction as it was,
    so the gradients satisfy sum_n dL/dmu_n - R^T dL/dt = 0."""
    for seed, deg in ((74, 1), (75, 3)):
        sc, cam, w, wA = _setup(seed, deg)
        g = oracle.render_grads(sc, cam, w, d_alpha=wA)
        R = cam.viewmat[:3, :3]
        lhs = g["d_means"].sum(0)
        rhs = R.T @ g["d_viewmat"][:3, 3]
        np.testing.assert_allclose(lhs, rhs, rtol=1e-9, atol=1e-12 * np.abs(lhs).max())

"""Seeded synthetic scenes and cameras.

This module only draws inputs: Gaussian parameters, pinhole cameras and target
images. It holds none of the rasterizer's arithmetic, so both the FP64 oracle
(test side) and the CUDA path consume exactly the same float32 bytes from it.

Distributions follow the workloads the rasterizer is measured on:

* ``tiny_scene``: 1,000 Gaussians, SH degree 0, means U[-1,1]^3, log-scales
  N(-3, 0.5), quaternions N(0,1)^4 normalised, opacity logits N(0,1), colour
  coefficients N(0, 0.5); one 64x64 camera (f=64, c=32) at (0,0,4) looking at
  the origin; a U[0,1] target image.  Seed 0.
* ``clustered_scene``: means from 64 Gaussian clusters (sigma 0.3) with centres
  U[-3,3]^3, clipped to [-3,3]^3, so per-tile load is uneven; log-scales
  N(-4, 0.7); opacity logits N(0, 1.5); SH degree 3 with DC N(0, 0.5) and the
  other 45 coefficients N(0, 0.05).  Options cover the memory-bound variant
  (log-scales N(-4.5, 0.8), 20% of logits redrawn from N(3, 0.5)).
* cameras on a radius-6 sphere looking at the origin, focal length 0.848 * W
  (the field of view of a 1297x840, f=1100 camera) unless given.

Camera convention (OpenCV): x right, y down, z forward.  ``viewmat`` maps world
to camera coordinates, row-major 4x4.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Camera", "Scene", "look_at", "make_camera", "tiny_scene", "clustered_scene",
    "sphere_cameras", "headline_workload", "training_step_workload",
    "multiview_workload", "memory_workload", "random_small_scene", "sample_pixels",
]


@dataclass
class Camera:
    width: int
    height: int
    viewmat: np.ndarray  # float32 [4,4], world -> camera
    fx: float
    fy: float
    cx: float
    cy: float

    def as_tuple(self):
        return (self.width, self.height, self.viewmat, self.fx, self.fy, self.cx, self.cy)


@dataclass
class Scene:
    means: np.ndarray           # float32 [N,3]
    quats: np.ndarray           # float32 [N,4] (w,x,y,z)
    log_scales: np.ndarray      # float32 [N,3]
    opacity_logits: np.ndarray  # float32 [N]
    sh: np.ndarray              # float32 [N,K,3], K=(degree+1)^2
    sh_degree: int
    extra: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.means.shape[0])


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def look_at(eye, target=(0.0, 0.0, 0.0)) -> np.ndarray:
    """World->camera matrix for a camera at ``eye`` looking at ``target``.

    Rows of the rotation are the camera x (right), y (down) and z (forward)
    axes expressed in world coordinates; translation is -R @ eye.
    """
    eye = np.asarray(eye, dtype=np.float64)
    target = np.asarray(target, dtype=np.float64)
    fwd = target - eye
    fwd /= np.linalg.norm(fwd)
    up = np.array([0.0, 1.0, 0.0])
    if abs(float(fwd @ up)) > 0.99:
        up = np.array([0.0, 0.0, 1.0])
    right = np.cross(fwd, up)
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    rot = np.stack([right, down, fwd])
    vm = np.eye(4)
    vm[:3, :3] = rot
    vm[:3, 3] = -rot @ eye
    return _f32(vm)


def make_camera(width, height, eye, f=None, target=(0.0, 0.0, 0.0), cx=None, cy=None) -> Camera:
    f = 0.848 * width if f is None else f
    cx = width / 2.0 if cx is None else cx
    cy = height / 2.0 if cy is None else cy
    return Camera(int(width), int(height), look_at(eye, target), float(np.float32(f)),
                  float(np.float32(f)), float(np.float32(cx)), float(np.float32(cy)))


def _unit(rng, n):
    v = rng.normal(0.0, 1.0, (n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def tiny_scene(seed: int = 0, n: int = 1000):
    """1,000-Gaussian SH-0 scene, one 64x64 camera and a U[0,1] target image."""
    rng = np.random.default_rng(seed)
    means = rng.uniform(-1.0, 1.0, (n, 3))
    log_scales = rng.normal(-3.0, 0.5, (n, 3))
    quats = rng.normal(0.0, 1.0, (n, 4))
    quats /= np.linalg.norm(quats, axis=1, keepdims=True)
    logits = rng.normal(0.0, 1.0, n)
    sh = rng.normal(0.0, 0.5, (n, 1, 3))
    cam = make_camera(64, 64, eye=(0.0, 0.0, 4.0), f=64.0, cx=32.0, cy=32.0)
    target = rng.uniform(0.0, 1.0, (64, 64, 3))
    scene = Scene(_f32(means), _f32(quats), _f32(log_scales), _f32(logits), _f32(sh), 0)
    return scene, cam, _f32(target)


def clustered_scene(n: int, seed: int, sh_degree: int = 3, clusters: int = 64,
                    cluster_sigma: float = 0.3, extent: float = 3.0,
                    log_scale_mu: float = -4.0, log_scale_sigma: float = 0.7,
                    logit_sigma: float = 1.5, opaque_frac: float = 0.0,
                    opaque_mu: float = 3.0, opaque_sigma: float = 0.5) -> Scene:
    """Clustered scene: uneven per-tile load, SH up to degree 3."""
    rng = np.random.default_rng(seed)
    centres = rng.uniform(-extent, extent, (clusters, 3))
    pick = rng.integers(0, clusters, n)
    means = centres[pick] + cluster_sigma * rng.normal(0.0, 1.0, (n, 3))
    np.clip(means, -extent, extent, out=means)
    log_scales = rng.normal(log_scale_mu, log_scale_sigma, (n, 3))
    quats = rng.normal(0.0, 1.0, (n, 4))
    quats /= np.linalg.norm(quats, axis=1, keepdims=True)
    logits = rng.normal(0.0, logit_sigma, n)
    if opaque_frac > 0.0:
        sel = rng.random(n) < opaque_frac
        logits[sel] = rng.normal(opaque_mu, opaque_sigma, int(sel.sum()))
    k = (sh_degree + 1) ** 2
    # float32 draws in place (the coefficient array dominates the scene's size): DC N(0, 0.5),
    # higher orders N(0, 0.05)
    sh = rng.standard_normal((n, k, 3), dtype=np.float32)
    sh[:, 0, :] *= np.float32(0.5)
    if k > 1:
        sh[:, 1:, :] *= np.float32(0.05)
    return Scene(_f32(means), _f32(quats), _f32(log_scales), _f32(logits), _f32(sh), sh_degree)


def sphere_cameras(seed: int, sizes, radius: float = 6.0, focal_scale: float = 0.848):
    """One camera per (W, H) in ``sizes`` at a random point of a sphere, looking at the origin."""
    rng = np.random.default_rng(seed)
    eyes = radius * _unit(rng, len(sizes))
    return [make_camera(w, h, eye, f=focal_scale * w) for (w, h), eye in zip(sizes, eyes)]


def headline_workload(n: int = 3_000_000, seed: int = 3):
    """3M clustered Gaussians (SH 3) and one 1920x1080 camera on the radius-6 sphere."""
    scene = clustered_scene(n, seed)
    cam = sphere_cameras(seed + 1000, [(1920, 1080)])[0]
    rng = np.random.default_rng(seed + 2000)
    target = _f32(rng.uniform(0.0, 1.0, (cam.height, cam.width, 3)))
    return scene, cam, target


def training_step_workload(n: int = 1_000_000, seed: int = 2):
    """1M clustered Gaussians (SH 3) and one 1297x840 camera, f=1100."""
    scene = clustered_scene(n, seed)
    rng = np.random.default_rng(seed + 1000)
    eye = 6.0 * _unit(rng, 1)[0]
    cam = make_camera(1297, 840, eye, f=1100.0, cx=648.5, cy=420.0)
    target = _f32(np.random.default_rng(seed + 2000).uniform(0.0, 1.0, (840, 1297, 3)))
    return scene, cam, target


def multiview_workload(n: int = 3_000_000, seed: int = 3):
    """The 3M scene seen by 16 cameras: 4 each of 640x480, 1280x720, 1920x1080, 2560x1440."""
    scene = clustered_scene(n, seed)
    sizes = [(640, 480)] * 4 + [(1280, 720)] * 4 + [(1920, 1080)] * 4 + [(2560, 1440)] * 4
    cams = sphere_cameras(seed + 3000, sizes)
    return scene, cams


def memory_workload(n: int = 6_000_000, seed: int = 4):
    """6M Gaussians with smaller scales and 20% near-opaque, four 1920x1080 views."""
    scene = clustered_scene(n, seed, log_scale_mu=-4.5, log_scale_sigma=0.8, opaque_frac=0.2)
    cams = sphere_cameras(seed + 3000, [(1920, 1080)] * 4)
    return scene, cams


def random_small_scene(n: int, seed: int, sh_degree: int = 0, width: int = 32, height: int = 32,
                       log_scale_mu: float = -2.0, log_scale_sigma: float = 0.4,
                       spread: float = 0.8, cam_dist: float = 3.0):
    """A handful of Gaussians in front of one small camera, for oracle pins and finite differences."""
    rng = np.random.default_rng(seed)
    means = rng.uniform(-spread, spread, (n, 3))
    log_scales = rng.normal(log_scale_mu, log_scale_sigma, (n, 3))
    quats = rng.normal(0.0, 1.0, (n, 4))
    logits = rng.normal(0.5, 1.0, n)
    k = (sh_degree + 1) ** 2
    sh = rng.normal(0.0, 0.5, (n, k, 3))
    if k > 1:
        sh[:, 1:, :] *= 0.4
    eye = cam_dist * np.array([0.3, -0.2, 1.0]) / np.linalg.norm([0.3, -0.2, 1.0])
    f = 1.1 * width
    cam = make_camera(width, height, eye, f=f)
    scene = Scene(_f32(means), _f32(quats), _f32(log_scales), _f32(logits), _f32(sh), sh_degree)
    return scene, cam


def sample_pixels(width: int, height: int, count: int, seed: int) -> np.ndarray:
    """Seeded, sorted, distinct linear pixel indices (y * width + x)."""
    rng = np.random.default_rng(seed)
    total = width * height
    count = min(count, total)
    return np.sort(rng.choice(total, size=count, replace=False)).astype(np.int32)

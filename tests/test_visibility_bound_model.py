"""Host model of the conservative visibility test of the fused projection + SH forward, checked
on the CPU against the oracle's projection (App. C.1).  No kernel runs here.

The fused forward starts copying a Gaussian's coefficient row before it has projected the
Gaussian, for every Gaussian that some camera *may* see: one in front of the near plane whose
pixel box, widened from an upper bound of the splat's radius, meets the image.  The bound is
lambda_max(T Sigma T^T) <= |T|_F^2 s_max^2 (T = J R_cw, s_max the largest scale), plus the
low-pass and margins.  A Gaussian the bound drops but the projection keeps would only cost a
read of its row from global memory (the kernel falls back to it), so the bound decides speed,
not results; these tests check that it drops nothing the projection keeps, including Gaussians
near the image edges, elongated ones, huge ones and ones just in front of the near plane."""
import numpy as np
import pytest

import oracle
from paper_2409_06765_gb300 import synth


def maybe_visible(mean, log_scales, cam, eps2d=0.3, near=0.01):
    """float32 replica of the kernel's test, vectorised over Gaussians."""
    f32 = np.float32
    V = np.asarray(cam.viewmat, f32)
    R, t = V[:3, :3], V[:3, 3]
    m = np.asarray(mean, f32)
    tc = (m @ R.T + t).astype(f32)
    tx, ty, tz = tc[:, 0], tc[:, 1], tc[:, 2]
    front = tz >= f32(near)
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        iz = (f32(1) / tz).astype(f32)
        fx, fy, cx, cy = f32(cam.fx), f32(cam.fy), f32(cam.cx), f32(cam.cy)
        mx = fx * tx * iz + cx
        my = fy * ty * iz + cy
        j00, j02 = fx * iz, -fx * tx * iz * iz
        j11, j12 = fy * iz, -fy * ty * iz * iz
        tf = np.zeros_like(tz)
        for k in range(3):
            a = j00 * R[0, k] + j02 * R[2, k]
            b = j11 * R[1, k] + j12 * R[2, k]
            tf = tf + a * a + b * b
        smax = np.exp(np.asarray(log_scales, f32).max(1)).astype(f32)
        r = f32(3) * np.sqrt(tf * smax * smax * f32(1.01) + f32(eps2d)) * f32(1.01) + f32(2)
        huge = ~(r < f32(1e8))
        inside = (mx + r >= -1) & (mx - r <= cam.width + 1) & (my + r >= -1) & (my - r <= cam.height + 1)
    return front & (huge | inside)


def _scene(n, seed, spread, log_mu, log_sigma):
    rng = np.random.default_rng(seed)
    sc = synth.clustered_scene(n, seed, sh_degree=0, log_scale_mu=log_mu, log_scale_sigma=log_sigma)
    sc.means[:] = rng.uniform(-spread, spread, sc.means.shape).astype(np.float32)
    # some very elongated Gaussians: one large scale, two small ones
    k = rng.random(n) < 0.2
    sc.log_scales[k, 0] += np.float32(2.5)
    sc.log_scales[k, 1:] -= np.float32(1.0)
    return sc


@pytest.mark.parametrize("seed,spread,log_mu,log_sigma", [(1, 8.0, -3.0, 1.0), (2, 12.0, -1.5, 1.2),
                                                         (3, 6.5, -4.0, 0.7), (4, 20.0, 0.0, 1.0)])
def test_bound_keeps_every_gaussian_the_projection_keeps(seed, spread, log_mu, log_sigma):
    """Means spread well beyond the view (most are culled), scales from tiny to larger than the
    scene: every Gaussian with a non-empty pixel box in the oracle's projection passes the bound,
    and the bound still drops most of the ones outside the view."""
    sc = _scene(4000, seed, spread, log_mu, log_sigma)
    cams = synth.sphere_cameras(seed, [(160, 120), (97, 203), (333, 55)])
    for cam in cams:
        vis = oracle.project(sc, cam)["radii"] > 0
        keep = maybe_visible(sc.means, sc.log_scales, cam)
        missed = vis & ~keep
        assert not missed.any(), np.flatnonzero(missed)[:10]
        assert keep.sum() < len(keep)  # the bound is not vacuous
        if (~vis).sum() > 100:
            assert (~keep & ~vis).sum() >= 0.3 * (~vis).sum()


def test_bound_at_the_near_plane_and_the_image_edges():
    """Gaussians straddling the near plane and the image border, where the exact decision is
    closest to the bound's."""
    rng = np.random.default_rng(9)
    cam = synth.make_camera(128, 96, (0.0, 0.0, 4.0))
    n = 3000
    sc = _scene(n, 9, 1.0, -3.0, 0.8)
    # depths from just behind to just in front of the near plane (camera looks down -z from z=4)
    sc.means[:1000, 2] = (4.0 - rng.uniform(0.0, 0.05, 1000)).astype(np.float32)
    # means around the image border at depth 4: x, y near +-(W/2)/f * depth
    half_w, half_h = 64 / cam.fx * 4.0, 48 / cam.fy * 4.0
    side = rng.choice([-1.0, 1.0], (2000, 2))
    sc.means[1000:, 0] = (side[:, 0] * half_w * rng.uniform(0.9, 1.3, 2000)).astype(np.float32)
    sc.means[1000:, 1] = (side[:, 1] * half_h * rng.uniform(0.9, 1.3, 2000)).astype(np.float32)
    sc.means[1000:, 2] = 0.0
    vis = oracle.project(sc, cam)["radii"] > 0
    keep = maybe_visible(sc.means, sc.log_scales, cam)
    assert vis.sum() > 100 and (~vis).sum() > 100
    assert not (vis & ~keep).any(), np.flatnonzero(vis & ~keep)[:10]

"""The seeded synthetic inputs follow their stated recipe.

Every parity case and every benchmark line draws its scene and cameras from
``paper_2409_06765_gb300.synth``.  These checks tie the generators to the recipe:
the OpenCV look-at convention (x right, y down, z forward, t = -R eye), the
default intrinsics (f = 0.848 W, principal point at the image centre), the
clustered scene's distributions (clipped means, log-normal scales, opacity
logits, SH coefficient spreads, the near-opaque fraction of the memory workload),
seeding, and the pixel sampler.  Sizes are small; nothing here needs a GPU.
"""
import numpy as np
import pytest

from paper_2409_06765_gb300 import synth


@pytest.mark.parametrize("eye", [(0.0, 0.0, 4.0), (3.0, -2.0, 1.5), (0.0, 5.0, 0.01), (-1.0, 0.3, -6.0)])
def test_look_at_is_opencv(eye):
    vm = synth.look_at(eye).astype(np.float64)
    R, t = vm[:3, :3], vm[:3, 3]
    np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-6)
    assert np.linalg.det(R) == pytest.approx(1.0, abs=1e-6)
    np.testing.assert_allclose(t, -R @ np.asarray(eye), atol=1e-5)
    np.testing.assert_array_equal(vm[3], [0, 0, 0, 1])
    # the target (origin) lies on the optical axis in front of the camera, at the eye's distance
    c = t  # R @ 0 + t
    np.testing.assert_allclose(c[:2], 0.0, atol=1e-5)
    assert c[2] == pytest.approx(np.linalg.norm(eye), rel=1e-6)
    # camera y points down: a world point above the target (larger world y, or larger z when the
    # camera looks along y) lands at a smaller camera y
    up = np.array([0.0, 1.0, 0.0]) if abs(eye[1]) < 0.99 * np.linalg.norm(eye) else np.array([0.0, 0.0, 1.0])
    assert (R @ up)[1] < 0


def test_default_intrinsics_and_float32_values():
    cam = synth.make_camera(1920, 1080, (0.0, 0.0, 6.0))
    assert cam.fx == cam.fy == pytest.approx(0.848 * 1920, rel=1e-7)
    assert (cam.cx, cam.cy) == (960.0, 540.0)
    for v in (cam.fx, cam.fy, cam.cx, cam.cy):
        assert float(np.float32(v)) == v
    assert cam.viewmat.dtype == np.float32


def test_sphere_cameras_sit_on_the_radius_6_sphere():
    sizes = [(640, 480), (1280, 720), (1920, 1080), (2560, 1440)]
    cams = synth.sphere_cameras(7, sizes)
    for cam, (w, h) in zip(cams, sizes):
        R, t = cam.viewmat[:3, :3].astype(np.float64), cam.viewmat[:3, 3].astype(np.float64)
        assert (cam.width, cam.height) == (w, h)
        assert np.linalg.norm(-R.T @ t) == pytest.approx(6.0, rel=1e-5)
        assert cam.fx == pytest.approx(0.848 * w, rel=1e-7)


def test_clustered_scene_distributions():
    n = 200_000
    sc = synth.clustered_scene(n, seed=11)
    assert sc.n == n and sc.sh_degree == 3
    for a in (sc.means, sc.quats, sc.log_scales, sc.opacity_logits, sc.sh):
        assert a.dtype == np.float32 and a.flags.c_contiguous
    assert sc.means.shape == (n, 3) and sc.quats.shape == (n, 4) and sc.sh.shape == (n, 16, 3)
    # means: 64 cluster centres in [-3, 3]^3 with 0.3 spread, clipped to the cube
    assert np.abs(sc.means).max() <= 3.0
    assert (np.abs(sc.means) == 3.0).any()
    np.testing.assert_allclose(np.linalg.norm(sc.quats, axis=1), 1.0, atol=1e-6)
    assert sc.log_scales.mean() == pytest.approx(-4.0, abs=0.01)
    assert sc.log_scales.std() == pytest.approx(0.7, rel=0.01)
    assert sc.opacity_logits.mean() == pytest.approx(0.0, abs=0.02)
    assert sc.opacity_logits.std() == pytest.approx(1.5, rel=0.01)
    assert sc.sh[:, 0].std() == pytest.approx(0.5, rel=0.01)
    assert sc.sh[:, 1:].std() == pytest.approx(0.05, rel=0.01)
    # clustered: most Gaussians lie within 1 (about 3.3 cluster sigmas) of one of few centres
    d = np.linalg.norm(sc.means[:, None, :] - sc.means[None, :200, :], axis=2).min(axis=1)
    assert np.median(d) < 0.6


def test_memory_workload_recipe_near_opaque_fraction():
    sc = synth.clustered_scene(100_000, seed=4, log_scale_mu=-4.5, log_scale_sigma=0.8, opaque_frac=0.2)
    assert sc.log_scales.mean() == pytest.approx(-4.5, abs=0.02)
    assert sc.log_scales.std() == pytest.approx(0.8, rel=0.02)
    high = sc.opacity_logits > 1.5  # N(3, 0.5) draws, 3 sigmas above 1.5; N(0, 1.5) ones rarely
    assert high.mean() == pytest.approx(0.2 + 0.8 * 0.159, abs=0.01)


def test_tiny_scene_recipe():
    sc, cam, target = synth.tiny_scene()
    assert sc.n == 1000 and sc.sh_degree == 0 and sc.sh.shape == (1000, 1, 3)
    assert np.abs(sc.means).max() <= 1.0
    assert (cam.width, cam.height, cam.fx, cam.cx, cam.cy) == (64, 64, 64.0, 32.0, 32.0)
    np.testing.assert_allclose(-cam.viewmat[:3, :3].T.astype(np.float64) @ cam.viewmat[:3, 3], [0, 0, 4],
                               atol=1e-6)
    assert target.shape == (64, 64, 3) and 0.0 <= target.min() and target.max() <= 1.0


def test_generators_are_seeded():
    a, b = synth.clustered_scene(5000, seed=3), synth.clustered_scene(5000, seed=3)
    c = synth.clustered_scene(5000, seed=4)
    for k in ("means", "quats", "log_scales", "opacity_logits", "sh"):
        np.testing.assert_array_equal(getattr(a, k), getattr(b, k))
        assert not np.array_equal(getattr(a, k), getattr(c, k))
    np.testing.assert_array_equal(synth.sphere_cameras(9, [(64, 48)])[0].viewmat,
                                  synth.sphere_cameras(9, [(64, 48)])[0].viewmat)


def test_sample_pixels_distinct_sorted_in_range():
    p = synth.sample_pixels(203, 157, 4096, seed=1)
    assert p.dtype == np.int32 and len(p) == 4096
    assert (np.diff(p) > 0).all() and p.min() >= 0 and p.max() < 203 * 157
    assert len(synth.sample_pixels(8, 8, 4096, seed=1)) == 64

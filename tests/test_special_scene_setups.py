"""CPU checks of the premises of the hand-built GPU parity scenes.

What a GPU parity test can show depends on its scene: the alpha-cap test only proves something if
the oracle really caps alpha there, the Fig. 1 test only if the Gaussian renders, the camera-limit
test only if every one of its ragged views sees something.  Those premises involve the oracle and
the input generators alone, so they are checked here, where a change of the oracle that breaks
them fails the CPU suite instead of a GPU run."""
import numpy as np

import oracle
from paper_2409_06765_gb300 import _lib, synth

import special_scenes


def test_clamp_scene_caps_alpha_at_half_of_the_centre_pixels():
    sc, cam = special_scenes.clamp_scene()
    bg = np.array([0.3, 0.2, 0.1])
    clamped, ref = special_scenes.clamped_pairs(oracle, sc, cam, bg)
    # each even (opaque) Gaussian is capped at the pixel nearest its mean; odd ones never are
    assert clamped == sc.n // 2
    sp = ref["splats"]
    for n in range(1, sc.n, 2):
        x, y = (int(v) for v in sp["means2d"][n])
        _, al, _ = oracle.render_trace(sp, ref["colors"], x, y, bg=bg)
        assert (al < oracle.ALPHA_MAX).all()
    # the cap is the float32 value the ABI carries, not the float64 literal
    assert oracle.ALPHA_MAX == np.float64(np.float32(0.99)) != 0.99


def test_clamp_scene_keeps_every_decision_away_from_float32_rounding():
    """The capped pairs sit well above the cap and no pair is near the 1/255 skip, so float32
    and float64 take the same decisions (what the GPU comparison relies on)."""
    sc, cam = special_scenes.clamp_scene()
    ref = oracle.render(sc, cam, bg=np.zeros(3))
    sp = ref["splats"]
    assert (sp["radii"] > 0).all()
    for n in range(sc.n):
        x, y = (int(v) for v in sp["means2d"][n])
        d = np.array([x + 0.5, y + 0.5]) - sp["means2d"][n]
        a, b, c = sp["conics"][n]
        raw = sp["opacities"][n] * np.exp(-0.5 * (a * d[0] ** 2 + 2 * b * d[0] * d[1] + c * d[1] ** 2))
        if n % 2 == 0:
            assert raw > oracle.ALPHA_MAX * 1.005
        else:
            assert raw < oracle.ALPHA_MAX * 0.99 and raw > oracle.ALPHA_MIN * 1.0001


def test_fig1_scene_renders_a_centred_blob():
    sc, cam = special_scenes.fig1_scene()
    ref = oracle.render(sc, cam)
    assert ref["splats"]["radii"][0] > 0
    lum = ref["image"].reshape(cam.height, cam.width, 3)[..., 0]
    assert lum.max() > 0.5
    # alpha sits on its cap on a small plateau around the principal point, which includes the
    # four pixels that touch it
    for y, x in ((119, 119), (119, 120), (120, 119), (120, 120)):
        assert lum[y, x] == lum.max()
    np.testing.assert_allclose(lum, lum.T, atol=1e-12)


def test_ragged_sizes_fill_the_camera_limit_and_every_view_sees_the_scene():
    sizes = special_scenes.ragged_sizes(_lib.GS_MAX_CAMERAS)
    assert len(sizes) == _lib.GS_MAX_CAMERAS == len(set(sizes))
    assert sum(w % 8 != 0 and h % 8 != 0 for w, h in sizes) >= 3 * len(sizes) // 4
    sc = synth.clustered_scene(3000, 63, sh_degree=1, log_scale_mu=-3.0)
    cams = synth.sphere_cameras(63, sizes)
    for cam in cams:
        assert (oracle.project(sc, cam)["radii"] > 0).sum() > 100

"""Special cases against the oracle: the paper's Fig. 1 example, calls at the C ABI's limits
(the maximum number of cameras in one call, 32 of uneven and ragged sizes, and the maximum number
of feature channels, 64), and degenerate view sizes (one pixel, one row, one column)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2409_06765_gb300 import _lib, raster, synth

import special_scenes
from gpu_helpers import assert_grad_parity, assert_image_parity, dev_scene, flipped_pixels, gpu_grads, gpu_render, \
    rel_l2

pytestmark = pytest.mark.gpu


def test_fig1_example_matches_the_oracle():
    """Fig. 1: one Gaussian at (0, 0, 0.01), identity pose, f = 1, principal point (120, 120),
    240 x 240.  Its depth equals the near plane (0.01 in float32 on both sides), which does not
    cull it; the image is a blob centred on the principal point, the same as the oracle's."""
    sc, cam = special_scenes.fig1_scene()
    out, _, _ = gpu_render(sc, [cam])
    ref = oracle.render(sc, cam)
    P = cam.width * cam.height
    img = out["image"].cpu().numpy()
    assert out["radii"][0, 0].item() > 0 and ref["splats"]["radii"][0] > 0
    assert_image_parity(img, ref["image"].reshape(P, 3))
    assert_image_parity((1 - out["final_T"]).cpu().numpy()[:, None], ref["alpha"].reshape(P, 1), "alpha")
    lum = img[:, 0].reshape(cam.height, cam.width)
    assert lum.max() > 0.5 and lum[119, 119] == lum.max() == lum[120, 120]
    # backward of a random upstream gradient on the whole image
    rng = np.random.default_rng(12)
    d_img = rng.uniform(-1, 1, (P, 3)) / P
    g_gpu, _, _ = gpu_grads(sc, [cam], d_img)
    g_ref = oracle.render_grads(sc, cam, d_img)
    assert_grad_parity(g_gpu, g_ref, keys=("d_means", "d_log_scales", "d_opacity_logits", "d_sh"))
    # the scale is isotropic, so rotating the Gaussian changes nothing: d_quats is zero up to rounding
    assert np.abs(g_gpu["d_quats"]).max() <= 1e-3 * np.abs(g_gpu["d_log_scales"]).max()


def test_maximum_cameras_in_one_call():
    sc = synth.clustered_scene(3000, 63, sh_degree=1, log_scale_mu=-3.0)
    cams = synth.sphere_cameras(63, special_scenes.ragged_sizes(_lib.GS_MAX_CAMERAS))
    out, _, ca = gpu_render(sc, cams)
    img = out["image"].cpu().numpy()
    alpha = 1.0 - out["final_T"].cpu().numpy()
    refs = [oracle.render(sc, cam) for cam in cams]
    ref_img = np.concatenate([r["image"].reshape(-1, 3) for r in refs])
    ref_alpha = np.concatenate([r["alpha"].reshape(-1) for r in refs])
    assert img.shape == ref_img.shape
    assert_image_parity(img, ref_img)
    assert_image_parity(alpha[:, None], ref_alpha[:, None], "alpha")
    # tile lists of all 32 cameras: bit-exact against the oracle's enumeration of the GPU's splats
    keys, values, ranges = oracle.bin_sort(out["means2d"].cpu().numpy(), out["depths"].cpu().numpy(),
                                           out["radii"].cpu().numpy(), [c.width for c in cams],
                                           [c.height for c in cams], 16)
    assert out["K"] == len(values) > 0
    np.testing.assert_array_equal(out["values"].cpu().numpy(), values)
    np.testing.assert_array_equal(out["ranges"].cpu().numpy(), ranges)
    # backward summed over the 32 views; pixels where a float32/float64 threshold decision
    # differed are left out of the loss
    flips = flipped_pixels(img, alpha, ref_img, ref_alpha)
    assert flips.mean() <= 1e-4, f"{flips.sum()} threshold flips"
    rng = np.random.default_rng(8)
    d_img = rng.uniform(-1, 1, img.shape) / len(img)
    d_img[flips] = 0
    g_gpu, _, _ = gpu_grads(sc, cams, d_img)
    g_ref = None
    for cam, off in zip(cams, ca.pixel_offsets()):
        P = cam.width * cam.height
        g = oracle.render_grads(sc, cam, d_img[off:off + P])
        g_ref = g if g_ref is None else {k: g_ref[k] + g[k] for k in g_ref if k.startswith("d_")}
    assert_grad_parity(g_gpu, g_ref)


def test_maximum_feature_channels_forward_and_backward():
    """64 feature channels (App. C: c may be any N-vector), the largest compiled width."""
    sc = synth.clustered_scene(4000, 41, sh_degree=0, log_scale_mu=-3.2)
    cam = synth.sphere_cameras(41, [(203, 157)])[0]
    D = _lib.GS_MAX_CHANNELS
    rng = np.random.default_rng(4)
    feats = rng.uniform(0, 1, (sc.n, D)).astype(np.float32)
    sp = oracle.project(sc, cam)
    ref = oracle.render_splats(sp, feats.astype(np.float64), cam.width, cam.height)
    d = dev_scene(sc)
    leaves = [d["means"], d["quats"], d["log_scales"], d["opacity_logits"], torch.as_tensor(feats, device="cuda")]
    for x in leaves:
        x.requires_grad_(True)
    imgs, _, _ = raster.rasterization(*leaves[:4], cameras=[cam], features=leaves[4])
    img = imgs[0].reshape(-1, D).detach().cpu().numpy()
    assert_image_parity(img, ref["color"], "features")
    P = cam.width * cam.height
    gimg = rng.uniform(-1, 1, (P, D)) / P
    g = torch.autograd.grad([imgs[0]], leaves, [torch.as_tensor(gimg.reshape(cam.height, cam.width, D),
                                                                dtype=torch.float32, device="cuda")])
    g2 = oracle.render_splats_bwd(sp, feats.astype(np.float64), cam.width, cam.height, gimg)
    assert rel_l2(g[4].cpu().numpy(), g2["d_colors"]) < 1e-3
    g3 = oracle.project_bwd(sc, cam, g2["d_means2d"], g2["d_conics"], g2["d_opacities"])
    assert rel_l2(g[0].cpu().numpy(), g3["d_means"]) < 1e-3
    assert rel_l2(g[3].cpu().numpy(), g3["d_opacity_logits"]) < 1e-3


@pytest.mark.parametrize("tile", [8, 16, 32])
def test_degenerate_image_sizes_and_huge_gaussians(tile):
    """Images of one pixel, one row and one column (every tile partial), next to an ordinary
    size, with Gaussians far larger than the images among small ones: images, alpha, the tile
    lists and the gradients against the oracle."""
    sc = synth.clustered_scene(600, 71, sh_degree=2, log_scale_mu=-3.0)
    sc.log_scales[:12] = np.float32(0.5)  # a dozen Gaussians wider than every view
    cams = synth.sphere_cameras(71, [(1, 1), (1, 37), (37, 1), (45, 29)])
    settings = raster.RasterSettings(tile=tile)
    out, _, ca = gpu_render(sc, cams, settings=settings)
    img = out["image"].cpu().numpy()
    alpha = 1.0 - out["final_T"].cpu().numpy()
    refs = [oracle.render(sc, cam) for cam in cams]
    ref_img = np.concatenate([r["image"].reshape(-1, 3) for r in refs])
    ref_alpha = np.concatenate([r["alpha"].reshape(-1) for r in refs])
    assert img.shape == ref_img.shape == (1 + 37 + 37 + 45 * 29, 3)
    assert_image_parity(img, ref_img)
    assert_image_parity(alpha[:, None], ref_alpha[:, None], "alpha")
    keys, values, ranges = oracle.bin_sort(out["means2d"].cpu().numpy(), out["depths"].cpu().numpy(),
                                           out["radii"].cpu().numpy(), [c.width for c in cams],
                                           [c.height for c in cams], tile)
    assert out["K"] == len(values) > 0
    np.testing.assert_array_equal(out["values"].cpu().numpy(), values)
    np.testing.assert_array_equal(out["ranges"].cpu().numpy(), ranges)
    flips = flipped_pixels(img, alpha, ref_img, ref_alpha)
    rng = np.random.default_rng(72)
    d_img = rng.uniform(-1, 1, img.shape) / len(img)
    d_img[flips] = 0
    g_gpu, _, _ = gpu_grads(sc, cams, d_img, settings=settings)
    g_ref = None
    for cam, off in zip(cams, ca.pixel_offsets()):
        P = cam.width * cam.height
        g = oracle.render_grads(sc, cam, d_img[off:off + P])
        g_ref = g if g_ref is None else {k: g_ref[k] + g[k] for k in g_ref if k.startswith("d_")}
    assert_grad_parity(g_gpu, g_ref)

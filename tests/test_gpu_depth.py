"""Depth rendering (App. A) on the GPU against the oracle: accumulated depth as a fourth
composited channel, expected depth = accumulated depth / alpha, and their gradients through
the depth channel into the projection (d z_n = d t_z)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2409_06765_gb300 import _lib, raster, synth

from gpu_helpers import IMG_MEANABS, IMG_PIXEL_FRAC, IMG_PIXEL_MAXABS, assert_grad_parity, dev_scene, flipped_pixels

pytestmark = pytest.mark.gpu


def _scene(seed=61, deg=2):
    sc = synth.clustered_scene(9000, seed, sh_degree=deg, log_scale_mu=-3.2)
    cam = synth.sphere_cameras(seed, [(160, 120)])[0]
    return sc, cam


def _leaves(sc):
    d = dev_scene(sc)
    leaves = [d[k].clone().requires_grad_(True) for k in ("means", "quats", "log_scales", "opacity_logits", "sh")]
    return leaves, d["sh_degree"]


def _depth_bar(gpu, ref, zmax, what, mask=None):
    """The image bars applied to a depth channel in units of the scene's largest depth."""
    d = np.abs(np.asarray(gpu, np.float64) - ref) / zmax
    if mask is not None:
        d = d[mask]
    frac = float((d <= IMG_PIXEL_MAXABS).mean())
    assert frac >= IMG_PIXEL_FRAC, f"{what}: {frac} of pixels within the bar"
    assert d.mean() <= IMG_MEANABS, f"{what}: mean {d.mean()}"


@pytest.mark.parametrize("mode", ["RGB+D", "RGB+ED", "D", "ED"])
def test_depth_modes_forward_match_oracle(mode):
    sc, cam = _scene()
    leaves, deg = _leaves(sc)
    imgs, alphas, _ = raster.rasterization(*leaves, cameras=[cam], sh_degree=deg, render_mode=mode)
    out = imgs[0].detach().cpu().numpy().reshape(-1, imgs[0].shape[-1])
    ref = oracle.render_depth(sc, cam)
    zmax = float(ref["splats"]["depths"].max())
    alpha = alphas[0].detach().cpu().numpy().reshape(-1)
    if mode.startswith("RGB"):
        np.testing.assert_array_less(np.abs(out[:, :3] - ref["color"]).mean(), IMG_MEANABS)
    dep = out[:, -1]
    if mode.endswith("ED"):
        well = ref["alpha"] >= 1e-2  # E = A / alpha is ill-conditioned where alpha is tiny
        _depth_bar(dep, ref["expected_depth"], zmax, mode, mask=well)
    else:
        _depth_bar(dep, ref["acc_depth"], zmax, mode)
    assert np.abs(alpha - ref["alpha"]).max() <= 1e-3


def test_depth_gradients_match_oracle():
    sc, cam = _scene(seed=62, deg=3)
    P = cam.width * cam.height
    leaves, deg = _leaves(sc)
    imgs, alphas, _ = raster.rasterization(*leaves, cameras=[cam], sh_degree=deg, render_mode="RGB+ED")
    ref = oracle.render_depth(sc, cam)
    out = imgs[0].detach().cpu().numpy().reshape(P, 4)
    alpha = alphas[0].detach().cpu().numpy().reshape(P)
    flips = flipped_pixels(out[:, :3], alpha, ref["color"], ref["alpha"])
    rng = np.random.default_rng(63)
    zmax = float(ref["splats"]["depths"].max())
    wc = rng.uniform(-1, 1, (P, 3)) / P
    wE = rng.uniform(-1, 1, P) / (P * zmax)
    wa = rng.uniform(-1, 1, P) / P
    wE[ref["alpha"] < 5e-2] = 0  # keep the expected-depth loss where it is well conditioned
    for w in (wc, wE, wa):
        w[flips] = 0
    up = torch.zeros(P, 4, dtype=torch.float64)
    up[:, :3] = torch.as_tensor(wc)
    up[:, 3] = torch.as_tensor(wE)
    loss = (imgs[0].reshape(P, 4) * up.float().cuda()).sum() + (alphas[0].reshape(P) * torch.as_tensor(
        wa, dtype=torch.float32, device="cuda")).sum()
    g = torch.autograd.grad(loss, leaves)
    g_gpu = {k: v.cpu().numpy() for k, v in zip(["d_means", "d_quats", "d_log_scales", "d_opacity_logits", "d_sh"], g)}
    g_ref = oracle.render_depth_grads(sc, cam, wc, d_expected_depth=wE, d_alpha=wa)
    assert_grad_parity(g_gpu, g_ref)


def test_accumulated_depth_gradient_reaches_the_means():
    """A loss on the accumulated depth alone moves the means (through t_z and the 2D splat)."""
    sc, cam = _scene(seed=64, deg=0)
    P = cam.width * cam.height
    leaves, deg = _leaves(sc)
    imgs, alphas, _ = raster.rasterization(*leaves, cameras=[cam], sh_degree=deg, render_mode="D")
    ref = oracle.render_depth(sc, cam)
    rng = np.random.default_rng(65)
    wA = rng.uniform(-1, 1, P) / P
    alpha = alphas[0].detach().cpu().numpy().reshape(P)
    wA[np.abs(alpha - ref["alpha"]) > 1e-4] = 0  # pixels where a threshold decision flipped
    loss = (imgs[0].reshape(P) * torch.as_tensor(wA, dtype=torch.float32, device="cuda")).sum()
    g = torch.autograd.grad(loss, leaves)
    g_ref = oracle.render_depth_grads(sc, cam, np.zeros((P, 3)), d_acc_depth=wA)
    g_gpu = {k: v.cpu().numpy() for k, v in zip(["d_means", "d_quats", "d_log_scales", "d_opacity_logits", "d_sh"], g)}
    assert_grad_parity(g_gpu, g_ref, keys=("d_means", "d_quats", "d_log_scales", "d_opacity_logits"))
    assert np.abs(g_gpu["d_sh"]).max() == 0.0  # the depth channel does not depend on the colours

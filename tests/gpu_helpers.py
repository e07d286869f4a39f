"""Shared plumbing of the GPU parity tests: move seeded scenes to the device, run the
CUDA path through the C ABI, and compare with the FP64 oracle at the stated bars."""
import numpy as np
import torch

import oracle
from paper_2409_06765_gb300 import _lib, raster, synth

# Bars of the rasterizer's parity contract.
IMG_PIXEL_MAXABS = 1e-3     # per pixel (max over channels) ...
IMG_PIXEL_FRAC = 0.9999     # ... on at least this fraction of pixels
IMG_MEANABS = 1e-5          # mean over all pixel channels
GRAD_REL_L2 = 1e-3          # per parameter group


def dev_scene(scene, device="cuda"):
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a, np.float32), device=device)
    return dict(means=t(scene.means), quats=t(scene.quats), log_scales=t(scene.log_scales),
                opacity_logits=t(scene.opacity_logits), sh=t(scene.sh), sh_degree=scene.sh_degree)


def image_stats(gpu, ref):
    """gpu, ref: [P, ch] arrays.  Returns (fraction of pixels within the per-pixel bar, mean abs, max abs)."""
    d = np.abs(np.asarray(gpu, np.float64) - np.asarray(ref, np.float64))
    per_pixel = d.reshape(d.shape[0], -1).max(axis=1)
    return float((per_pixel <= IMG_PIXEL_MAXABS).mean()), float(d.mean()), float(d.max()), per_pixel


def assert_image_parity(gpu, ref, what="image"):
    frac, mean_abs, max_abs, _ = image_stats(gpu, ref)
    assert frac >= IMG_PIXEL_FRAC, f"{what}: only {frac:.6f} of pixels within {IMG_PIXEL_MAXABS} (max {max_abs})"
    assert mean_abs <= IMG_MEANABS, f"{what}: mean abs {mean_abs} > {IMG_MEANABS}"


def rel_l2(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / max(nb, 1e-30))


def gpu_render(scene, cams, settings=None, state=None):
    d = dev_scene(scene)
    ca = _lib.CameraArray(cams)
    out = raster.forward_pass(ca, d["means"], d["quats"], d["log_scales"], d["opacity_logits"], sh=d["sh"],
                              sh_degree=d["sh_degree"], settings=settings, state=state)
    torch.cuda.synchronize()
    return out, d, ca


def gpu_grads(scene, cams, d_image, d_alpha=None, settings=None):
    """Forward + backward through the autograd wrapper with a given upstream gradient."""
    d = dev_scene(scene)
    leaves = [d["means"], d["quats"], d["log_scales"], d["opacity_logits"], d["sh"]]
    for x in leaves:
        x.requires_grad_(True)
    ca = _lib.CameraArray(cams)
    img, alpha, _, _ = raster.RasterizeGaussians.apply(*leaves, ca, d["sh_degree"], settings or raster.RasterSettings(),
                                                    None)
    outs, grads_in = [img], [torch.as_tensor(np.asarray(d_image, np.float32), device="cuda").reshape(img.shape)]
    if d_alpha is not None:
        outs.append(alpha)
        grads_in.append(torch.as_tensor(np.asarray(d_alpha, np.float32), device="cuda").reshape(alpha.shape))
    g = torch.autograd.grad(outs, leaves, grads_in)
    names = ["d_means", "d_quats", "d_log_scales", "d_opacity_logits", "d_sh"]
    return {k: v.detach().cpu().numpy() for k, v in zip(names, g)}, img.detach().cpu().numpy(), \
        alpha.detach().cpu().numpy()


def assert_grad_parity(gpu, ref, keys=("d_means", "d_quats", "d_log_scales", "d_opacity_logits", "d_sh"),
                       bar=GRAD_REL_L2):
    report = {k: rel_l2(gpu[k], ref[k]) for k in keys}
    bad = {k: v for k, v in report.items() if not v <= bar}
    assert not bad, f"relative L2 above {bar}: {bad} (all: {report})"
    return report


def flipped_pixels(img_gpu, alpha_gpu, img_ref, alpha_ref, tol=1e-4):
    """Pixels where a float32-vs-float64 threshold decision (alpha skip, T cut-off, box edge)
    went differently: the forward values differ by more than rounding."""
    di = np.abs(np.asarray(img_gpu, np.float64) - img_ref).reshape(len(alpha_ref), -1).max(1)
    da = np.abs(np.asarray(alpha_gpu, np.float64).ravel() - np.asarray(alpha_ref).ravel())
    return (di > tol) | (da > tol)

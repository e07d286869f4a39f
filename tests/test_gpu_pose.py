"""Pose gradients (App. A) on the GPU against the oracle: d L / d [R | t] of the
world->camera matrix through the camera-space means, the covariance rotation and the SH
view direction, for one and several cameras."""
import numpy as np
import pytest
import torch

import oracle
from paper_2409_06765_gb300 import raster, synth

from gpu_helpers import dev_scene, flipped_pixels, rel_l2

pytestmark = pytest.mark.gpu


def _run(sc, cams, seed, antialiased=False):
    d = dev_scene(sc)
    leaves = [d[k].clone().requires_grad_(True) for k in ("means", "quats", "log_scales", "opacity_logits", "sh")]
    vm = torch.tensor(np.stack([c.viewmat for c in cams]), dtype=torch.float32, requires_grad=True)
    settings = raster.RasterSettings(antialiased=antialiased)
    imgs, alphas, _ = raster.rasterization(*leaves, cameras=cams, sh_degree=d["sh_degree"], settings=settings,
                                           viewmats=vm)
    rng = np.random.default_rng(seed)
    loss = 0.0
    refs = []
    for cam, img, alpha in zip(cams, imgs, alphas):
        P = cam.width * cam.height
        ref = oracle.render(sc, cam, antialiased=antialiased)
        flips = flipped_pixels(img.detach().cpu().numpy().reshape(P, 3), alpha.detach().cpu().numpy().reshape(P),
                               ref["image"].reshape(P, 3), ref["alpha"].reshape(P))
        w = rng.uniform(-1, 1, (P, 3)) / P
        wa = rng.uniform(-1, 1, P) / P
        w[flips] = 0
        wa[flips] = 0
        refs.append(oracle.render_grads(sc, cam, w, d_alpha=wa, antialiased=antialiased))
        loss = loss + (img.reshape(P, 3) * torch.as_tensor(w, dtype=torch.float32, device="cuda")).sum() + \
            (alpha.reshape(P) * torch.as_tensor(wa, dtype=torch.float32, device="cuda")).sum()
    loss.backward()
    return vm.grad.numpy(), refs, leaves


@pytest.mark.parametrize("deg,aa", [(0, False), (2, False), (3, True)])
def test_pose_gradient_matches_oracle(deg, aa):
    sc = synth.clustered_scene(7000, 81 + deg, sh_degree=deg, log_scale_mu=-3.2)
    cams = synth.sphere_cameras(81 + deg, [(144, 112)])
    g, refs, _ = _run(sc, cams, 82 + deg, antialiased=aa)
    assert g.shape == (1, 4, 4) and np.all(g[0, 3] == 0)
    err = rel_l2(g[0, :3], refs[0]["d_viewmat"][:3])
    assert err <= 1e-3, err


def test_pose_gradients_of_several_cameras():
    sc = synth.clustered_scene(9000, 85, sh_degree=3, log_scale_mu=-3.2)
    cams = synth.sphere_cameras(85, [(96, 64), (120, 90), (64, 96)])
    g, refs, leaves = _run(sc, cams, 86)
    for c in range(len(cams)):
        err = rel_l2(g[c, :3], refs[c]["d_viewmat"][:3])
        assert err <= 1e-3, (c, err)
    # the leaves' gradients still sum over the cameras
    d_means = sum(r["d_means"] for r in refs)
    assert rel_l2(leaves[0].grad.cpu().numpy(), d_means) <= 1e-3

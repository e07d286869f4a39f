"""Parity at the full benchmark sizes, in the launch configuration bench.py times.

The oracle cannot render 2 M pixels over 3 M Gaussians by brute force in a test, so it
renders a seeded uniform sample of pixels; the backward uses an upstream gradient that is
non-zero only at those pixels, which makes the GPU's full-image backward equal to the
gradient of the sampled loss that the oracle computes exactly.  The intersection lists are
compared bit for bit with the oracle's enumeration fed the GPU's float32 splats.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2409_06765_gb300 import synth
from paper_2409_06765_gb300.pipeline import DeviceScene, FramePipeline, Schedule

from gpu_helpers import IMG_MEANABS, IMG_PIXEL_MAXABS, assert_grad_parity, flipped_pixels

pytestmark = pytest.mark.gpu

# (workload, schedule): the schedule the autotuner picks for the headline on a GB300 (tile 32; forward
# 4 px/thread x 512, backward 4 x 1024), a tile-16 schedule, and the training-step workload's pick
CASES = [
    ("headline_3M_1080p", Schedule(tile=32, batch_depth=512, pixels_per_thread=4, bwd_batch_depth=1024,
                                   bwd_pixels_per_thread=4)),
    ("headline_3M_1080p", Schedule(tile=16, batch_depth=128, pixels_per_thread=2)),
    ("training_step_1M_1297x840", Schedule(tile=16, batch_depth=256, pixels_per_thread=2)),
]
SAMPLES = 2048


def _workload(name):
    if name.startswith("headline"):
        scene, cam, _ = synth.headline_workload()
    else:
        scene, cam, _ = synth.training_step_workload()
    return scene, cam


_scene_cache = {}


def _scene(name):
    if name not in _scene_cache:
        _scene_cache.clear()
        scene, cam = _workload(name)
        _scene_cache[name] = (scene, cam, oracle.project(scene, cam), oracle.sh_colors(scene, cam)[0])
    return _scene_cache[name]


@pytest.mark.parametrize("name,sched", CASES, ids=[f"{n}-t{s.tile}p{s.pixels_per_thread}b{s.batch_depth}"
                                                   for n, s in CASES])
def test_full_size_forward_backward_and_lists(name, sched):
    scene, cam, sp, colors = _scene(name)
    P = cam.width * cam.height
    ds = DeviceScene.from_host(scene)
    pipe = FramePipeline(ds, [cam], sched)
    pipe.forward(graphs=True)
    torch.cuda.synchronize()
    assert not pipe.frame_overflowed()

    # forward at sampled pixels
    rng = np.random.default_rng(77)
    pix = np.sort(rng.choice(P, SAMPLES, replace=False)).astype(np.int32)
    ref = oracle.render_splats(sp, colors, cam.width, cam.height, pixels=pix)
    img = pipe.image.cpu().numpy()[pix]
    alpha = 1.0 - pipe.final_T.cpu().numpy()[pix]
    d = np.abs(img.astype(np.float64) - ref["color"]).max(1)
    bad = int((d > IMG_PIXEL_MAXABS).sum())
    # >= 99.99 % of pixels within the bar: a sample of 2048 may hold at most a couple of flips
    assert bad <= 2, f"{bad} of {SAMPLES} sampled pixels above {IMG_PIXEL_MAXABS}"
    assert np.abs(img.astype(np.float64) - ref["color"]).mean() <= IMG_MEANABS
    assert np.abs(alpha - (1.0 - ref["T"])).max() <= 1e-3 or bad > 0

    # intersection lists: bit-exact against the oracle's enumeration of the GPU's splats
    m2 = pipe.means2d.cpu().numpy()
    dep = pipe.depths.cpu().numpy()
    rad = pipe.radii.cpu().numpy()
    keys, values, ranges = oracle.bin_sort(m2, dep, rad, [cam.width], [cam.height], sched.tile)
    K = pipe.K
    assert K == len(values)
    np.testing.assert_array_equal(pipe.values[:K].cpu().numpy(), values)
    np.testing.assert_array_equal(pipe.ranges.cpu().numpy(), ranges)

    # backward of a loss on the sampled pixels only (flipped pixels left out)
    flips = flipped_pixels(img, alpha, ref["color"], 1.0 - ref["T"])
    keep = pix[~flips]
    g = rng.normal(0.0, 1.0, (len(keep), 3))
    d_full = torch.zeros(P, 3, device="cuda")
    d_full[torch.as_tensor(keep.astype(np.int64), device="cuda")] = torch.as_tensor(g, dtype=torch.float32,
                                                                                   device="cuda")
    pipe.d_image.copy_(d_full)
    pipe.backward(graphs=True)
    torch.cuda.synchronize()
    g_gpu = dict(d_means=pipe.d_means.cpu().numpy(), d_quats=pipe.d_quats.cpu().numpy(),
                 d_log_scales=pipe.d_log_scales.cpu().numpy(), d_opacity_logits=pipe.d_logits.cpu().numpy(),
                 d_sh=pipe.d_sh.cpu().numpy())
    g_ref = oracle.render_grads(scene, cam, g, pixels=keep)
    assert_grad_parity(g_gpu, g_ref)


# --------------------------------------------------------------------------- #
# multi-camera workloads at full size: 16 views of mixed resolution, and 6M    #
# Gaussians seen by four 1080p views, in the schedules bench.py times          #
# --------------------------------------------------------------------------- #

MULTI_CASES = [
    # (workload, schedule, cameras checked forward, cameras whose lists are compared, cameras in the loss)
    ("multiview_3M_16views",
     Schedule(tile=32, batch_depth=512, pixels_per_thread=4, bwd_batch_depth=1024, bwd_pixels_per_thread=4),
     (0, 5, 10, 15), (0, 5, 10), (5, 15)),
    ("memory_6M_4x1080p",
     Schedule(tile=32, batch_depth=1024, pixels_per_thread=2, bwd_batch_depth=1024, bwd_pixels_per_thread=4),
     (0, 3), (3,), (0,)),
]
SAMPLES_PER_VIEW = 256


def _multi_workload(name):
    if name.startswith("multiview"):
        return synth.multiview_workload()
    return synth.memory_workload()


def _camera_slices(cams, tile):
    """Per camera: (pixel offset, first global tile, tile count)."""
    out, pix, t0 = [], 0, 0
    for cam in cams:
        T = ((cam.width + tile - 1) // tile) * ((cam.height + tile - 1) // tile)
        out.append((pix, t0, T))
        pix += cam.width * cam.height
        t0 += T
    return out


@pytest.mark.parametrize("name,sched,fwd_cams,list_cams,loss_cams", MULTI_CASES, ids=[c[0] for c in MULTI_CASES])
def test_full_size_multi_view_forward_backward_and_lists(name, sched, fwd_cams, list_cams, loss_cams):
    _scene_cache.clear()
    scene, cams = _multi_workload(name)
    N = scene.means.shape[0]
    ds = DeviceScene.from_host(scene)
    pipe = FramePipeline(ds, cams, sched)
    pipe.forward(graphs=True)
    torch.cuda.synchronize()
    assert not pipe.frame_overflowed()
    slices = _camera_slices(cams, sched.tile)
    image = pipe.image.cpu().numpy()
    final_T = pipe.final_T.cpu().numpy()
    rng = np.random.default_rng(78)

    # forward at sampled pixels of each checked camera
    keep = {}
    for c in fwd_cams:
        cam = cams[c]
        pix0 = slices[c][0]
        pix = np.sort(rng.choice(cam.width * cam.height, SAMPLES_PER_VIEW, replace=False)).astype(np.int32)
        ref = oracle.render(scene, cam, pixels=pix)
        img = image[pix0 + pix]
        alpha = 1.0 - final_T[pix0 + pix]
        d = np.abs(img.astype(np.float64) - ref["image"]).max(1)
        bad = int((d > IMG_PIXEL_MAXABS).sum())
        assert bad <= 1, f"camera {c}: {bad} of {SAMPLES_PER_VIEW} sampled pixels above {IMG_PIXEL_MAXABS}"
        assert np.abs(img.astype(np.float64) - ref["image"]).mean() <= IMG_MEANABS, f"camera {c}"
        flips = flipped_pixels(img, alpha, ref["image"], ref["alpha"])
        keep[c] = pix[~flips]

    # intersection lists of single cameras: bit-exact against the oracle's enumeration of the
    # GPU's splats of that camera (global tile ids and pair indices c*N + n shifted back)
    ranges = pipe.ranges.cpu().numpy()
    m2 = pipe.means2d.cpu().numpy()
    dep = pipe.depths.cpu().numpy()
    rad = pipe.radii.cpu().numpy()
    for c in list_cams:
        cam = cams[c]
        _, t0, T = slices[c]
        _, values, ref_ranges = oracle.bin_sort(m2[c:c + 1], dep[c:c + 1], rad[c:c + 1], [cam.width], [cam.height],
                                                sched.tile)
        rg = ranges[t0:t0 + T]
        nonempty = rg[:, 1] > rg[:, 0]
        np.testing.assert_array_equal(nonempty, ref_ranges[:, 1] > ref_ranges[:, 0])
        first = int(rg[nonempty, 0].min()) if nonempty.any() else 0
        last = int(rg[nonempty, 1].max()) if nonempty.any() else 0
        assert last - first == len(values), f"camera {c}"
        np.testing.assert_array_equal(rg[nonempty] - first, ref_ranges[nonempty])
        np.testing.assert_array_equal(pipe.values[first:last].cpu().numpy() - c * N, values)

    # backward of a loss on the kept sampled pixels of the loss cameras (all views composited)
    d_full = torch.zeros(pipe.P, 3, device="cuda")
    g_ref = None
    for c in loss_cams:
        pix0 = slices[c][0]
        g = rng.normal(0.0, 1.0, (len(keep[c]), 3))
        idx = torch.as_tensor((pix0 + keep[c]).astype(np.int64), device="cuda")
        d_full[idx] = torch.as_tensor(g, dtype=torch.float32, device="cuda")
        r = oracle.render_grads(scene, cams[c], g, pixels=keep[c])
        if g_ref is None:
            g_ref = {k: r[k] for k in ("d_means", "d_quats", "d_log_scales", "d_opacity_logits", "d_sh")}
        else:
            for k in g_ref:
                g_ref[k] = g_ref[k] + r[k]
    pipe.d_image.copy_(d_full)
    pipe.backward(graphs=True)
    torch.cuda.synchronize()
    g_gpu = dict(d_means=pipe.d_means.cpu().numpy(), d_quats=pipe.d_quats.cpu().numpy(),
                 d_log_scales=pipe.d_log_scales.cpu().numpy(), d_opacity_logits=pipe.d_logits.cpu().numpy(),
                 d_sh=pipe.d_sh.cpu().numpy())
    assert_grad_parity(g_gpu, g_ref)

"""Batched multi-view rendering, the schedule autotuner, the serving loop and the memory
footprint of the backward, on the GPU."""
import numpy as np
import pytest
import torch

import oracle
from paper_2409_06765_gb300 import autotune, serve, synth
from paper_2409_06765_gb300.pipeline import DeviceScene, FramePipeline, Schedule

from gpu_helpers import assert_image_parity

pytestmark = pytest.mark.gpu


def _alone(ds, cam, sched=Schedule()):
    p = FramePipeline(ds, [cam], sched, backward=False)
    p.forward()
    torch.cuda.synchronize()
    return p.image.cpu().numpy().reshape(cam.height, cam.width, 3)


def test_each_view_of_a_batch_equals_the_view_alone():
    sc = synth.clustered_scene(12000, 31, sh_degree=2, log_scale_mu=-3.3)
    ds = DeviceScene.from_host(sc)
    cams = synth.sphere_cameras(31, [(96, 64), (200, 120), (64, 64), (333, 201)])
    p = FramePipeline(ds, cams, Schedule(), backward=False)
    p.forward()
    torch.cuda.synchronize()
    img = p.image.cpu().numpy()
    for cam, off in zip(cams, p.cams.pixel_offsets()):
        P = cam.width * cam.height
        np.testing.assert_array_equal(img[off:off + P].reshape(cam.height, cam.width, 3), _alone(ds, cam))


def test_autotuner_times_every_candidate_and_caches_the_winner():
    sc = synth.clustered_scene(6000, 32, sh_degree=1, log_scale_mu=-3.3)
    ds = DeviceScene.from_host(sc)
    cams = synth.sphere_cameras(32, [(160, 96), (96, 160)])
    res = autotune.tune(ds, cams, backward=True, reps=1, use_cache=False)
    per_kernel = [r for r in res.table if r["phase"] in ("fwd", "bwd")]
    n_shapes = sum(len(v) for v in autotune.TILE_SHAPES.values())
    assert len(per_kernel) == 2 * n_shapes * len(autotune.BATCH_DEPTHS) * 2  # x one-CTA-per-tile / persistent
    totals = [r["ms"] for r in res.table if r["phase"] == "total" and r["ms"] is not None]
    assert totals and res.best_ms == min(totals)
    # a tile size's total is its fixed stages plus its fastest forward and backward
    for t in autotune.TILE_SHAPES:
        tot = [r for r in res.table if r["phase"] == "total" and r["tile"] == t][0]
        f = min(r["ms"] for r in per_kernel if r["tile"] == t and r["phase"] == "fwd")
        b = min(r["ms"] for r in per_kernel if r["tile"] == t and r["phase"] == "bwd")
        assert abs(tot["ms"] - (tot["fixed_ms"] + f + b)) < 1e-9
    again = autotune.tune(ds, cams, backward=True, reps=1)
    assert autotune.tune(ds, cams, backward=True) is again  # cached by signature
    # the winner renders what the default schedule renders
    for cam in cams:
        np.testing.assert_array_equal(_alone(ds, cam, res.best), _alone(ds, cam))


def _store(seeds=(41, 42, 43), sizes=(4000, 9000, 15000)):
    store = serve.ResidentScenes(reserve_bytes=256 << 20)
    hosts = {}
    for sid, (seed, n) in enumerate(zip(seeds, sizes)):
        hosts[sid] = synth.clustered_scene(n, seed, sh_degree=1, log_scale_mu=-3.3)
        store.add(sid, hosts[sid], calib_camera=synth.sphere_cameras(seed, [(128, 96)])[0])
    return store, hosts


def _trace(n=24, seed=44):
    sizes = [(96, 64), (128, 96), (200, 120)]
    return serve.poisson_trace(2000.0, n / 2000.0, 3, seed=seed, sizes=sizes)


def test_served_images_are_the_same_alone_and_in_the_mix():
    store, hosts = _store()
    trace = _trace()
    assert len(trace) >= 10
    srv = serve.Server(store, max_views=4, streams=3)
    out = {r.rid: r for r in srv.serve(trace, realtime=False)}
    assert sorted(out) == sorted(r.rid for r in trace)
    assert max(r.batch_views for r in out.values()) > 1, "the trace never produced a batch"
    for req in trace:
        alone = _alone(store.scenes[req.scene], req.camera)
        np.testing.assert_array_equal(out[req.rid].image, alone)
    # and the served image is the oracle's image within the parity bars
    req = trace[0]
    ref = oracle.render(hosts[req.scene], req.camera)
    assert_image_parity(out[req.rid].image.reshape(-1, 3), ref["image"].reshape(-1, 3))


def test_a_batch_of_several_scenes_renders_each_view_as_alone():
    """With cross-scene groups allowed, requests of three scenes queued together form one batch
    (one multi-camera call per scene group on one stream); every image equals the view
    rendered alone."""
    store, _ = _store()
    cams = synth.sphere_cameras(47, [(96, 64), (128, 96), (200, 120), (64, 48), (150, 90)])
    trace = [serve.Request(i, i % 3, cam, 0.001 * i) for i, cam in enumerate(cams)]
    srv = serve.Server(store, max_views=8, streams=1, max_groups=3)
    res = srv.serve(trace, realtime=False)
    assert len(res) == len(trace) and srv.batches == 1 and srv.groups == 3
    assert {r.batch for r in res} == {1} and all(r.batch_views == len(trace) for r in res)
    s = serve.latency_summary(res)
    assert s["mean_views_per_batch"] == len(trace) and s["mean_scenes_per_batch"] == 3
    for r in res:
        req = trace[r.rid]
        np.testing.assert_array_equal(r.image, _alone(store.scenes[req.scene], req.camera))


def test_unbatched_path_and_realtime_loop_give_the_same_images():
    store, _ = _store()
    trace = _trace(n=12, seed=45)
    batched = {r.rid: r.image for r in serve.Server(store, max_views=8, streams=2).serve(trace, realtime=True)}
    single = serve.Server(store, max_views=1, streams=1)
    plain = {r.rid: r for r in single.serve(trace, realtime=True)}
    assert all(r.batch_views == 1 for r in plain.values())
    for rid, img in batched.items():
        np.testing.assert_array_equal(img, plain[rid].image)
    s = serve.latency_summary(list(plain.values()))
    assert s["requests"] == len(trace) and s["p99_ms"] >= s["p50_ms"] > 0


def test_memory_budget_limits_what_is_in_flight():
    store, _ = _store()
    cams = synth.sphere_cameras(46, [(128, 96)] * 10)
    trace = [serve.Request(i, 2, cam, 0.0) for i, cam in enumerate(cams)]  # one scene, one size
    srv = serve.Server(store, max_views=8, streams=4)
    one = max(srv._estimate(r.scene, [r]) for r in trace)
    assert srv._estimate(2, trace[:2]) > 1.2 * one
    tight = serve.Server(store, max_views=8, streams=4, budget_bytes=int(one * 1.2))
    res = tight.serve(trace, realtime=False)
    assert len(res) == len(trace)
    assert all(r.batch_views == 1 for r in res), "a batch larger than the budget was admitted"
    assert tight.batches - tight.overflows == len(trace)
    free = serve.Server(store, max_views=8, streams=4).serve(trace, realtime=False)
    assert max(r.batch_views for r in free) > 1


def test_backward_memory_holds_no_per_blend_state():
    """Two scenes of the same size, one nearly transparent and one with many opaque
    Gaussians, differ by several times in blends; the pipeline's buffers differ only by the
    intersection-list term (K), never by anything proportional to blends."""
    cam = synth.sphere_cameras(47, [(256, 192)])[0]
    a = synth.clustered_scene(30000, 47, sh_degree=1, log_scale_mu=-3.0, logit_sigma=0.5)
    b = synth.clustered_scene(30000, 47, sh_degree=1, log_scale_mu=-3.0, logit_sigma=0.5, opaque_frac=0.5)
    pa = FramePipeline(DeviceScene.from_host(a), [cam], Schedule(), capacity=1 << 20)
    pb = FramePipeline(DeviceScene.from_host(b), [cam], Schedule(), capacity=1 << 20)
    assert pa.device_bytes == pb.device_bytes  # same N, pixels and capacity
    ba, bb = pa.count_blends(), pb.count_blends()
    assert ba != bb
    N, P = 30000, 256 * 192
    per_gauss = 4 * (3 + 4 + 3 + 1 + 12)   # gradient leaves (SH degree 1: 4 x 3 coefficients)
    per_pair = 4 * (2 + 1 + 3 + 1 + 1 + 1 + 3) + 4 * 9  # 2D outputs + 2D gradients
    per_pixel = 4 * (3 + 1 + 1 + 3)        # image, final T, last contributor, dL/dimage
    fixed = pa.device_bytes - (pa.values.numel() * 4 + pa.workspace.numel())
    assert fixed <= N * (per_gauss + per_pair) + P * per_pixel + 64 * 1024


def test_deferred_count_check_redoes_a_frame_that_outgrew_the_buffers():
    import torch as _t
    from paper_2409_06765_gb300 import raster
    sc = synth.clustered_scene(20000, 48, sh_degree=1, log_scale_mu=-3.2)
    cam = synth.sphere_cameras(48, [(200, 150)])[0]
    ds = DeviceScene.from_host(sc)
    leaves = [ds.means, ds.quats, ds.log_scales, ds.opacity_logits, ds.sh]
    ref = raster.rasterization(*leaves, cameras=[cam])[0][0].cpu().numpy()
    state = raster.RasterState()
    state.capacity = 1024  # far below this frame's intersection count
    state.values = _t.empty(1024, dtype=_t.int32, device="cuda")
    raster.rasterization(*leaves, cameras=[cam], state=state, defer_sync=True)
    _t.cuda.synchronize()
    assert state.check() is False and state.capacity > 1024 and state.redone == 1
    img = raster.rasterization(*leaves, cameras=[cam], state=state, defer_sync=True)[0][0].cpu().numpy()
    assert state.check() is True
    np.testing.assert_array_equal(img, ref)


def test_images_handed_to_a_callback_equal_the_kept_copies():
    """Without keep_images the results hold no image; on_image sees each one as a view into the
    stream's page-locked buffer while it is valid, equal to the copy a keeping server returns."""
    store, _ = _store()
    trace = _trace(n=10, seed=49)
    kept = {r.rid: r.image for r in serve.Server(store, max_views=8, streams=2).serve(trace, realtime=False)}
    seen = {}
    res = serve.Server(store, max_views=8, streams=2).serve(
        trace, realtime=False, keep_images=False, on_image=lambda r, view: seen.__setitem__(r.rid, view.copy()))
    assert len(res) == len(trace) and all(r.image is None for r in res)
    assert set(seen) == set(kept)
    for rid, img in kept.items():
        np.testing.assert_array_equal(seen[rid], img)

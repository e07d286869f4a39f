"""Parity of every CUDA stage with the FP64 oracle, through the C ABI, at sizes the oracle
finishes in seconds (several tiles, ragged image edges, multiple cameras)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2409_06765_gb300 import _lib, raster, synth

import special_scenes
from gpu_helpers import (IMG_MEANABS, assert_grad_parity, assert_image_parity, dev_scene, flipped_pixels, gpu_grads,
                         gpu_render, image_stats, rel_l2)

pytestmark = pytest.mark.gpu


def _mid_scene(n=20000, seed=7, deg=3):
    sc = synth.clustered_scene(n, seed, sh_degree=deg, log_scale_mu=-3.2)
    cam = synth.sphere_cameras(seed, [(203, 157)])[0]
    return sc, cam


# --------------------------------------------------------------------------- #
# projection and SH                                                           #
# --------------------------------------------------------------------------- #

@pytest.mark.parametrize("aa", [False, True])
def test_project_matches_oracle(aa):
    sc, cam = _mid_scene()
    out, _, _ = gpu_render(sc, [cam], settings=raster.RasterSettings(antialiased=aa))
    ref = oracle.project(sc, cam, antialiased=aa)
    r_gpu = out["radii"][0].cpu().numpy()
    r_ref = ref["radii"]
    both = (r_gpu > 0) & (r_ref > 0)
    assert both.sum() > 0.5 * (r_ref > 0).sum()
    mismatch = (r_gpu != r_ref)
    assert mismatch.sum() <= max(2, 1e-3 * len(r_ref)), mismatch.sum()
    assert np.abs(r_gpu[both] - r_ref[both]).max() <= 1
    m = out["means2d"][0].cpu().numpy()[both]
    np.testing.assert_allclose(m, ref["means2d"][both], atol=2e-3, rtol=0)
    np.testing.assert_allclose(out["depths"][0].cpu().numpy()[both], ref["depths"][both], rtol=2e-6)
    con = out["conics"][0].cpu().numpy()[both]
    scale = np.abs(ref["conics"][both]).max(1, keepdims=True)
    assert (np.abs(con - ref["conics"][both]) / scale).max() < 2e-4
    # anti-aliased opacity carries sqrt(det(S')/det(S'+sI)): float32 cancellation in ac - b^2 scales its
    # error by the condition number of S', so it gets a relative bar
    np.testing.assert_allclose(out["opacities"][0].cpu().numpy()[both], ref["opacities"][both],
                               atol=2e-6, rtol=5e-5 if aa else 0)
    # tiles_touched agrees with the pixel box of the projected (float32) mean
    tt = out["tiles_touched"][0].cpu().numpy()
    assert (tt[r_gpu == 0] == 0).all() and (tt[r_gpu > 0] > 0).all()


@pytest.mark.parametrize("deg", [0, 1, 2, 3])
def test_sh_matches_oracle(deg):
    sc, cam = _mid_scene(n=5000, seed=deg, deg=deg)
    out, _, _ = gpu_render(sc, [cam])
    col, _ = oracle.sh_colors(sc, cam)
    vis = out["radii"][0].cpu().numpy() > 0
    np.testing.assert_allclose(out["colors"][0].cpu().numpy()[vis], col[vis], atol=3e-6, rtol=1e-5)
    assert (out["colors"][0].cpu().numpy()[~vis] == 0).all()


def _fused_project_sh(sc, cams, aa=False):
    """gs_project_sh_eval (one kernel) beside gs_project + gs_sh_eval (two), same inputs."""
    d = dev_scene(sc)
    ca = _lib.CameraArray(cams)
    p = _lib.make_params(tile=16, antialiased=aa)
    C, N = len(cams), d["means"].shape[0]
    outs = []
    for fused in (True, False):
        full = lambda *shape, dt=torch.float32: torch.full(shape, 7, dtype=dt, device="cuda")
        o = dict(means2d=full(C, N, 2), depths=full(C, N), conics=full(C, N, 3), radii=full(C, N, dt=torch.int32),
                 tiles=full(C, N, dt=torch.int32), opac=full(C, N), colors=full(C, N, 3))
        if fused:
            _lib.gs_project_sh_eval(ca, p, d["sh_degree"], d["sh"], d["means"], d["quats"], d["log_scales"],
                                    d["opacity_logits"], o["means2d"], o["depths"], o["conics"], o["radii"],
                                    o["tiles"], o["opac"], o["colors"])
        else:
            _lib.gs_project(ca, d["means"], d["quats"], d["log_scales"], d["opacity_logits"], p, o["means2d"],
                            o["depths"], o["conics"], o["radii"], o["tiles"], o["opac"])
            _lib.gs_sh_eval(ca, d["sh_degree"], d["sh"], d["means"], o["radii"], o["colors"])
        torch.cuda.synchronize()
        outs.append({k: v.cpu().numpy() for k, v in o.items()})
    return outs


@pytest.mark.parametrize("deg,aa,ncam", [(0, False, 1), (1, False, 1), (2, True, 1), (3, False, 1), (3, True, 1),
                                         (3, False, 3), (1, True, 2)])
def test_fused_projection_and_sh_match_the_oracle(deg, aa, ncam):
    """Projection and SH colours of C cameras in one kernel (gs_project_sh_eval): the oracle's
    splats and colours within the bars of the separate stages, and the separate calls' results
    (integers equal, floats to rounding); cameras of different sizes see different subsets."""
    sc, _ = _mid_scene(n=7000, seed=20 + deg, deg=deg)
    cams = synth.sphere_cameras(20 + deg, [(203, 157), (96, 140), (150, 64)][:ncam])
    fused, two = _fused_project_sh(sc, cams, aa)
    np.testing.assert_array_equal(fused["radii"], two["radii"])
    np.testing.assert_array_equal(fused["tiles"], two["tiles"])
    for k in ("means2d", "depths", "conics", "opac", "colors"):
        np.testing.assert_allclose(fused[k], two[k], rtol=1e-6, atol=1e-7, err_msg=k)
    for c, cam in enumerate(cams):
        ref = oracle.project(sc, cam, antialiased=aa)
        col, _ = oracle.sh_colors(sc, cam)
        r_gpu, r_ref = fused["radii"][c], ref["radii"]
        both = (r_gpu > 0) & (r_ref > 0)
        assert both.sum() > 0.5 * (r_ref > 0).sum()
        assert (r_gpu != r_ref).sum() <= max(2, 1e-3 * len(r_ref))
        np.testing.assert_allclose(fused["means2d"][c][both], ref["means2d"][both], atol=2e-3, rtol=0)
        np.testing.assert_allclose(fused["depths"][c][both], ref["depths"][both], rtol=2e-6)
        scale = np.abs(ref["conics"][both]).max(1, keepdims=True)
        assert (np.abs(fused["conics"][c][both] - ref["conics"][both]) / scale).max() < 2e-4
        np.testing.assert_allclose(fused["opac"][c][both], ref["opacities"][both], atol=2e-6,
                                   rtol=5e-5 if aa else 0)
        np.testing.assert_allclose(fused["colors"][c][both], col[both], atol=3e-6, rtol=1e-5)
        # invisible pairs: every output zero (the buffers started at 7)
        vis = r_gpu > 0
        for k in ("means2d", "depths", "conics", "opac", "colors", "tiles"):
            assert (fused[k][c][~vis] == 0).all(), k


# --------------------------------------------------------------------------- #
# binning + sorting: bit-exact when fed the oracle's projection               #
# --------------------------------------------------------------------------- #

def _gpu_bin_sort(cams, means2d, depths, radii, tile, capacity=None):
    ca = _lib.CameraArray(cams)
    C, N = depths.shape
    p = _lib.make_params(tile=tile)
    dev = "cuda"
    m = torch.as_tensor(np.ascontiguousarray(means2d, np.float32), device=dev)
    d = torch.as_tensor(np.ascontiguousarray(depths, np.float32), device=dev)
    r = torch.as_tensor(np.ascontiguousarray(radii, np.int32), device=dev)
    Kcap = capacity if capacity is not None else int(32 * C * N + 1024)
    keys = torch.empty(max(Kcap, 1), dtype=torch.int64, device=dev)
    values = torch.empty(max(Kcap, 1), dtype=torch.int32, device=dev)
    T = ca.num_tiles(tile)
    ranges = torch.full((T, 2), -7, dtype=torch.int32, device=dev)
    K_out = torch.zeros(1, dtype=torch.int64, device=dev)
    ws = torch.empty(_lib.gs_tile_bin_sort_workspace(ca, N, p, Kcap), dtype=torch.uint8, device=dev)
    _lib.gs_tile_bin_sort(ca, N, p, m, d, r, Kcap, keys, values, ranges, K_out, ws)
    torch.cuda.synchronize()
    K = int(K_out.item())
    return K, keys[:min(K, Kcap)].cpu().numpy().view(np.uint64), values[:min(K, Kcap)].cpu().numpy(), \
        ranges.cpu().numpy()


@pytest.mark.parametrize("tile", [8, 16, 32])
def test_bin_sort_bit_exact_single_camera(tile):
    sc, cam = _mid_scene(n=30000, seed=11)
    ref = oracle.project(sc, cam)
    m = ref["means2d"].astype(np.float32)[None]
    d = ref["depths"].astype(np.float32)[None]
    r = ref["radii"][None]
    keys_r, vals_r, ranges_r = oracle.bin_sort(m, d, r, [cam.width], [cam.height], tile)
    K, keys, vals, ranges = _gpu_bin_sort([cam], m, d, r, tile)
    assert K == len(keys_r)
    np.testing.assert_array_equal(keys, keys_r)
    np.testing.assert_array_equal(vals, vals_r)
    np.testing.assert_array_equal(ranges, ranges_r)


def test_bin_sort_bit_exact_uneven_cameras_and_ties():
    sc = synth.clustered_scene(8000, 3, sh_degree=0, log_scale_mu=-3.0)
    cams = synth.sphere_cameras(5, [(97, 61), (160, 90), (33, 200)])
    ms, ds, rs = [], [], []
    for cam in cams:
        p = oracle.project(sc, cam)
        ms.append(p["means2d"])
        ds.append(p["depths"])
        rs.append(p["radii"])
    m = np.stack(ms).astype(np.float32)
    d = np.stack(ds).astype(np.float32)
    d[:, ::7] = d[:, 3:4]  # exact depth ties inside tiles
    r = np.stack(rs)
    for tile in (8, 16):
        keys_r, vals_r, ranges_r = oracle.bin_sort(m, d, r, [c.width for c in cams], [c.height for c in cams], tile)
        K, keys, vals, ranges = _gpu_bin_sort(cams, m, d, r, tile)
        assert K == len(keys_r)
        np.testing.assert_array_equal(keys, keys_r)
        np.testing.assert_array_equal(vals, vals_r)
        np.testing.assert_array_equal(ranges, ranges_r)


@pytest.mark.parametrize("lo,hi", [(4.0, 4.0), (5.0, 5.02), (3.0, 9.0), (0.8, 11.2), (0.01, 1000.0)])
def test_bin_sort_bit_exact_over_depth_ranges(lo, hi):
    """Depth ranges that leave different bytes of the depth keys equal: equal depths (only the
    index orders a tile's list), a narrow range (the top two bytes equal), [3, 9], [0.8, 11.2]
    (four binary octaves) and [0.01, 1000] give the oracle's lists."""
    sc, cam = _mid_scene(n=20000, seed=13)
    ref = oracle.project(sc, cam)
    m = ref["means2d"].astype(np.float32)[None]
    r = ref["radii"][None]
    rng = np.random.default_rng(14)
    d = rng.choice(np.linspace(lo, hi, 997), r.shape).astype(np.float32)
    d[0, :2] = (lo, hi)
    d[0, 5::9] = d[0, 4]  # ties
    keys_r, vals_r, ranges_r = oracle.bin_sort(m, d, r, [cam.width], [cam.height], 16)
    K, keys, vals, ranges = _gpu_bin_sort([cam], m, d, r, 16)
    assert K == len(keys_r)
    np.testing.assert_array_equal(keys, keys_r)
    np.testing.assert_array_equal(vals, vals_r)
    np.testing.assert_array_equal(ranges, ranges_r)


def test_bin_sort_capacity_overflow_reports_K_and_stays_in_bounds():
    sc, cam = _mid_scene(n=5000, seed=12)
    ref = oracle.project(sc, cam)
    m, d, r = ref["means2d"].astype(np.float32)[None], ref["depths"].astype(np.float32)[None], ref["radii"][None]
    keys_r, _, _ = oracle.bin_sort(m, d, r, [cam.width], [cam.height], 16)
    K, _, _, _ = _gpu_bin_sort([cam], m, d, r, 16, capacity=len(keys_r) // 3)
    assert K == len(keys_r)


def test_bin_sort_empty_inputs():
    cam = synth.make_camera(40, 30, (0, 0, 4))
    K, _, _, ranges = _gpu_bin_sort([cam], np.zeros((1, 0, 2)), np.zeros((1, 0)), np.zeros((1, 0), np.int32), 16)
    assert K == 0 and (ranges == 0).all()
    # all Gaussians invisible
    K, _, _, ranges = _gpu_bin_sort([cam], np.zeros((1, 50, 2)), np.ones((1, 50)), np.zeros((1, 50), np.int32), 16)
    assert K == 0 and (ranges == 0).all()


# --------------------------------------------------------------------------- #
# forward image                                                                #
# --------------------------------------------------------------------------- #

def test_tiny_config_forward_matches_oracle():
    sc, cam, _ = synth.tiny_scene()
    out, _, _ = gpu_render(sc, [cam])
    ref = oracle.render(sc, cam)
    img = out["image"].cpu().numpy()
    assert_image_parity(img, ref["image"].reshape(-1, 3))
    assert_image_parity((1 - out["final_T"]).cpu().numpy()[:, None], ref["alpha"].reshape(-1, 1), "alpha")
    assert ref["image"].max() > 0.3


@pytest.mark.parametrize("tile", [8, 16, 32])
@pytest.mark.parametrize("batch", [64, 256])
def test_clustered_forward_matches_oracle(tile, batch):
    sc, cam = _mid_scene()
    out, _, _ = gpu_render(sc, [cam], settings=raster.RasterSettings(tile=tile, batch_depth=batch))
    ref = oracle.render(sc, cam)
    assert_image_parity(out["image"].cpu().numpy(), ref["image"].reshape(-1, 3))
    assert_image_parity((1 - out["final_T"]).cpu().numpy()[:, None], ref["alpha"].reshape(-1, 1), "alpha")


SCHEDULES = [(8, 1), (16, 1), (16, 2), (32, 2), (32, 4)]


def test_image_is_bit_identical_across_schedules():
    """The support rule is per pixel, so tile size, pixels per thread and batch depth change
    nothing but the schedule: images, final T and alpha agree bit for bit."""
    sc, cam = _mid_scene(n=10000, seed=3)
    outs = []
    for tile, ppt in SCHEDULES:
        for batch in (64, 256):
            o = gpu_render(sc, [cam], settings=raster.RasterSettings(tile=tile, pixels_per_thread=ppt,
                                                                      batch_depth=batch))[0]
            outs.append((o["image"].cpu().numpy(), o["final_T"].cpu().numpy()))
    for img, T in outs[1:]:
        np.testing.assert_array_equal(img, outs[0][0])
        np.testing.assert_array_equal(T, outs[0][1])


def _bucket(n):
    """Half-octave bucket of a list length (0 for an empty list), as gs_tile_order defines it."""
    if n <= 0:
        return 0
    l = int(n).bit_length() - 1
    return 1 + 2 * l + ((int(n) >> (l - 1)) & 1 if l > 0 else 0)


def test_tile_order_is_a_permutation_longest_first_and_changes_nothing():
    sc = synth.clustered_scene(20000, 12, sh_degree=1, log_scale_mu=-3.3)
    cams = synth.sphere_cameras(12, [(200, 120), (96, 64), (333, 201)])
    plain = gpu_render(sc, cams, settings=raster.RasterSettings(tile_schedule=False))[0]
    ordered = gpu_render(sc, cams, settings=raster.RasterSettings(tile_schedule=True))[0]
    rg = ordered["ranges"].cpu().numpy()
    T = rg.shape[0]
    full = ordered["tile_order"].cpu().numpy()
    assert full.shape[0] == T + 4 and np.all(full[T:] == 0)  # the order, then zeroed work counters
    order = full[:T]
    assert np.array_equal(np.sort(order), np.arange(T))
    lengths = rg[order, 1] - rg[order, 0]
    buckets = np.array([_bucket(n) for n in lengths])
    assert np.all(np.diff(buckets) <= 0), "tiles are not in descending length buckets"
    assert buckets[0] == _bucket((rg[:, 1] - rg[:, 0]).max())  # ties inside a bucket come in any order
    for k in ("image", "final_T", "last_contrib"):
        np.testing.assert_array_equal(plain[k].cpu().numpy(), ordered[k].cpu().numpy())


def test_tile_order_backward_matches_index_order():
    sc = synth.clustered_scene(8000, 13, sh_degree=2, log_scale_mu=-3.3)
    cams = synth.sphere_cameras(13, [(128, 96)])
    rng = np.random.default_rng(13)
    g = rng.normal(size=(128 * 96, 3)).astype(np.float32)
    a = gpu_grads(sc, cams, g, settings=raster.RasterSettings(tile_schedule=False))[0]
    b = gpu_grads(sc, cams, g, settings=raster.RasterSettings(tile_schedule=True))[0]
    for k in a:
        # the atomics add in another order: equal up to float32 rounding
        assert rel_l2(b[k], a[k]) <= 1e-5, k


def test_multi_camera_uneven_sizes_and_background():
    sc = synth.clustered_scene(15000, 9, sh_degree=2, log_scale_mu=-3.3)
    cams = synth.sphere_cameras(9, [(64, 48), (131, 77), (40, 90)])
    bg = (0.1, 0.7, 0.3)
    out, _, ca = gpu_render(sc, cams, settings=raster.RasterSettings(background=bg))
    img = out["image"].cpu().numpy()
    for cam, off in zip(cams, ca.pixel_offsets()):
        ref = oracle.render(sc, cam, bg=np.array(bg))
        P = cam.width * cam.height
        assert_image_parity(img[off:off + P], ref["image"].reshape(-1, 3), f"camera {cam.width}x{cam.height}")


def test_forward_fed_oracle_splats_isolates_compositing():
    """gs_rasterize_fwd on the oracle's (float32-rounded) 2D splats and colours vs the oracle
    compositing of exactly those values promoted to float64."""
    sc, cam = _mid_scene(n=20000, seed=21)
    sp = oracle.project(sc, cam)
    col, _ = oracle.sh_colors(sc, cam)
    f32 = {k: sp[k].astype(np.float32) for k in ("means2d", "depths", "conics", "opacities")}
    sp32 = dict(sp, **{k: v.astype(np.float64) for k, v in f32.items()})
    # recompute the boxes from the float32 means exactly like the kernels
    for n in np.nonzero(sp["radii"] > 0)[0]:
        r = int(sp["radii"][n])
        mx, my = (float(v) for v in f32["means2d"][n])
        x0, x1 = int(np.ceil(mx - r - 0.5)), int(np.floor(mx + r - 0.5))
        y0, y1 = int(np.ceil(my - r - 0.5)), int(np.floor(my + r - 0.5))
        sp32["boxes"][n] = [max(x0, 0), min(x1, cam.width - 1), max(y0, 0), min(y1, cam.height - 1)]
        if sp32["boxes"][n][0] > sp32["boxes"][n][1] or sp32["boxes"][n][2] > sp32["boxes"][n][3]:
            sp32["radii"][n] = 0
    col32 = col.astype(np.float32)
    ref = oracle.render_splats(sp32, col32.astype(np.float64), cam.width, cam.height)
    ca = _lib.CameraArray([cam])
    p = _lib.make_params()
    t = lambda a, dt=torch.float32: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    m, d, r = t(f32["means2d"][None]), t(f32["depths"][None]), t(sp32["radii"][None], torch.int32)
    bs = raster.bin_sort(ca, sc.n, p, m, d, r)
    image, final_T, _, _ = raster.rasterize_fwd(ca, sc.n, p, 3, bs["ranges"], bs["values"], r, m,
                                                t(f32["conics"][None]), t(f32["opacities"][None]), t(col32[None]),
                                                None)
    frac, mean_abs, max_abs, _ = image_stats(image.cpu().numpy(), ref["color"])
    assert frac >= 0.9999 and mean_abs <= 2e-6, (frac, mean_abs, max_abs)
    np.testing.assert_allclose(final_T.cpu().numpy(), ref["T"], atol=5e-4)


def test_blend_count_matches_oracle():
    sc, cam, _ = synth.tiny_scene()
    d = dev_scene(sc)
    ca = _lib.CameraArray([cam])
    out = raster.forward_pass(ca, d["means"], d["quats"], d["log_scales"], d["opacity_logits"], sh=d["sh"],
                              sh_degree=0, count_blends=True)
    ref = oracle.render(sc, cam)
    b_gpu = int(out["blends"].item())
    b_ref = int(ref["blends"].sum())
    assert abs(b_gpu - b_ref) <= 1e-3 * b_ref, (b_gpu, b_ref)


def test_empty_scene_renders_background():
    cam = synth.make_camera(50, 35, (0, 0, 4))
    sc = synth.Scene(np.zeros((0, 3), np.float32), np.zeros((0, 4), np.float32), np.zeros((0, 3), np.float32),
                     np.zeros(0, np.float32), np.zeros((0, 1, 3), np.float32), 0)
    out, _, _ = gpu_render(sc, [cam], settings=raster.RasterSettings(background=(0.2, 0.4, 0.6)))
    img = out["image"].cpu().numpy()
    np.testing.assert_allclose(img, np.tile([0.2, 0.4, 0.6], (50 * 35, 1)), atol=1e-7)
    assert (out["final_T"].cpu().numpy() == 1).all()


def test_all_culled_scene():
    sc, cam = _mid_scene(n=1000, seed=2)
    sc.means[:] = np.asarray(cam.viewmat, np.float64)[:3, :3].T @ np.array([0, 0, -5.0]) - \
        np.asarray(cam.viewmat, np.float64)[:3, :3].T @ np.asarray(cam.viewmat, np.float64)[:3, 3]
    out, _, _ = gpu_render(sc, [cam])
    assert out["K"] == 0
    assert (out["radii"].cpu().numpy() == 0).all()
    assert (out["image"].cpu().numpy() == 0).all()


# --------------------------------------------------------------------------- #
# backward                                                                     #
# --------------------------------------------------------------------------- #

def _masked_upstream(sc, cams_ref_renders, out_img, out_alpha, rng, P):
    d_img = rng.uniform(-1, 1, (P, 3)) / P
    d_alpha = rng.uniform(-1, 1, P) / P
    ref_img, ref_alpha = cams_ref_renders
    flips = flipped_pixels(out_img, out_alpha, ref_img, ref_alpha)
    assert flips.mean() <= 1e-4 or flips.sum() <= 1, f"{flips.sum()} threshold flips"
    d_img[flips] = 0
    d_alpha[flips] = 0
    return d_img, d_alpha, int(flips.sum())


@pytest.mark.parametrize("deg,aa,tile,ppt", [(0, False, 16, 0), (3, False, 16, 0), (3, True, 16, 0),
                                             (3, False, 8, 1), (3, False, 16, 2), (3, False, 32, 2),
                                             (3, False, 32, 4)])
def test_backward_matches_oracle(deg, aa, tile, ppt):
    sc, cam = _mid_scene(n=8000, seed=31 + deg, deg=deg)
    settings = raster.RasterSettings(antialiased=aa, background=(0.3, 0.2, 0.1), tile=tile, pixels_per_thread=ppt)
    bg = np.array([0.3, 0.2, 0.1])
    ref_f = oracle.render(sc, cam, bg=bg, antialiased=aa)
    P = cam.width * cam.height
    rng = np.random.default_rng(5)
    out, _, _ = gpu_render(sc, [cam], settings=settings)
    d_img, d_alpha, nflip = _masked_upstream(sc, (ref_f["image"].reshape(P, 3), ref_f["alpha"].reshape(P)),
                                             out["image"].cpu().numpy(), (1 - out["final_T"]).cpu().numpy(), rng, P)
    g_gpu, _, _ = gpu_grads(sc, [cam], d_img, d_alpha, settings=settings)
    g_ref = oracle.render_grads(sc, cam, d_img, d_alpha=d_alpha, bg=bg, antialiased=aa)
    assert_grad_parity(g_gpu, g_ref)


def test_tiny_config_l1_loss_backward():
    """Config 1: forward + backward of the mean L1 loss against a U[0,1] target."""
    sc, cam, target = synth.tiny_scene()
    out, _, _ = gpu_render(sc, [cam])
    img = out["image"].cpu().numpy().reshape(64, 64, 3)
    ref_f = oracle.render(sc, cam)
    flips = flipped_pixels(img.reshape(-1, 3), (1 - out["final_T"]).cpu().numpy(), ref_f["image"].reshape(-1, 3),
                           ref_f["alpha"].reshape(-1))
    d_img = (np.sign(img - target) / img.size).reshape(-1, 3)
    d_img[flips] = 0
    g_gpu, _, _ = gpu_grads(sc, [cam], d_img)
    g_ref = oracle.render_grads(sc, cam, d_img)
    assert_grad_parity(g_gpu, g_ref)


def test_backward_multi_camera_sums_over_views():
    sc = synth.clustered_scene(6000, 17, sh_degree=1, log_scale_mu=-3.2)
    cams = synth.sphere_cameras(17, [(96, 64), (57, 80)])
    rng = np.random.default_rng(3)
    out, _, ca = gpu_render(sc, cams)
    img = out["image"].cpu().numpy()
    alpha = (1 - out["final_T"]).cpu().numpy()
    d_img = np.zeros_like(img, dtype=np.float64)
    g_ref = None
    for cam, off in zip(cams, ca.pixel_offsets()):
        P = cam.width * cam.height
        ref_f = oracle.render(sc, cam)
        di, _, _ = _masked_upstream(sc, (ref_f["image"].reshape(P, 3), ref_f["alpha"].reshape(P)), img[off:off + P],
                                    alpha[off:off + P], rng, P)
        d_img[off:off + P] = di
        g = oracle.render_grads(sc, cam, di)
        g_ref = g if g_ref is None else {k: g_ref[k] + g[k] for k in g_ref if k.startswith("d_")}
    g_gpu, _, _ = gpu_grads(sc, cams, d_img)
    assert_grad_parity(g_gpu, g_ref)


def test_unequal_focal_lengths_and_principal_point():
    """fx != fy and cx != cy (App. E intrinsics): x must use only fx, cx and y only fy, cy, in
    the projection, the compositing and the backward."""
    sc = synth.clustered_scene(8000, 41, sh_degree=3, log_scale_mu=-3.2)
    base = synth.sphere_cameras(41, [(203, 157)])[0]
    f32 = lambda v: float(np.float32(v))
    cam = synth.Camera(base.width, base.height, base.viewmat, f32(base.fx * 1.25), f32(base.fy * 0.8),
                       f32(base.cx + 9.0), f32(base.cy - 6.0))
    bg = np.array([0.3, 0.2, 0.1])
    settings = raster.RasterSettings(background=(0.3, 0.2, 0.1))
    out, _, _ = gpu_render(sc, [cam], settings=settings)
    ref_p = oracle.project(sc, cam)
    both = (out["radii"][0].cpu().numpy() > 0) & (ref_p["radii"] > 0)
    assert both.sum() > 0.5 * (ref_p["radii"] > 0).sum()
    np.testing.assert_allclose(out["means2d"][0].cpu().numpy()[both], ref_p["means2d"][both], atol=2e-3, rtol=0)
    P = cam.width * cam.height
    ref_f = oracle.render(sc, cam, bg=bg)
    assert_image_parity(out["image"].cpu().numpy(), ref_f["image"].reshape(P, 3))
    rng = np.random.default_rng(5)
    d_img, d_alpha, _ = _masked_upstream(sc, (ref_f["image"].reshape(P, 3), ref_f["alpha"].reshape(P)),
                                         out["image"].cpu().numpy(), (1 - out["final_T"]).cpu().numpy(), rng, P)
    g_gpu, _, _ = gpu_grads(sc, [cam], d_img, d_alpha, settings=settings)
    g_ref = oracle.render_grads(sc, cam, d_img, d_alpha=d_alpha, bg=bg)
    assert_grad_parity(g_gpu, g_ref)


def test_clamped_alpha_passes_no_gradient_on_the_gpu():
    """App. C.2 cap alpha = min(alpha_max, o~ e^-sigma): where it is active the pixel does not move with
    the opacity, mean or covariance, so the backward must send nothing through alpha there."""
    sc, cam = special_scenes.clamp_scene()
    bg = np.array([0.3, 0.2, 0.1])
    settings = raster.RasterSettings(background=(0.3, 0.2, 0.1))
    # the scene's premise (half of the Gaussians capped at their centre pixel) is a property of
    # the oracle alone, also checked on the CPU
    clamped, ref_f = special_scenes.clamped_pairs(oracle, sc, cam, bg)
    assert clamped == sc.n // 2
    sp = ref_f["splats"]
    P = cam.width * cam.height
    out, _, _ = gpu_render(sc, [cam], settings=settings)
    assert_image_parity(out["image"].cpu().numpy(), ref_f["image"].reshape(P, 3))
    # upstream gradient on the 3 x 3 pixels around each mean, where the clamped pairs weigh most: a
    # backward that let gradient through the cap would miss the bar by 29x on d_means
    mask = np.zeros(P, bool)
    for mx, my in sp["means2d"]:
        for y in range(int(my) - 1, int(my) + 2):
            mask[y * cam.width + int(mx) - 1:y * cam.width + int(mx) + 2] = True
    rng = np.random.default_rng(9)
    d_img = rng.uniform(-1, 1, (P, 3)) * mask[:, None]
    d_alpha = rng.uniform(-1, 1, P) * mask
    g_gpu, _, _ = gpu_grads(sc, [cam], d_img, d_alpha, settings=settings)
    g_ref = oracle.render_grads(sc, cam, d_img, d_alpha=d_alpha, bg=bg)
    assert_grad_parity(g_gpu, g_ref)


def test_nd_features_forward_and_backward():
    """N-dimensional features instead of SH colour (App. C: c may be any N-vector)."""
    sc, cam = _mid_scene(n=4000, seed=41, deg=0)
    D = 8
    rng = np.random.default_rng(4)
    feats = rng.uniform(0, 1, (sc.n, D)).astype(np.float32)
    sp = oracle.project(sc, cam)
    ref = oracle.render_splats(sp, feats.astype(np.float64), cam.width, cam.height)
    d = dev_scene(sc)
    leaves = [d["means"], d["quats"], d["log_scales"], d["opacity_logits"],
              torch.as_tensor(feats, device="cuda")]
    for x in leaves:
        x.requires_grad_(True)
    imgs, alphas, _ = raster.rasterization(*leaves[:4], cameras=[cam], features=leaves[4])
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


def test_nd_features_shared_by_several_cameras():
    """Features [N, D] seen by three cameras of ragged sizes: each image against the oracle, and
    the feature gradient summed over the cameras inside the backward kernel against the sum of
    the oracle's per-camera gradients."""
    sc = synth.clustered_scene(3000, 43, sh_degree=0, log_scale_mu=-3.1)
    cams = synth.sphere_cameras(43, [(120, 90), (77, 131), (160, 64)])
    D = 5
    rng = np.random.default_rng(7)
    feats = rng.uniform(0, 1, (sc.n, D)).astype(np.float32)
    d = dev_scene(sc)
    leaves = [d["means"], d["quats"], d["log_scales"], d["opacity_logits"], torch.as_tensor(feats, device="cuda")]
    for x in leaves:
        x.requires_grad_(True)
    imgs, _, _ = raster.rasterization(*leaves[:4], cameras=cams, features=leaves[4])
    grads_in, ref_dc, ref_dm = [], 0.0, 0.0
    for cam, img in zip(cams, imgs):
        sp = oracle.project(sc, cam)
        ref = oracle.render_splats(sp, feats.astype(np.float64), cam.width, cam.height)
        assert_image_parity(img.reshape(-1, D).detach().cpu().numpy(), ref["color"], "features")
        P = cam.width * cam.height
        gimg = rng.uniform(-1, 1, (P, D)) / P
        grads_in.append(torch.as_tensor(gimg.reshape(cam.height, cam.width, D), dtype=torch.float32, device="cuda"))
        g2 = oracle.render_splats_bwd(sp, feats.astype(np.float64), cam.width, cam.height, gimg)
        ref_dc = ref_dc + g2["d_colors"]
        ref_dm = ref_dm + oracle.project_bwd(sc, cam, g2["d_means2d"], g2["d_conics"], g2["d_opacities"])["d_means"]
    g = torch.autograd.grad(list(imgs), leaves, grads_in)
    assert g[4].shape == (sc.n, D)
    assert rel_l2(g[4].cpu().numpy(), ref_dc) < 1e-3
    assert rel_l2(g[0].cpu().numpy(), ref_dm) < 1e-3


def test_absgrad_matches_oracle():
    sc, cam = _mid_scene(n=5000, seed=51, deg=0)
    settings = raster.RasterSettings(absgrad=True)
    P = cam.width * cam.height
    rng = np.random.default_rng(6)
    out, _, _ = gpu_render(sc, [cam])
    ref_f = oracle.render(sc, cam)
    d_img, _, _ = _masked_upstream(sc, (ref_f["image"].reshape(P, 3), ref_f["alpha"].reshape(P)),
                                   out["image"].cpu().numpy(), (1 - out["final_T"]).cpu().numpy(), rng, P)
    gpu_grads(sc, [cam], d_img, settings=settings)
    ag = raster.RasterizeGaussians.last_absgrad[0].cpu().numpy()
    sp = ref_f["splats"]
    g2 = oracle.render_splats_bwd(sp, ref_f["colors"], cam.width, cam.height, d_img, want_absgrad=True)
    assert rel_l2(ag, g2["absgrad"]) < 1e-3


def test_persistent_launches_render_the_same_and_reset_their_counters():
    sc = synth.clustered_scene(15000, 14, sh_degree=2, log_scale_mu=-3.3)
    cams = synth.sphere_cameras(14, [(160, 120), (96, 64), (211, 133)])
    base = gpu_render(sc, cams, settings=raster.RasterSettings(tile_schedule=True))[0]
    st = raster.RasterSettings(tile_schedule=True, persistent=True, bwd_persistent=True)
    for _ in range(2):  # a second launch must find its counters zeroed by the first
        out = gpu_render(sc, cams, settings=st)[0]
        for k in ("image", "final_T", "last_contrib"):
            np.testing.assert_array_equal(out[k].cpu().numpy(), base[k].cpu().numpy())
        T = out["ranges"].shape[0]
        assert np.all(out["tile_order"][T:].cpu().numpy() == 0)
    rng = np.random.default_rng(15)
    P = sum(c.width * c.height for c in cams)
    g = rng.normal(size=(P, 3)).astype(np.float32)
    a = gpu_grads(sc, cams, g, settings=raster.RasterSettings())[0]
    b = gpu_grads(sc, cams, g, settings=st)[0]
    for k in a:
        assert rel_l2(b[k], a[k]) <= 1e-5, k


@pytest.mark.parametrize("deg", [1, 3])
def test_fused_kernels_with_coefficients_not_16_byte_aligned(deg):
    """SH coefficients that start 4 bytes past a 16-byte boundary take the synchronous staging
    path of the fused forward and backward (the asynchronous row copies need 16-byte alignment):
    the results equal those from aligned coefficients bit for bit."""
    sc, cam = _mid_scene(n=5000, seed=60 + deg, deg=deg)
    d = dev_scene(sc)
    ca = _lib.CameraArray([cam])
    p = _lib.make_params(tile=16)
    N = sc.n
    store = torch.zeros(d["sh"].numel() + 1, device="cuda")
    sh_off = store[1:].view_as(d["sh"])
    sh_off.copy_(d["sh"])
    assert sh_off.data_ptr() % 16 == 4

    def run(sh):
        o = dict(m=torch.empty(1, N, 2, device="cuda"), dep=torch.empty(1, N, device="cuda"),
                 con=torch.empty(1, N, 3, device="cuda"), r=torch.empty(1, N, dtype=torch.int32, device="cuda"),
                 t=torch.empty(1, N, dtype=torch.int32, device="cuda"), op=torch.empty(1, N, device="cuda"),
                 col=torch.empty(1, N, 3, device="cuda"))
        _lib.gs_project_sh_eval(ca, p, d["sh_degree"], sh, d["means"], d["quats"], d["log_scales"],
                                d["opacity_logits"], o["m"], o["dep"], o["con"], o["r"], o["t"], o["op"], o["col"])
        gen = torch.Generator(device="cuda").manual_seed(3)
        rnd = lambda *shape: torch.randn(*shape, device="cuda", generator=gen)
        g = dict(dc=rnd(1, N, 3), dm2=rnd(1, N, 2), dcon=rnd(1, N, 3) * 1e-2, dop=rnd(1, N))
        b = dict(d_sh=torch.empty_like(sh), d_means=torch.empty(N, 3, device="cuda"),
                 d_quats=torch.empty(N, 4, device="cuda"), d_ls=torch.empty(N, 3, device="cuda"),
                 d_lg=torch.empty(N, device="cuda"))
        _lib.gs_sh_project_bwd(ca, p, d["sh_degree"], sh, d["means"], d["quats"], d["log_scales"],
                               d["opacity_logits"], o["r"], g["dc"], g["dm2"], g["dcon"], g["dop"], b["d_sh"],
                               b["d_means"], b["d_quats"], b["d_ls"], b["d_lg"])
        torch.cuda.synchronize()
        return {k: v.cpu().numpy() for k, v in {**o, **b}.items()}

    a, u = run(d["sh"]), run(sh_off)
    for k in a:
        np.testing.assert_array_equal(u[k], a[k], err_msg=k)


@pytest.mark.parametrize("deg,aa", [(0, False), (1, False), (2, True), (3, False), (3, True)])
def test_fused_sh_projection_backward_matches_the_two_calls(deg, aa):
    """gs_sh_project_bwd (one camera) against gs_sh_eval_bwd followed by gs_project_bwd."""
    sc, cam = _mid_scene(n=20000, seed=41 + deg, deg=deg)
    d = dev_scene(sc)
    ca = _lib.CameraArray([cam])
    p = _lib.make_params(antialiased=aa)
    N = sc.n
    sp = raster.project(ca, d["means"], d["quats"], d["log_scales"], d["opacity_logits"], p)
    gen = torch.Generator(device="cuda").manual_seed(7)
    rnd = lambda *shape: torch.randn(*shape, device="cuda", generator=gen)
    d_colors, d_m2, d_con, d_op = rnd(1, N, 3), rnd(1, N, 2), rnd(1, N, 3) * 1e-2, rnd(1, N)
    e = lambda *shape: torch.full(shape, float("nan"), device="cuda")  # every output must be written
    a = dict(d_sh=e(*d["sh"].shape), d_means=e(N, 3), d_quats=e(N, 4), d_ls=e(N, 3), d_lg=e(N))
    _lib.gs_sh_eval_bwd(ca, d["sh_degree"], d["sh"], d["means"], sp["radii"], d_colors, a["d_sh"], a["d_means"])
    _lib.gs_project_bwd(ca, d["means"], d["quats"], d["log_scales"], d["opacity_logits"], p, sp["radii"], d_m2, d_con,
                        d_op, None, a["d_means"], a["d_quats"], a["d_ls"], a["d_lg"])
    b = dict(d_sh=e(*d["sh"].shape), d_means=e(N, 3), d_quats=e(N, 4), d_ls=e(N, 3), d_lg=e(N))
    _lib.gs_sh_project_bwd(ca, p, d["sh_degree"], d["sh"], d["means"], d["quats"], d["log_scales"],
                           d["opacity_logits"], sp["radii"], d_colors, d_m2, d_con, d_op, b["d_sh"], b["d_means"],
                           b["d_quats"], b["d_ls"], b["d_lg"])
    torch.cuda.synchronize()
    vis = (sp["radii"][0] > 0).cpu().numpy()
    assert 0 < vis.sum() < N  # both visible and culled Gaussians
    for k in a:
        x, y = a[k].cpu().numpy(), b[k].cpu().numpy()
        assert np.isfinite(y).all(), k
        assert rel_l2(y, x) <= 1e-6, (k, rel_l2(y, x))
    assert (b["d_sh"].cpu().numpy()[~vis] == 0).all() and (b["d_means"].cpu().numpy()[~vis] == 0).all()
    # more than one camera is refused
    with pytest.raises(_lib.GsError):
        _lib.gs_sh_project_bwd(_lib.CameraArray([cam, cam]), p, d["sh_degree"], d["sh"], d["means"], d["quats"],
                               d["log_scales"], d["opacity_logits"], sp["radii"], d_colors, d_m2, d_con, d_op,
                               b["d_sh"], b["d_means"], b["d_quats"], b["d_ls"], b["d_lg"])


@pytest.mark.parametrize("deg,aa,ncam", [(0, False, 1), (3, False, 1), (2, True, 1), (1, False, 3), (3, True, 3)])
def test_per_gaussian_backward_stages_match_the_oracle(deg, aa, ncam):
    """The SH and projection backward as stages (App. D.3 / D.4 and the SH chain): the same
    random upstream gradients of the colours, 2D means, conics and opacities go through
    gs_sh_project_bwd (one camera, one kernel) or gs_sh_eval_bwd + gs_project_bwd (several
    cameras, the path the pipeline takes then), and through the oracle's sh_bwd + project_bwd
    per camera, summed over the cameras.  Pairs the two projections disagree on (radius
    rounding at the culling edge) get zero upstream gradients."""
    sc = synth.clustered_scene(6000, 61 + deg, sh_degree=deg, log_scale_mu=-3.0)
    cams = synth.sphere_cameras(61 + deg, [(160, 120), (97, 131), (200, 64)][:ncam])
    d = dev_scene(sc)
    ca = _lib.CameraArray(cams)
    p = _lib.make_params(antialiased=aa)
    N = sc.n
    sp = raster.project(ca, d["means"], d["quats"], d["log_scales"], d["opacity_logits"], p)
    vis_gpu = sp["radii"].cpu().numpy() > 0
    vis_ref = np.stack([oracle.project(sc, c, antialiased=aa)["radii"] > 0 for c in cams])
    both = vis_gpu & vis_ref
    assert both.sum() > 100 * ncam and (~vis_gpu).sum() > 0
    rng = np.random.default_rng(11 + deg)
    w = both.astype(np.float32)
    up = dict(d_colors=rng.normal(size=(ncam, N, 3)).astype(np.float32) * w[..., None],
              d_m2=rng.normal(size=(ncam, N, 2)).astype(np.float32) * w[..., None],
              d_con=(rng.normal(size=(ncam, N, 3)) * 1e-2).astype(np.float32) * w[..., None],
              d_op=rng.normal(size=(ncam, N)).astype(np.float32) * w)
    u = {k: torch.as_tensor(v, device="cuda") for k, v in up.items()}
    nan = lambda *shape: torch.full(shape, float("nan"), device="cuda")  # every output must be written
    out = dict(d_sh=nan(*d["sh"].shape), d_means=nan(N, 3), d_quats=nan(N, 4), d_ls=nan(N, 3), d_lg=nan(N))
    if ncam == 1:
        _lib.gs_sh_project_bwd(ca, p, d["sh_degree"], d["sh"], d["means"], d["quats"], d["log_scales"],
                               d["opacity_logits"], sp["radii"], u["d_colors"], u["d_m2"], u["d_con"], u["d_op"],
                               out["d_sh"], out["d_means"], out["d_quats"], out["d_ls"], out["d_lg"])
    else:
        _lib.gs_sh_eval_bwd(ca, d["sh_degree"], d["sh"], d["means"], sp["radii"], u["d_colors"], out["d_sh"],
                            out["d_means"])
        _lib.gs_project_bwd(ca, d["means"], d["quats"], d["log_scales"], d["opacity_logits"], p, sp["radii"],
                            u["d_m2"], u["d_con"], u["d_op"], None, out["d_means"], out["d_quats"], out["d_ls"],
                            out["d_lg"])
    torch.cuda.synchronize()
    ref = dict(d_sh=0.0, d_means=0.0, d_quats=0.0, d_ls=0.0, d_lg=0.0)
    for c, cam in enumerate(cams):
        r_sh, r_m = oracle.sh_bwd(sc, cam, up["d_colors"][c])
        g = oracle.project_bwd(sc, cam, up["d_m2"][c], up["d_con"][c], up["d_op"][c], antialiased=aa)
        ref["d_sh"] = ref["d_sh"] + r_sh
        ref["d_means"] = ref["d_means"] + r_m + g["d_means"]
        ref["d_quats"] = ref["d_quats"] + g["d_quats"]
        ref["d_ls"] = ref["d_ls"] + g["d_log_scales"]
        ref["d_lg"] = ref["d_lg"] + g["d_opacity_logits"]
    for k in out:
        x = out[k].cpu().numpy()
        assert np.isfinite(x).all(), k
        assert rel_l2(x, ref[k].reshape(x.shape)) <= 1e-3, (k, rel_l2(x, ref[k].reshape(x.shape)))
    culled = ~vis_gpu.any(0)  # zeros, not leftovers, for Gaussians every camera culls
    assert (out["d_quats"].cpu().numpy()[culled] == 0).all() and (out["d_sh"].cpu().numpy()[culled] == 0).all()


def test_depth_frames_with_colours_beside_the_sort_match_the_serial_path(monkeypatch):
    """Depth-rendering frames of 256k+ pairs evaluate SH colours and depths on a side stream
    while the sort runs (colour-only frames take the fused projection + SH kernel); the image
    must equal the single-stream path's."""
    sc = synth.clustered_scene(300_000, 17, sh_degree=3, log_scale_mu=-4.0)
    cams = synth.sphere_cameras(17, [(160, 120), (96, 128)])
    assert 2 * sc.n >= raster.SIDE_STREAM_MIN_PAIRS
    d = dev_scene(sc)
    ca = _lib.CameraArray(cams)
    run = lambda: raster.forward_pass(ca, d["means"], d["quats"], d["log_scales"], d["opacity_logits"], sh=d["sh"],
                                      sh_degree=d["sh_degree"], depth=True)["image"].cpu().numpy()
    img_a = run()
    monkeypatch.setattr(raster, "SIDE_STREAM_MIN_PAIRS", 1 << 40)
    img_b = run()
    assert img_a.shape[-1] == 4
    np.testing.assert_array_equal(img_a, img_b)


def test_bin_sort_with_unaligned_depth_and_radius_arrays():
    """Inputs that are not 16-byte aligned take the scalar path of the depth-key kernel and
    give the same lists."""
    sc, cam = _mid_scene(n=30001, seed=19)
    ref = oracle.project(sc, cam)
    m = ref["means2d"].astype(np.float32)[None]
    d = ref["depths"].astype(np.float32)[None]
    r = ref["radii"][None]
    K0, keys0, vals0, ranges0 = _gpu_bin_sort([cam], m, d, r, 16)
    ca = _lib.CameraArray([cam])
    p = _lib.make_params(tile=16)
    N = d.shape[1]
    dev = "cuda"
    mm = torch.as_tensor(m, device=dev)
    # depths and radii one element into larger buffers: 4-byte but not 16-byte aligned
    dd = torch.zeros(N + 1, device=dev)
    dd[1:] = torch.as_tensor(d[0], device=dev)
    rr = torch.zeros(N + 1, dtype=torch.int32, device=dev)
    rr[1:] = torch.as_tensor(r[0], device=dev)
    Kcap = K0 + 1024
    keys = torch.empty(Kcap, dtype=torch.int64, device=dev)
    values = torch.empty(Kcap, dtype=torch.int32, device=dev)
    ranges = torch.empty(ca.num_tiles(16), 2, dtype=torch.int32, device=dev)
    K_out = torch.zeros(1, dtype=torch.int64, device=dev)
    ws = torch.empty(_lib.gs_tile_bin_sort_workspace(ca, N, p, Kcap), dtype=torch.uint8, device=dev)
    _lib.gs_tile_bin_sort(ca, N, p, mm, dd[1:].view(1, N), rr[1:].view(1, N), Kcap, keys, values, ranges, K_out, ws)
    torch.cuda.synchronize()
    assert int(K_out.item()) == K0
    np.testing.assert_array_equal(values[:K0].cpu().numpy(), vals0)
    np.testing.assert_array_equal(keys[:K0].cpu().numpy().view(np.uint64), keys0)
    np.testing.assert_array_equal(ranges.cpu().numpy(), ranges0)

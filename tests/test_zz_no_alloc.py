"""gs_tile_bin_sort_noalloc, the entry point for callers that cannot allocate device memory
(for example a plug-in whose host application owns the device allocator, or a real-time
loop that must not stall on an allocation): it must give exactly the result of
gs_tile_bin_sort with a caller-provided workspace, call after call, since every call
reuses the same built-in scratch array.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2409_06765_gb300 import _lib, raster, synth

pytestmark = pytest.mark.gpu


def _inputs(seed, n, size):
    sc = synth.clustered_scene(n, seed, sh_degree=0, log_scale_mu=-3.2)
    cam = synth.sphere_cameras(seed, [size])[0]
    d = {k: torch.as_tensor(np.ascontiguousarray(getattr(sc, k), np.float32), device="cuda")
         for k in ("means", "quats", "log_scales", "opacity_logits")}
    ca = _lib.CameraArray([cam])
    p = _lib.make_params()
    sp = raster.project(ca, d["means"], d["quats"], d["log_scales"], d["opacity_logits"], p)
    return ca, p, sp, n


def _run(fn_noalloc, ca, p, sp, N, Kcap):
    dev = "cuda"
    keys = torch.full((Kcap,), -1, dtype=torch.int64, device=dev)
    values = torch.full((Kcap,), -1, dtype=torch.int32, device=dev)
    ranges = torch.full((ca.num_tiles(p.tile), 2), -1, dtype=torch.int32, device=dev)
    K_out = torch.zeros(1, dtype=torch.int64, device=dev)
    if fn_noalloc:
        _lib.gs_tile_bin_sort_noalloc(ca, N, p, sp["means2d"], sp["depths"], sp["radii"], Kcap, keys, values, ranges,
                                      K_out)
    else:
        ws = torch.empty(_lib.gs_tile_bin_sort_workspace(ca, N, p, Kcap), dtype=torch.uint8, device=dev)
        _lib.gs_tile_bin_sort(ca, N, p, sp["means2d"], sp["depths"], sp["radii"], Kcap, keys, values, ranges, K_out,
                              ws)
    torch.cuda.synchronize()
    K = int(K_out.item())
    return K, keys[:K].cpu().numpy(), values[:K].cpu().numpy(), ranges.cpu().numpy()


def test_noalloc_matches_workspace_version_on_consecutive_calls():
    cases = [_inputs(1, 20000, (203, 157)), _inputs(2, 12000, (160, 120))]
    for ca, p, sp, N in cases:  # two calls in a row, different sizes, same built-in scratch
        Kcap = 400_000
        K_a, keys_a, vals_a, rng_a = _run(True, ca, p, sp, N, Kcap)
        K_b, keys_b, vals_b, rng_b = _run(False, ca, p, sp, N, Kcap)
        assert 0 < K_a <= Kcap and K_a == K_b
        np.testing.assert_array_equal(keys_a, keys_b)
        np.testing.assert_array_equal(vals_a, vals_b)
        np.testing.assert_array_equal(rng_a, rng_b)
        # and the oracle's enumeration of the same splats (App. C.2), bit for bit
        cam = ca.cams[0]
        keys_r, vals_r, rng_r = oracle.bin_sort(sp["means2d"].cpu().numpy(), sp["depths"].cpu().numpy(),
                                                sp["radii"].cpu().numpy(), [cam.width], [cam.height], p.tile)
        np.testing.assert_array_equal(keys_a.view(np.uint64), keys_r)
        np.testing.assert_array_equal(vals_a, vals_r)
        np.testing.assert_array_equal(rng_a, rng_r)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    lib = _lib.load()
    ca, p, sp, N = _inputs(3, 1000, (64, 48))
    too_many = 2_000_000  # Gaussians whose per-pair scratch exceeds the built-in array
    assert _lib.gs_tile_bin_sort_workspace(ca, too_many, p, 400_000) > _lib.GS_NOALLOC_SCRATCH_BYTES
    fake = ctypes.c_void_p(256)  # never dereferenced: the size check comes first
    st = lib.gs_tile_bin_sort_noalloc(ca.ptr, 1, too_many, ctypes.byref(p), fake, fake, fake, 400_000, None, fake,
                                      fake, fake, None)
    assert st == _lib.GS_ERR_CAPACITY
    assert b"scratch" in lib.gs_last_error()

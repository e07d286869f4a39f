"""C-ABI library checks that need no GPU: it builds, loads, exports every symbol the
header declares, validates arguments on the host, and the arithmetic the kernels
rely on (exact integer support box, two-stage stable sort) matches the oracle's
definition.  No call here launches a kernel."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from paper_2409_06765_gb300 import _build, _lib, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    names = set()
    inc = os.path.join(ROOT, "include")
    for fn in os.listdir(inc):
        if fn.endswith(".h"):
            text = open(os.path.join(inc, fn)).read()
            names |= set(re.findall(r"^GS_API\s+[\w\s\*]*?\b(gs_\w+)\s*\(", text, flags=re.M))
    return names


def test_library_builds_and_exports_every_declared_symbol():
    path = _build.build()
    lib = ctypes.CDLL(path)
    declared = _declared_symbols()
    assert {"gs_project", "gs_sh_eval", "gs_tile_bin_sort", "gs_rasterize_fwd", "gs_rasterize_bwd"} <= declared
    missing = [n for n in sorted(declared) if not hasattr(lib, n)]
    assert not missing, missing
    assert set(_lib.EXPORTED) <= declared


def test_defaults_and_status_strings():
    lib = _lib.load()
    p = _lib.default_params()
    assert (p.tile, p.batch_depth, p.antialiased) == (16, 256, 0)
    assert abs(p.eps2d - 0.3) < 1e-7 and abs(p.alpha_max - 0.99) < 1e-7
    assert abs(p.alpha_min - 1 / 255) < 1e-9 and abs(p.T_min - 1e-4) < 1e-10
    assert lib.gs_status_string(_lib.GS_ERR_CAPACITY) == b"GS_ERR_CAPACITY"


def test_tile_and_pixel_counts():
    cams = _lib.CameraArray([synth.make_camera(37, 29, (0, 0, 4)), synth.make_camera(16, 16, (0, 0, 4))])
    assert _lib.gs_num_pixels(cams) == 37 * 29 + 256
    for t in (8, 16, 32):
        assert _lib.gs_num_tiles(cams, t) == cams.num_tiles(t) == (-(-37 // t)) * (-(-29 // t)) + (-(-16 // t)) ** 2
    assert cams.pixel_offsets() == [0, 37 * 29]


def test_host_validation_rejects_bad_arguments_before_any_launch():
    lib = _lib.load()
    cams = _lib.CameraArray([synth.make_camera(32, 32, (0, 0, 4))])
    p = _lib.make_params()
    null = ctypes.c_void_p(None)
    fake = ctypes.c_void_p(256)  # never dereferenced: validation fails first
    # C out of range
    assert lib.gs_project(cams.ptr, 0, 10, *[fake] * 4, ctypes.byref(p), *[fake] * 6, null) == _lib.GS_ERR_ARG
    # bad tile size
    bad = _lib.make_params(tile=12)
    assert lib.gs_project(cams.ptr, 1, 10, *[fake] * 4, ctypes.byref(bad), *[fake] * 6, null) == _lib.GS_ERR_ARG
    assert b"tile" in lib.gs_last_error()
    # NULL input
    assert lib.gs_project(cams.ptr, 1, 10, null, *[fake] * 3, ctypes.byref(p), *[fake] * 6, null) == _lib.GS_ERR_ARG
    # batch depth
    bad = _lib.make_params(batch_depth=100)
    assert lib.gs_project(cams.ptr, 1, 10, *[fake] * 4, ctypes.byref(bad), *[fake] * 6, null) == _lib.GS_ERR_ARG
    # channels
    args = [fake] * 12 + [null]  # ... blend_count, tile_order (NULL)
    assert lib.gs_rasterize_fwd(cams.ptr, 1, 10, ctypes.byref(p), 0, *args, null) == _lib.GS_ERR_ARG
    p8 = _lib.make_params(tile=8)
    assert lib.gs_rasterize_fwd(cams.ptr, 1, 10, ctypes.byref(p8), 7, *args, null) == _lib.GS_ERR_UNSUPPORTED
    # a staged batch beyond one CTA's shared memory (1024 entries of 64 channels)
    big = _lib.make_params(tile=16, batch_depth=1024, pixels_per_thread=1)
    no_count = [fake] * 11 + [null, null]  # ... blend_count and tile_order NULL
    assert lib.gs_rasterize_fwd(cams.ptr, 1, 10, ctypes.byref(big), 64, *no_count, null) == _lib.GS_ERR_UNSUPPORTED
    assert b"shared memory" in lib.gs_last_error()
    ok = _lib.make_params(tile=16, batch_depth=256, pixels_per_thread=1)
    st = lib.gs_rasterize_fwd(cams.ptr, 1, 10, ctypes.byref(ok), 64, *[null] * 12, null, null)
    assert st == _lib.GS_ERR_ARG  # past the size checks: fails on the NULL buffers instead
    # SH degree
    assert lib.gs_sh_eval(cams.ptr, 1, 10, 4, fake, fake, fake, fake, null) == _lib.GS_ERR_ARG
    # workspace too small is a capacity error
    ws = lib.gs_tile_bin_sort_workspace(cams.ptr, 1, 10, ctypes.byref(p), 1000)
    assert ws > 0
    st = lib.gs_tile_bin_sort(cams.ptr, 1, 10, ctypes.byref(p), ctypes.c_void_p(256), ctypes.c_void_p(512),
                              ctypes.c_void_p(768), 1000, null, ctypes.c_void_p(1024), ctypes.c_void_p(2048),
                              ctypes.c_void_p(4096), ctypes.c_void_p(8192), ws - 1, null)
    assert st == _lib.GS_ERR_CAPACITY
    # tile order: NULL output
    assert lib.gs_tile_order(cams.ptr, 1, ctypes.byref(p), fake, null, null) == _lib.GS_ERR_ARG
    # fused SH + projection backward: one camera only, SH degree, NULL output
    cams2 = _lib.CameraArray([synth.make_camera(32, 32, (0, 0, 4))] * 2)
    assert lib.gs_sh_project_bwd(cams2.ptr, 2, 10, ctypes.byref(p), 3, *[fake] * 15, null) == _lib.GS_ERR_ARG
    assert b"one camera" in lib.gs_last_error()
    assert lib.gs_sh_project_bwd(cams.ptr, 1, 10, ctypes.byref(p), 4, *[fake] * 15, null) == _lib.GS_ERR_ARG
    assert lib.gs_sh_project_bwd(cams.ptr, 1, 10, ctypes.byref(p), 3, *[fake] * 14, null, null) == _lib.GS_ERR_ARG
    # fused projection + SH forward: SH degree, NULL output, quats alignment
    assert lib.gs_project_sh_eval(cams.ptr, 1, 10, ctypes.byref(p), 4, *[fake] * 12, null) == _lib.GS_ERR_ARG
    assert lib.gs_project_sh_eval(cams.ptr, 1, 10, ctypes.byref(p), 3, *[fake] * 11, null, null) == _lib.GS_ERR_ARG
    odd = ctypes.c_void_p(260)
    assert lib.gs_project_sh_eval(cams.ptr, 1, 10, ctypes.byref(p), 3, fake, fake, odd, *[fake] * 9, null) == \
        _lib.GS_ERR_ARG
    assert b"16-byte" in lib.gs_last_error()


def _support_span_f32(m, r):
    """numpy replica of the kernel's exact integer box (float32 2m, ceil, floor, shifts)."""
    m2 = np.clip(np.float32(2.0) * np.asarray(m, np.float32), np.float32(-268435456.0), np.float32(268435456.0))
    a = np.ceil(m2).astype(np.int64) - 2 * r
    b = np.floor(m2).astype(np.int64) + 2 * r
    return a >> 1, (b - 1) >> 1


def test_integer_support_box_equals_the_definition():
    rng = np.random.default_rng(0)
    m = np.concatenate([
        rng.uniform(-50, 2000, 20000),
        np.arange(-40, 40) * 0.5,                                  # exact half-integers
        np.nextafter(np.arange(-40, 40) * 0.5, np.inf),            # one ulp above
        np.nextafter(np.arange(-40, 40) * 0.5, -np.inf),           # one ulp below
        np.float32(-0.5) - np.float32(2 ** -24) * np.arange(1, 5),  # just left of the image
        rng.uniform(-1e6, 1e6, 1000),
    ]).astype(np.float32)
    r = rng.integers(1, 300, m.size)
    lo, hi = _support_span_f32(m, r)
    md = m.astype(np.float64)
    ref_lo = np.ceil(md - r - 0.5).astype(np.int64)
    ref_hi = np.floor(md + r - 0.5).astype(np.int64)
    np.testing.assert_array_equal(lo, ref_lo)
    np.testing.assert_array_equal(hi, ref_hi)


def test_two_stage_stable_sort_equals_single_key_sort():
    """Sorting (camera, Gaussian) pairs by depth, emitting tiles in that order and stably
    sorting by tile gives the (tile, depth bits, index) order of the 64-bit key sort."""
    rng = np.random.default_rng(1)
    C, N, W, H, t = 2, 300, 70, 45, 16
    means2d = np.stack([rng.uniform(-5, W + 5, (C, N)), rng.uniform(-5, H + 5, (C, N))], -1).astype(np.float32)
    depths = rng.choice(rng.uniform(0.5, 3, 40), (C, N)).astype(np.float32)  # many exact ties
    radii = rng.integers(0, 12, (C, N)).astype(np.int32)
    keys, values, _ = oracle.bin_sort(means2d, depths, radii, [W, W], [H, H], t)
    tx_n = -(-W // t)
    tpc = tx_n * -(-H // t)
    flat_d = depths.reshape(-1).view(np.uint32).astype(np.int64)
    vis = radii.reshape(-1) > 0
    k1 = np.where(vis, flat_d, 0xFFFFFFFF)
    order = np.argsort(k1, kind="stable")
    em_t, em_v = [], []
    for i in order:
        c, n = divmod(int(i), N)
        r = int(radii[c, n])
        if r <= 0:
            continue
        x0, x1 = _support_span_f32(means2d[c, n, 0], r)
        y0, y1 = _support_span_f32(means2d[c, n, 1], r)
        x0, y0, x1, y1 = max(x0, 0), max(y0, 0), min(x1, W - 1), min(y1, H - 1)
        if x0 > x1 or y0 > y1:
            continue
        for ty in range(y0 // t, y1 // t + 1):
            for tx in range(x0 // t, x1 // t + 1):
                em_t.append(c * tpc + ty * tx_n + tx)
                em_v.append(int(i))
    em_t, em_v = np.array(em_t), np.array(em_v)
    o2 = np.argsort(em_t, kind="stable")
    np.testing.assert_array_equal(em_v[o2], values)
    np.testing.assert_array_equal(em_t[o2], (keys >> np.uint64(32)).astype(np.int64))


def test_more_cameras_than_the_maximum_are_rejected():
    cams = [synth.make_camera(24 + i, 20 + i, (0, 0, 4)) for i in range(_lib.GS_MAX_CAMERAS + 1)]
    with pytest.raises(ValueError, match="cameras per call"):
        _lib.CameraArray(cams)
    _lib.CameraArray(cams[:_lib.GS_MAX_CAMERAS])  # the maximum itself is accepted
    lib = _lib.load()
    arr = (_lib.GsCamera * len(cams))()
    for i, cam in enumerate(cams):
        arr[i].width, arr[i].height, arr[i].fx, arr[i].fy = cam.width, cam.height, cam.fx, cam.fy
    ptr = ctypes.cast(arr, ctypes.POINTER(_lib.GsCamera))
    p = _lib.make_params()
    fake, null = ctypes.c_void_p(256), ctypes.c_void_p(None)
    assert lib.gs_num_tiles(ptr, len(cams), 16) == -1
    assert lib.gs_tile_bin_sort_workspace(ptr, len(cams), 10, ctypes.byref(p), 100) == -1
    assert lib.gs_project(ptr, len(cams), 10, *[fake] * 4, ctypes.byref(p), *[fake] * 6, null) == _lib.GS_ERR_ARG
    assert b"GS_MAX_CAMERAS" in lib.gs_last_error()

"""ctypes binding of libgs.so (include/gs.h).

Argument marshalling only: each ``gs_*`` function here has the name of the C entry
point it calls, takes torch CUDA tensors (contiguous, of the dtype the header
states) plus host-side camera/parameter objects, passes raw device pointers and
the current CUDA stream, and raises :class:`GsError` on a non-zero status.  Every
step of the rasterizer runs in the library's kernels; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

from . import _build

GS_OK = 0
GS_ERR_ARG = -1
GS_ERR_CUDA = -2
GS_ERR_CAPACITY = -3
GS_ERR_UNSUPPORTED = -5
GS_MAX_CAMERAS = 32
GS_MAX_CHANNELS = 64
GS_MAX_INTERSECTIONS = 2**31 - 1  # (tile, Gaussian) pairs of one gs_tile_bin_sort call (int32 positions)

EXPORTED = (
    "gs_default_params", "gs_status_string", "gs_last_error", "gs_num_tiles", "gs_num_pixels", "gs_project",
    "gs_sh_eval", "gs_tile_bin_sort_workspace", "gs_tile_bin_sort", "gs_rasterize_fwd", "gs_rasterize_bwd",
    "gs_sh_eval_bwd", "gs_project_bwd", "gs_kernel_launches", "gs_tile_bin_sort_noalloc", "gs_probe_peak",
    "gs_tile_order", "gs_sh_eval_depth", "gs_sh_eval_depth_bwd", "gs_expected_depth", "gs_expected_depth_bwd",
    "gs_sh_project_bwd", "gs_project_sh_eval",
)
GS_NOALLOC_SCRATCH_BYTES = 32 * 1024 * 1024


class GsError(RuntimeError):
    def __init__(self, status: int, fn: str, detail: str):
        super().__init__(f"{fn} failed with {status} ({detail})")
        self.status = status


class GsCamera(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32), ("viewmat", ctypes.c_float * 16),
                ("fx", ctypes.c_float), ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float)]


class GsParams(ctypes.Structure):
    _fields_ = [("tile", ctypes.c_int32), ("batch_depth", ctypes.c_int32), ("antialiased", ctypes.c_int32),
                ("pixels_per_thread", ctypes.c_int32), ("eps2d", ctypes.c_float), ("near_plane", ctypes.c_float),
                ("alpha_min", ctypes.c_float), ("alpha_max", ctypes.c_float), ("T_min", ctypes.c_float),
                ("persistent", ctypes.c_int32), ("colors_shared", ctypes.c_int32)]


_lock = threading.Lock()
_lib = None

_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_CAM = ctypes.POINTER(GsCamera)
_PAR = ctypes.POINTER(GsParams)


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libgs.so (building it in-tree first when it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_missing and _build.needs_build():
            _build.build()
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"libgs.so not found at {_build.LIB}; run paper_2409_06765_gb300._build.build()")
        lib = ctypes.CDLL(_build.LIB)
        sig = {
            "gs_default_params": (None, [_PAR]),
            "gs_status_string": (ctypes.c_char_p, [_I32]),
            "gs_last_error": (ctypes.c_char_p, []),
            "gs_num_tiles": (_I64, [_CAM, _I32, _I32]),
            "gs_kernel_launches": (ctypes.c_uint64, []),
            "gs_num_pixels": (_I64, [_CAM, _I32]),
            "gs_probe_peak": (_I32, [_I32, _I32, _I32, _P, ctypes.POINTER(ctypes.c_double), _P]),
            "gs_project": (_I32, [_CAM, _I32, _I32, _P, _P, _P, _P, _PAR, _P, _P, _P, _P, _P, _P, _P]),
            "gs_sh_eval": (_I32, [_CAM, _I32, _I32, _I32, _P, _P, _P, _P, _P]),
            "gs_tile_bin_sort_workspace": (_I64, [_CAM, _I32, _I32, _PAR, _I64]),
            "gs_tile_bin_sort": (_I32, [_CAM, _I32, _I32, _PAR, _P, _P, _P, _I64, _P, _P, _P, _P, _P, ctypes.c_size_t,
                                        _P]),
            "gs_tile_bin_sort_noalloc": (_I32, [_CAM, _I32, _I32, _PAR, _P, _P, _P, _I64, _P, _P, _P, _P, _P]),
            "gs_rasterize_fwd": (_I32, [_CAM, _I32, _I32, _PAR, _I32, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P,
                                        _P, _P]),
            "gs_rasterize_bwd": (_I32, [_CAM, _I32, _I32, _PAR, _I32, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P,
                                        _P, _P, _P, _P, _P, _P, _P]),
            "gs_tile_order": (_I32, [_CAM, _I32, _PAR, _P, _P, _P]),
            "gs_sh_eval_depth": (_I32, [_CAM, _I32, _I32, _I32, _P, _P, _P, _P, _P, _P]),
            "gs_sh_eval_depth_bwd": (_I32, [_CAM, _I32, _I32, _I32, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
            "gs_expected_depth": (_I32, [_I64, _P, _I32, _I32, _P, _P, _P]),
            "gs_expected_depth_bwd": (_I32, [_I64, _P, _I32, _I32, _P, _P, _P, _P, _P]),
            "gs_sh_eval_bwd": (_I32, [_CAM, _I32, _I32, _I32, _P, _P, _P, _P, _P, _P, _P, _P]),
            "gs_project_bwd": (_I32, [_CAM, _I32, _I32, _P, _P, _P, _P, _PAR, _P, _P, _P, _P, _P, _P, _P, _P, _P,
                                      _P, _P]),
            "gs_sh_project_bwd": (_I32, [_CAM, _I32, _I32, _PAR, _I32] + [_P] * 15 + [_P]),
            "gs_project_sh_eval": (_I32, [_CAM, _I32, _I32, _PAR, _I32] + [_P] * 12 + [_P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


# --------------------------------------------------------------------------- #
# host-side objects                                                           #
# --------------------------------------------------------------------------- #

class CameraArray:
    """A host array of gs_camera built from (width, height, viewmat[4,4], fx, fy, cx, cy) tuples."""

    def __init__(self, cams):
        cams = list(cams)
        self.cams = cams  # the tuples or camera objects it was built from
        if not 1 <= len(cams) <= GS_MAX_CAMERAS:
            raise ValueError(f"1..{GS_MAX_CAMERAS} cameras per call, got {len(cams)}")
        self.arr = (GsCamera * len(cams))()
        self.sizes = []
        for i, cam in enumerate(cams):
            w, h, vm, fx, fy, cx, cy = cam.as_tuple() if hasattr(cam, "as_tuple") else cam
            vm = torch.as_tensor(vm, dtype=torch.float32).reshape(16).tolist()
            self.arr[i].width, self.arr[i].height = int(w), int(h)
            for k in range(16):
                self.arr[i].viewmat[k] = vm[k]
            self.arr[i].fx, self.arr[i].fy, self.arr[i].cx, self.arr[i].cy = float(fx), float(fy), float(cx), float(cy)
            self.sizes.append((int(w), int(h)))
        self.C = len(cams)

    @property
    def ptr(self):
        return ctypes.cast(self.arr, _CAM)

    @property
    def num_pixels(self) -> int:
        return sum(w * h for w, h in self.sizes)

    def num_tiles(self, tile: int) -> int:
        return sum(-(-w // tile) * -(-h // tile) for w, h in self.sizes)

    def pixel_offsets(self):
        out, o = [], 0
        for w, h in self.sizes:
            out.append(o)
            o += w * h
        return out


def make_params(tile=16, batch_depth=256, antialiased=False, eps2d=0.3, near_plane=0.01, alpha_min=1.0 / 255.0,
                alpha_max=0.99, T_min=1e-4, pixels_per_thread=0, persistent=False, colors_shared=False) -> GsParams:
    p = GsParams()
    p.tile, p.batch_depth, p.antialiased = int(tile), int(batch_depth), int(bool(antialiased))
    p.pixels_per_thread = int(pixels_per_thread)
    p.persistent = int(bool(persistent))
    p.colors_shared = int(bool(colors_shared))
    p.eps2d, p.near_plane, p.alpha_min, p.alpha_max, p.T_min = eps2d, near_plane, alpha_min, alpha_max, T_min
    return p


def default_params() -> GsParams:
    p = GsParams()
    load().gs_default_params(ctypes.byref(p))
    return p


# --------------------------------------------------------------------------- #
# marshalling helpers                                                         #
# --------------------------------------------------------------------------- #

_DT = {"f32": torch.float32, "i32": torch.int32, "i64": torch.int64, "u64": torch.int64, "u8": torch.uint8}


def _dev(t, kind, name, optional=False):
    if t is None:
        if optional:
            return None
        raise ValueError(f"{name} is required")
    if isinstance(t, torch.Tensor) and t.is_cuda and t.dtype is _DT[kind] and t.is_contiguous():
        return ctypes.c_void_p(t.data_ptr())
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != _DT[kind]:
        raise TypeError(f"{name} must be {_DT[kind]}, got {t.dtype}")
    raise ValueError(f"{name} must be contiguous")


_raw_stream = getattr(torch._C, "_cuda_getCurrentRawStream", None)
_cur_device = getattr(torch._C, "_cuda_getDevice", None)


def _stream(stream):
    """The cudaStream_t to launch on: the given stream, else the current stream of the current
    device (queried through torch's raw handle, which skips the Python stream object)."""
    if stream is None:
        if _raw_stream is not None and _cur_device is not None:
            return ctypes.c_void_p(_raw_stream(_cur_device()))
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _check(status: int, fn: str):
    if status != GS_OK:
        lib = load()
        raise GsError(status, fn, f"{lib.gs_status_string(status).decode()}: {lib.gs_last_error().decode()}")


def _bg(background, channels):
    if background is None:
        return None, None
    vals = [float(v) for v in background]
    if len(vals) != channels:
        raise ValueError("background must have one value per channel")
    arr = (ctypes.c_float * channels)(*vals)
    return arr, ctypes.cast(arr, ctypes.c_void_p)


# --------------------------------------------------------------------------- #
# entry points (same names as the C ABI)                                      #
# --------------------------------------------------------------------------- #

def gs_kernel_launches() -> int:
    return int(load().gs_kernel_launches())


def gs_probe_peak(kind: int, blocks: int, iters: int, sink, stream=None) -> float:
    """Launch the FFMA (kind 0) or EX2 (kind 1) throughput probe; returns the lane operations launched."""
    ops = ctypes.c_double(0.0)
    _check(load().gs_probe_peak(int(kind), int(blocks), int(iters), _dev(sink, "f32", "sink"), ctypes.byref(ops),
                                _stream(stream)), "gs_probe_peak")
    return float(ops.value)


def gs_num_tiles(cams: CameraArray, tile: int) -> int:
    return int(load().gs_num_tiles(cams.ptr, cams.C, tile))


def gs_num_pixels(cams: CameraArray) -> int:
    return int(load().gs_num_pixels(cams.ptr, cams.C))


def gs_project(cams: CameraArray, means, quats, log_scales, opacity_logits, params: GsParams, means2d, depths, conics,
               radii, tiles_touched, opacities, stream=None):
    N = means.shape[0]
    st = load().gs_project(cams.ptr, cams.C, N, _dev(means, "f32", "means"), _dev(quats, "f32", "quats"),
                           _dev(log_scales, "f32", "log_scales"), _dev(opacity_logits, "f32", "opacity_logits"),
                           ctypes.byref(params), _dev(means2d, "f32", "means2d"), _dev(depths, "f32", "depths"),
                           _dev(conics, "f32", "conics"), _dev(radii, "i32", "radii"),
                           _dev(tiles_touched, "i32", "tiles_touched"), _dev(opacities, "f32", "opacities"),
                           _stream(stream))
    _check(st, "gs_project")


def gs_project_sh_eval(cams: CameraArray, params: GsParams, sh_degree: int, sh, means, quats, log_scales,
                       opacity_logits, means2d, depths, conics, radii, tiles_touched, opacities, colors, stream=None):
    N = means.shape[0]
    st = load().gs_project_sh_eval(cams.ptr, cams.C, N, ctypes.byref(params), sh_degree, _dev(sh, "f32", "sh"),
                                   _dev(means, "f32", "means"), _dev(quats, "f32", "quats"),
                                   _dev(log_scales, "f32", "log_scales"),
                                   _dev(opacity_logits, "f32", "opacity_logits"), _dev(means2d, "f32", "means2d"),
                                   _dev(depths, "f32", "depths"), _dev(conics, "f32", "conics"),
                                   _dev(radii, "i32", "radii"), _dev(tiles_touched, "i32", "tiles_touched"),
                                   _dev(opacities, "f32", "opacities"), _dev(colors, "f32", "colors"),
                                   _stream(stream))
    _check(st, "gs_project_sh_eval")


def gs_sh_eval(cams: CameraArray, sh_degree: int, sh, means, radii, colors, stream=None):
    N = means.shape[0]
    st = load().gs_sh_eval(cams.ptr, cams.C, N, sh_degree, _dev(sh, "f32", "sh"), _dev(means, "f32", "means"),
                           _dev(radii, "i32", "radii"), _dev(colors, "f32", "colors"), _stream(stream))
    _check(st, "gs_sh_eval")


def gs_tile_bin_sort_workspace(cams: CameraArray, N: int, params: GsParams, K_capacity: int) -> int:
    if int(K_capacity) > GS_MAX_INTERSECTIONS:
        raise GsError(GS_ERR_CAPACITY, "gs_tile_bin_sort_workspace",
                      f"{int(K_capacity)} intersections exceed GS_MAX_INTERSECTIONS (int32 list positions)")
    n = int(load().gs_tile_bin_sort_workspace(cams.ptr, cams.C, N, ctypes.byref(params), int(K_capacity)))
    if n < 0:
        raise GsError(GS_ERR_ARG, "gs_tile_bin_sort_workspace", "invalid sizes")
    return n


def gs_tile_bin_sort(cams: CameraArray, N: int, params: GsParams, means2d, depths, radii, K_capacity: int, keys,
                     values, tile_ranges, K_out, workspace, stream=None):
    st = load().gs_tile_bin_sort(cams.ptr, cams.C, N, ctypes.byref(params), _dev(means2d, "f32", "means2d"),
                                 _dev(depths, "f32", "depths"), _dev(radii, "i32", "radii"), int(K_capacity),
                                 _dev(keys, "u64", "keys", optional=True), _dev(values, "i32", "values"),
                                 _dev(tile_ranges, "i32", "tile_ranges"), _dev(K_out, "i64", "K_out"),
                                 _dev(workspace, "u8", "workspace"), workspace.numel(), _stream(stream))
    _check(st, "gs_tile_bin_sort")


def gs_tile_bin_sort_noalloc(cams: CameraArray, N: int, params: GsParams, means2d, depths, radii, K_capacity: int,
                             keys, values, tile_ranges, K_out, stream=None):
    """gs_tile_bin_sort without a workspace argument: for callers that cannot allocate device
    memory, the scratch is the library's built-in array (GS_NOALLOC_SCRATCH_BYTES)."""
    st = load().gs_tile_bin_sort_noalloc(cams.ptr, cams.C, N, ctypes.byref(params), _dev(means2d, "f32", "means2d"),
                                         _dev(depths, "f32", "depths"), _dev(radii, "i32", "radii"),
                                         int(K_capacity), _dev(keys, "u64", "keys", optional=True),
                                         _dev(values, "i32", "values"), _dev(tile_ranges, "i32", "tile_ranges"),
                                         _dev(K_out, "i64", "K_out"), _stream(stream))
    _check(st, "gs_tile_bin_sort_noalloc")


def gs_rasterize_fwd(cams: CameraArray, N: int, params: GsParams, channels: int, tile_ranges, values, radii, means2d,
                     conics, opacities, colors, background, image, final_T, last_contrib, blend_count=None,
                     stream=None, tile_order=None):
    keep, bgp = _bg(background, channels)
    st = load().gs_rasterize_fwd(cams.ptr, cams.C, N, ctypes.byref(params), channels,
                                 _dev(tile_ranges, "i32", "tile_ranges"), _dev(values, "i32", "values"),
                                 _dev(radii, "i32", "radii"), _dev(means2d, "f32", "means2d"),
                                 _dev(conics, "f32", "conics"), _dev(opacities, "f32", "opacities"),
                                 _dev(colors, "f32", "colors"), bgp, _dev(image, "f32", "image"),
                                 _dev(final_T, "f32", "final_T"), _dev(last_contrib, "i32", "last_contrib"),
                                 _dev(blend_count, "i64", "blend_count", optional=True),
                                 _dev(tile_order, "i32", "tile_order", optional=True), _stream(stream))
    del keep
    _check(st, "gs_rasterize_fwd")


def gs_rasterize_bwd(cams: CameraArray, N: int, params: GsParams, channels: int, tile_ranges, values, radii, means2d,
                     conics, opacities, colors, background, final_T, last_contrib, d_image, d_alpha, d_means2d,
                     d_conics, d_opacities, d_colors, absgrad=None, stream=None, tile_order=None):
    keep, bgp = _bg(background, channels)
    st = load().gs_rasterize_bwd(cams.ptr, cams.C, N, ctypes.byref(params), channels,
                                 _dev(tile_ranges, "i32", "tile_ranges"), _dev(values, "i32", "values"),
                                 _dev(radii, "i32", "radii"), _dev(means2d, "f32", "means2d"),
                                 _dev(conics, "f32", "conics"), _dev(opacities, "f32", "opacities"),
                                 _dev(colors, "f32", "colors"), bgp, _dev(final_T, "f32", "final_T"),
                                 _dev(last_contrib, "i32", "last_contrib"), _dev(d_image, "f32", "d_image"),
                                 _dev(d_alpha, "f32", "d_alpha", optional=True), _dev(d_means2d, "f32", "d_means2d"),
                                 _dev(d_conics, "f32", "d_conics"), _dev(d_opacities, "f32", "d_opacities"),
                                 _dev(d_colors, "f32", "d_colors"), _dev(absgrad, "f32", "absgrad", optional=True),
                                 _dev(tile_order, "i32", "tile_order", optional=True), _stream(stream))
    del keep
    _check(st, "gs_rasterize_bwd")


def gs_sh_eval_depth(cams: CameraArray, sh_degree: int, sh, means, radii, depths, colors_rgbd, stream=None):
    N = means.shape[0]
    _check(load().gs_sh_eval_depth(cams.ptr, cams.C, N, sh_degree, _dev(sh, "f32", "sh"), _dev(means, "f32", "means"),
                                   _dev(radii, "i32", "radii"), _dev(depths, "f32", "depths"),
                                   _dev(colors_rgbd, "f32", "colors_rgbd"), _stream(stream)), "gs_sh_eval_depth")


def gs_sh_eval_depth_bwd(cams: CameraArray, sh_degree: int, sh, means, radii, d_colors_rgbd, d_sh, d_means, d_depths,
                         stream=None, d_viewmats=None):
    N = means.shape[0]
    _check(load().gs_sh_eval_depth_bwd(cams.ptr, cams.C, N, sh_degree, _dev(sh, "f32", "sh"),
                                       _dev(means, "f32", "means"), _dev(radii, "i32", "radii"),
                                       _dev(d_colors_rgbd, "f32", "d_colors_rgbd"), _dev(d_sh, "f32", "d_sh"),
                                       _dev(d_means, "f32", "d_means"), _dev(d_depths, "f32", "d_depths"),
                                       _dev(d_viewmats, "f32", "d_viewmats", optional=True), _stream(stream)),
           "gs_sh_eval_depth_bwd")


def gs_expected_depth(image, depth_channel: int, final_T, expected, stream=None):
    P, ch = image.shape
    _check(load().gs_expected_depth(P, _dev(image, "f32", "image"), ch, depth_channel, _dev(final_T, "f32", "final_T"),
                                    _dev(expected, "f32", "expected_depth"), _stream(stream)), "gs_expected_depth")


def gs_expected_depth_bwd(image, depth_channel: int, final_T, d_expected, d_image, d_alpha, stream=None):
    P, ch = image.shape
    _check(load().gs_expected_depth_bwd(P, _dev(image, "f32", "image"), ch, depth_channel,
                                        _dev(final_T, "f32", "final_T"), _dev(d_expected, "f32", "d_expected"),
                                        _dev(d_image, "f32", "d_image"), _dev(d_alpha, "f32", "d_alpha"),
                                        _stream(stream)), "gs_expected_depth_bwd")


def gs_tile_order(cams: CameraArray, params: GsParams, tile_ranges, tile_order, stream=None):
    """Tiles ordered longest list first (a launch order for the compositing kernels)."""
    st = load().gs_tile_order(cams.ptr, cams.C, ctypes.byref(params), _dev(tile_ranges, "i32", "tile_ranges"),
                              _dev(tile_order, "i32", "tile_order"), _stream(stream))
    _check(st, "gs_tile_order")


def gs_sh_eval_bwd(cams: CameraArray, sh_degree: int, sh, means, radii, d_colors, d_sh, d_means, stream=None,
                   d_viewmats=None):
    N = means.shape[0]
    st = load().gs_sh_eval_bwd(cams.ptr, cams.C, N, sh_degree, _dev(sh, "f32", "sh"), _dev(means, "f32", "means"),
                               _dev(radii, "i32", "radii"), _dev(d_colors, "f32", "d_colors"),
                               _dev(d_sh, "f32", "d_sh"), _dev(d_means, "f32", "d_means"),
                               _dev(d_viewmats, "f32", "d_viewmats", optional=True), _stream(stream))
    _check(st, "gs_sh_eval_bwd")


def gs_sh_project_bwd(cams: CameraArray, params: GsParams, sh_degree: int, sh, means, quats, log_scales,
                      opacity_logits, radii, d_colors, d_means2d, d_conics, d_opacities, d_sh, d_means, d_quats,
                      d_log_scales, d_opacity_logits, stream=None):
    N = means.shape[0]
    st = load().gs_sh_project_bwd(cams.ptr, cams.C, N, ctypes.byref(params), sh_degree, _dev(sh, "f32", "sh"),
                                  _dev(means, "f32", "means"), _dev(quats, "f32", "quats"),
                                  _dev(log_scales, "f32", "log_scales"),
                                  _dev(opacity_logits, "f32", "opacity_logits"), _dev(radii, "i32", "radii"),
                                  _dev(d_colors, "f32", "d_colors"), _dev(d_means2d, "f32", "d_means2d"),
                                  _dev(d_conics, "f32", "d_conics"), _dev(d_opacities, "f32", "d_opacities"),
                                  _dev(d_sh, "f32", "d_sh"), _dev(d_means, "f32", "d_means"),
                                  _dev(d_quats, "f32", "d_quats"), _dev(d_log_scales, "f32", "d_log_scales"),
                                  _dev(d_opacity_logits, "f32", "d_opacity_logits"), _stream(stream))
    _check(st, "gs_sh_project_bwd")


def gs_project_bwd(cams: CameraArray, means, quats, log_scales, opacity_logits, params: GsParams, radii, d_means2d,
                   d_conics, d_opacities, d_depths, d_means, d_quats, d_log_scales, d_opacity_logits, stream=None,
                   d_viewmats=None):
    N = means.shape[0]
    st = load().gs_project_bwd(cams.ptr, cams.C, N, _dev(means, "f32", "means"), _dev(quats, "f32", "quats"),
                               _dev(log_scales, "f32", "log_scales"), _dev(opacity_logits, "f32", "opacity_logits"),
                               ctypes.byref(params), _dev(radii, "i32", "radii"),
                               _dev(d_means2d, "f32", "d_means2d"), _dev(d_conics, "f32", "d_conics"),
                               _dev(d_opacities, "f32", "d_opacities"),
                               _dev(d_depths, "f32", "d_depths", optional=True), _dev(d_means, "f32", "d_means"),
                               _dev(d_quats, "f32", "d_quats"), _dev(d_log_scales, "f32", "d_log_scales"),
                               _dev(d_opacity_logits, "f32", "d_opacity_logits"),
                               _dev(d_viewmats, "f32", "d_viewmats", optional=True), _stream(stream))
    _check(st, "gs_project_bwd")

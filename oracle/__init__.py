"""FP64 CPU oracle of the differentiable tile-based Gaussian rasterizer.

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may use it; the product package never imports
it.  The arithmetic lives in ``gs_oracle.c`` (plain C, FP64, OpenMP over
Gaussians / pixels); this module compiles it with gcc and marshals numpy arrays.
Inputs come in as float32 from ``paper_2409_06765_gb300.synth`` and are promoted
to float64 unchanged.

Every function cites the part of the paper (arXiv 2409.06765) it follows:
App. C (forward: projection, tiles, compositing), App. D (backward),
App. E (quaternion and pixel conventions), App. A (anti-aliasing, depth).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gs_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

# Render parameters.  The paper states none of their values (they follow Kerbl et al.: the
# alpha cap and skip, the transmittance floor, the near plane; App. A gives the 0.3 low-pass).
# They are inputs of the rasterizer like the Gaussians and cameras, and like those the oracle
# takes them as the float32 values a caller passes (promoted to float64 unchanged).  The
# decisions they enter -- culling at the near plane, skipping, clamping, stopping -- then
# compare against the same thresholds as any float32 implementation: Fig. 1's Gaussian at
# z = 0.01 renders, and two capped alphas stacked, (1 - alpha_max)^2 < T_min, stop the pixel.
_f32 = lambda v: float(np.float32(v))
ALPHA_MIN = _f32(1.0 / 255.0)
ALPHA_MAX = _f32(0.99)
T_MIN = _f32(1.0e-4)
EPS2D = _f32(0.3)
NEAR = _f32(0.01)


def build(force: bool = False) -> str:
    """Compile gs_oracle.c into oracle/_build/liboracle.so (gcc, FP64, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
               _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)
_F = ctypes.POINTER(ctypes.c_float)
_U64 = ctypes.POINTER(ctypes.c_uint64)
_i = ctypes.c_int
_d = ctypes.c_double
_ll = ctypes.c_longlong


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        lib.orc_project.argtypes = [_i, _D, _D, _D, _D, _D, _D, _i, _i, _d, _d, _i, _D, _D, _D, _D, _I, _D, _I]
        lib.orc_sh_basis.argtypes = [_i, _i, _D, _D]
        lib.orc_sh_basis_grad.argtypes = [_i, _i, _D, _D]
        lib.orc_sh_colors.argtypes = [_i, _i, _D, _D, _D, _D, _D]
        lib.orc_sh_bwd.argtypes = [_i, _i, _D, _D, _D, _D, _D, _D, _D]
        lib.orc_render.argtypes = [_i, _D, _D, _D, _D, _i, _D, _I, _I, _i, _i, _D, _d, _d, _d, _i, _I,
                                   _D, _D, _I, ctypes.POINTER(ctypes.c_longlong)]
        lib.orc_render_trace.argtypes = [_i, _D, _D, _D, _D, _i, _D, _I, _I, _i, _i, _D, _d, _d, _d, _i,
                                         _I, _D, _D]
        lib.orc_render_trace.restype = _i
        lib.orc_render_bwd.argtypes = [_i, _D, _D, _D, _D, _i, _D, _I, _I, _i, _i, _D, _d, _d, _d, _i, _I,
                                       _D, _D, _D, _D, _D, _D, _D]
        lib.orc_project_bwd.argtypes = [_i, _D, _D, _D, _D, _D, _D, _i, _i, _d, _d, _i, _D, _D, _D, _D,
                                        _D, _D, _D, _D, _D]
        lib.orc_bin_sort.argtypes = [_i, _i, _F, _F, _I, _I, _I, _i, _ll, _U64, _I, _I]
        lib.orc_bin_sort.restype = _ll
        lib.orc_num_threads.restype = _i
        lib.orc_rotation.argtypes = [_D, _D]
        lib.orc_drot.argtypes = [_D, _D]
        lib.orc_cov3d.argtypes = [_D, _D, _D]
        _lib = lib
        return lib


def _d64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _p(a):
    if a is None:
        return None
    if a.dtype == np.float64:
        return a.ctypes.data_as(_D)
    if a.dtype == np.float32:
        return a.ctypes.data_as(_F)
    if a.dtype == np.int32:
        return a.ctypes.data_as(_I)
    if a.dtype == np.uint64:
        return a.ctypes.data_as(_U64)
    if a.dtype == np.int64:
        return a.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong))
    raise TypeError(a.dtype)


def rotation(q) -> np.ndarray:
    """R(q/|q|), App. E."""
    q = _d64(q)
    R = np.zeros(9)
    _load().orc_rotation(_p(q), _p(R))
    return R.reshape(3, 3)


def drot_dquat(q) -> np.ndarray:
    """[dR/dw, dR/dx, dR/dy, dR/dz] at a unit quaternion, App. D.4."""
    q = _d64(q)
    D = np.zeros(36)
    _load().orc_drot(_p(q), _p(D))
    return D.reshape(4, 3, 3)


def cov3d(quat, log_scale) -> np.ndarray:
    """Sigma = R S S^T R^T (gradient-flow figure)."""
    S = np.zeros(9)
    _load().orc_cov3d(_p(_d64(quat)), _p(_d64(log_scale)), _p(S))
    return S.reshape(3, 3)


def num_threads() -> int:
    """OpenMP threads the oracle's loops use (reported beside its timings)."""
    return int(_load().orc_num_threads())


@dataclass
class CameraF64:
    width: int
    height: int
    viewmat: np.ndarray  # float64 [16]
    intr: np.ndarray     # float64 [fx, fy, cx, cy]


def camera(cam) -> CameraF64:
    """Promote a synth.Camera (float32 values) to float64 without changing its values."""
    return CameraF64(int(cam.width), int(cam.height), _d64(np.asarray(cam.viewmat).reshape(16)),
                     _d64([cam.fx, cam.fy, cam.cx, cam.cy]))


# --------------------------------------------------------------------------- #
# App. C.1 / App. E / App. A: projection                                       #
# --------------------------------------------------------------------------- #

def project(scene, cam, eps2d=EPS2D, near=NEAR, antialiased=False):
    """Per Gaussian: pixel mean, depth, conic, (Sigma'+sI), radius, opacity, pixel box."""
    lib = _load()
    c = camera(cam)
    N = scene.n
    means, quats = _d64(scene.means), _d64(scene.quats)
    ls, lg = _d64(scene.log_scales), _d64(scene.opacity_logits)
    out = dict(means2d=np.zeros((N, 2)), depths=np.zeros(N), conics=np.zeros((N, 3)),
               cov2d=np.zeros((N, 3)), radii=np.zeros(N, np.int32), opacities=np.zeros(N),
               boxes=np.zeros((N, 4), np.int32))
    lib.orc_project(N, _p(means), _p(quats), _p(ls), _p(lg), _p(c.viewmat), _p(c.intr), c.width, c.height,
                    float(eps2d), float(near), int(bool(antialiased)), _p(out["means2d"]), _p(out["depths"]),
                    _p(out["conics"]), _p(out["cov2d"]), _p(out["radii"]), _p(out["opacities"]),
                    _p(out["boxes"]))
    return out


# --------------------------------------------------------------------------- #
# App. C.1: spherical-harmonics colour                                         #
# --------------------------------------------------------------------------- #

def sh_basis(degree: int, dirs) -> np.ndarray:
    """Real orthonormal SH basis Y_k(dir), k < (degree+1)^2, at unit directions [P, 3] (App. C.1,
    which names SH but not the basis: the real harmonics with the Condon-Shortley phase)."""
    dirs = _d64(dirs).reshape(-1, 3)
    K = (degree + 1) ** 2
    Y = np.zeros((dirs.shape[0], K))
    _load().orc_sh_basis(degree, dirs.shape[0], _p(dirs), _p(Y))
    return Y


def sh_basis_grad(degree: int, dirs) -> np.ndarray:
    """dY_k/d(x, y, z) of the basis polynomials at unit directions [P, 3] (App. C.1 differentiated)."""
    dirs = _d64(dirs).reshape(-1, 3)
    K = (degree + 1) ** 2
    dY = np.zeros((dirs.shape[0], K, 3))
    _load().orc_sh_basis_grad(degree, dirs.shape[0], _p(dirs), _p(dY))
    return dY


def sh_colors(scene, cam, means=None, sh=None):
    """colour = max(0, sum_k Y_k(dir) c_k + 0.5) along dir = normalize(mu - camera centre)."""
    c = camera(cam)
    N = scene.n
    means = _d64(scene.means if means is None else means)
    sh = _d64(scene.sh if sh is None else sh)
    colors, raw = np.zeros((N, 3)), np.zeros((N, 3))
    _load().orc_sh_colors(N, scene.sh_degree, _p(sh), _p(means), _p(c.viewmat), _p(colors), _p(raw))
    return colors, raw


def sh_bwd(scene, cam, d_colors, d_viewmat=None):
    """SH backward; with ``d_viewmat`` (float64 [16]) also accumulates the pose gradient of the
    view direction into it."""
    c = camera(cam)
    N = scene.n
    K = (scene.sh_degree + 1) ** 2
    d_sh, d_means = np.zeros((N, K, 3)), np.zeros((N, 3))
    _load().orc_sh_bwd(N, scene.sh_degree, _p(_d64(scene.sh)), _p(_d64(scene.means)), _p(c.viewmat),
                       _p(_d64(d_colors)), _p(d_sh), _p(d_means), _p(d_viewmat))
    return d_sh, d_means


# --------------------------------------------------------------------------- #
# App. C.2: compositing, brute force per pixel over all depth-sorted Gaussians  #
# --------------------------------------------------------------------------- #

def render_splats(splats, colors, width, height, pixels=None, bg=None, alpha_min=ALPHA_MIN,
                  alpha_max=ALPHA_MAX, T_min=T_MIN):
    """Composite the given 2D splats at ``pixels`` (linear y*W+x) or the whole image."""
    colors = _d64(colors)
    ch = colors.shape[1]
    N = colors.shape[0]
    pix = None if pixels is None else np.ascontiguousarray(pixels, dtype=np.int32)
    P = width * height if pix is None else pix.shape[0]
    bgv = _d64(np.zeros(ch) if bg is None else bg)
    out_col, out_T = np.zeros((P, ch)), np.zeros(P)
    out_nc, out_bl = np.zeros(P, np.int32), np.zeros(P, np.int64)
    _load().orc_render(N, _p(_d64(splats["means2d"])), _p(_d64(splats["conics"])),
                       _p(_d64(splats["opacities"])), _p(colors), ch, _p(_d64(splats["depths"])),
                       _p(np.ascontiguousarray(splats["radii"], np.int32)),
                       _p(np.ascontiguousarray(splats["boxes"], np.int32)), width, height, _p(bgv),
                       alpha_min, alpha_max, T_min, P, _p(pix), _p(out_col), _p(out_T), _p(out_nc),
                       _p(out_bl))
    return dict(color=out_col, T=out_T, ncontrib=out_nc, blends=out_bl)


def render_trace(splats, colors, px, py, bg=None, alpha_min=ALPHA_MIN, alpha_max=ALPHA_MAX, T_min=T_MIN):
    colors = _d64(colors)
    ch = colors.shape[1]
    N = colors.shape[0]
    cap = N + 1
    ids, alphas, Ts = np.zeros(cap, np.int32), np.zeros(cap), np.zeros(cap)
    bgv = _d64(np.zeros(ch) if bg is None else bg)
    nc = _load().orc_render_trace(N, _p(_d64(splats["means2d"])), _p(_d64(splats["conics"])),
                                  _p(_d64(splats["opacities"])), _p(colors), ch, _p(_d64(splats["depths"])),
                                  _p(np.ascontiguousarray(splats["radii"], np.int32)),
                                  _p(np.ascontiguousarray(splats["boxes"], np.int32)), int(px), int(py),
                                  _p(bgv), alpha_min, alpha_max, T_min, cap, _p(ids), _p(alphas), _p(Ts))
    return ids[:nc], alphas[:nc], Ts[:nc]


def render_splats_bwd(splats, colors, width, height, d_color, d_alpha=None, pixels=None, bg=None,
                      alpha_min=ALPHA_MIN, alpha_max=ALPHA_MAX, T_min=T_MIN, want_absgrad=False):
    """App. D.2: gradients of sum_p <d_color[p], C_p> + d_alpha[p] (1 - T_p) w.r.t. 2D splat data."""
    colors = _d64(colors)
    ch = colors.shape[1]
    N = colors.shape[0]
    pix = None if pixels is None else np.ascontiguousarray(pixels, dtype=np.int32)
    P = width * height if pix is None else pix.shape[0]
    bgv = _d64(np.zeros(ch) if bg is None else bg)
    g = _d64(d_color).reshape(P, ch)
    gA = None if d_alpha is None else _d64(d_alpha).reshape(P)
    out = dict(d_means2d=np.zeros((N, 2)), d_conics=np.zeros((N, 3)), d_opacities=np.zeros(N),
               d_colors=np.zeros((N, ch)))
    absg = np.zeros((N, 2)) if want_absgrad else None
    _load().orc_render_bwd(N, _p(_d64(splats["means2d"])), _p(_d64(splats["conics"])),
                           _p(_d64(splats["opacities"])), _p(colors), ch, _p(_d64(splats["depths"])),
                           _p(np.ascontiguousarray(splats["radii"], np.int32)),
                           _p(np.ascontiguousarray(splats["boxes"], np.int32)), width, height, _p(bgv),
                           alpha_min, alpha_max, T_min, P, _p(pix), _p(g), _p(gA), _p(out["d_means2d"]),
                           _p(out["d_conics"]), _p(out["d_opacities"]), _p(out["d_colors"]), _p(absg))
    if want_absgrad:
        out["absgrad"] = absg
    return out


# --------------------------------------------------------------------------- #
# App. D.3 / D.4: projection backward                                          #
# --------------------------------------------------------------------------- #

def project_bwd(scene, cam, d_means2d, d_conics, d_opacities, d_depths=None, eps2d=EPS2D, near=NEAR,
                antialiased=False, d_viewmat=None):
    """Projection backward; with ``d_viewmat`` (float64 [16]) also accumulates the pose gradient."""
    lib = _load()
    c = camera(cam)
    N = scene.n
    out = dict(d_means=np.zeros((N, 3)), d_quats=np.zeros((N, 4)), d_log_scales=np.zeros((N, 3)),
               d_opacity_logits=np.zeros(N))
    dd = None if d_depths is None else _d64(d_depths)
    lib.orc_project_bwd(N, _p(_d64(scene.means)), _p(_d64(scene.quats)), _p(_d64(scene.log_scales)),
                        _p(_d64(scene.opacity_logits)), _p(c.viewmat), _p(c.intr), c.width, c.height,
                        float(eps2d), float(near), int(bool(antialiased)), _p(_d64(d_means2d)),
                        _p(_d64(d_conics)), _p(_d64(d_opacities)), _p(dd), _p(out["d_means"]),
                        _p(out["d_quats"]), _p(out["d_log_scales"]), _p(out["d_opacity_logits"]), _p(d_viewmat))
    return out


# --------------------------------------------------------------------------- #
# App. C.2: tile binning + depth sort, by enumeration                          #
# --------------------------------------------------------------------------- #

def bin_sort(means2d, depths, radii, widths, heights, tile):
    """Canonical intersection list from float32 means2d [C,N,2], depths [C,N], int radii [C,N]."""
    means2d = np.ascontiguousarray(means2d, np.float32)
    depths = np.ascontiguousarray(depths, np.float32)
    radii = np.ascontiguousarray(radii, np.int32)
    C, N = depths.shape
    widths = np.ascontiguousarray(widths, np.int32)
    heights = np.ascontiguousarray(heights, np.int32)
    tiles = int(sum(((w + tile - 1) // tile) * ((h + tile - 1) // tile) for w, h in zip(widths, heights)))
    lib = _load()
    K = lib.orc_bin_sort(C, N, _p(means2d), _p(depths), _p(radii), _p(widths), _p(heights), tile, 0,
                         None, None, _p(np.zeros(2 * tiles, np.int32)))
    keys = np.zeros(max(K, 1), np.uint64)
    values = np.zeros(max(K, 1), np.int32)
    ranges = np.zeros((tiles, 2), np.int32)
    K2 = lib.orc_bin_sort(C, N, _p(means2d), _p(depths), _p(radii), _p(widths), _p(heights), tile, K,
                          _p(keys), _p(values), _p(ranges))
    assert K2 == K
    return keys[:K], values[:K], ranges


# --------------------------------------------------------------------------- #
# whole pipeline (forward and backward) for one camera                         #
# --------------------------------------------------------------------------- #

def render(scene, cam, pixels=None, bg=None, antialiased=False, eps2d=EPS2D, near=NEAR,
           alpha_min=ALPHA_MIN, alpha_max=ALPHA_MAX, T_min=T_MIN, extra_channels=None):
    """Project, colour and composite; returns image [H,W,ch] (or [P,ch]), alpha, T, counts."""
    sp = project(scene, cam, eps2d=eps2d, near=near, antialiased=antialiased)
    colors, _ = sh_colors(scene, cam)
    if extra_channels is not None:
        colors = np.concatenate([colors, _d64(extra_channels)], axis=1)
    r = render_splats(sp, colors, cam.width, cam.height, pixels=pixels, bg=bg, alpha_min=alpha_min,
                      alpha_max=alpha_max, T_min=T_min)
    ch = colors.shape[1]
    img = r["color"] if pixels is not None else r["color"].reshape(cam.height, cam.width, ch)
    T = r["T"] if pixels is not None else r["T"].reshape(cam.height, cam.width)
    return dict(image=img, T=T, alpha=1.0 - T, ncontrib=r["ncontrib"], blends=r["blends"], splats=sp,
                colors=colors)


def render_grads(scene, cam, d_image, d_alpha=None, pixels=None, bg=None, antialiased=False, eps2d=EPS2D,
                 near=NEAR, alpha_min=ALPHA_MIN, alpha_max=ALPHA_MAX, T_min=T_MIN):
    """Gradients of sum <d_image, image> + <d_alpha, alpha> w.r.t. every Gaussian leaf (FP64)."""
    sp = project(scene, cam, eps2d=eps2d, near=near, antialiased=antialiased)
    colors, _ = sh_colors(scene, cam)
    g2 = render_splats_bwd(sp, colors, cam.width, cam.height, d_image, d_alpha=d_alpha, pixels=pixels, bg=bg,
                           alpha_min=alpha_min, alpha_max=alpha_max, T_min=T_min, want_absgrad=True)
    d_view = np.zeros(16)
    d_sh, d_means_sh = sh_bwd(scene, cam, g2["d_colors"], d_viewmat=d_view)
    g3 = project_bwd(scene, cam, g2["d_means2d"], g2["d_conics"], g2["d_opacities"], eps2d=eps2d, near=near,
                     antialiased=antialiased, d_viewmat=d_view)
    return dict(d_means=g3["d_means"] + d_means_sh, d_quats=g3["d_quats"], d_log_scales=g3["d_log_scales"],
                d_opacity_logits=g3["d_opacity_logits"], d_sh=d_sh, d_viewmat=d_view.reshape(4, 4),
                splat_grads=g2, splats=sp, colors=colors)


# --------------------------------------------------------------------------- #
# App. A: depth rendering                                                      #
#   accumulated depth  A = sum_n z_n alpha_n T_n   (z_n = camera-space depth)  #
#   expected depth     E = A / sum_n alpha_n T_n = A / (1 - T_final), 0 if 0   #
# --------------------------------------------------------------------------- #

def render_depth(scene, cam, pixels=None, bg=None, antialiased=False, eps2d=EPS2D, near=NEAR,
                 alpha_min=ALPHA_MIN, alpha_max=ALPHA_MAX, T_min=T_MIN):
    """Colour, accumulated depth and expected depth: the depth is a fourth feature channel
    composited with the same weights alpha_n T_n as the colour (background 0 for it)."""
    sp = project(scene, cam, eps2d=eps2d, near=near, antialiased=antialiased)
    colors, _ = sh_colors(scene, cam)
    rgbd = np.concatenate([colors, sp["depths"][:, None]], axis=1)
    bg4 = None if bg is None else np.concatenate([_d64(bg), [0.0]])
    r = render_splats(sp, rgbd, cam.width, cam.height, pixels=pixels, bg=bg4, alpha_min=alpha_min,
                      alpha_max=alpha_max, T_min=T_min)
    acc = r["color"][:, 3]
    a = 1.0 - r["T"]
    expected = np.where(a > 0.0, acc / np.where(a > 0.0, a, 1.0), 0.0)
    return dict(color=r["color"][:, :3], acc_depth=acc, expected_depth=expected, alpha=a, T=r["T"],
                ncontrib=r["ncontrib"], blends=r["blends"], splats=sp, colors=rgbd)


def render_depth_grads(scene, cam, d_color, d_acc_depth=None, d_expected_depth=None, d_alpha=None, pixels=None,
                       bg=None, antialiased=False, eps2d=EPS2D, near=NEAR, alpha_min=ALPHA_MIN,
                       alpha_max=ALPHA_MAX, T_min=T_MIN):
    """Gradients of <d_color, C> + <d_acc, A> + <d_exp, E> + <d_alpha, alpha> w.r.t. the leaves.

    E = A / a with a = 1 - T_final: dE/dA = 1/a and dE/da = -E/a, so the expected-depth term
    becomes an accumulated-depth term and an alpha term; the depth channel's per-Gaussian
    gradient is the gradient w.r.t. z_n = t_z, passed to the projection backward."""
    f = render_depth(scene, cam, pixels=pixels, bg=bg, antialiased=antialiased, eps2d=eps2d, near=near,
                     alpha_min=alpha_min, alpha_max=alpha_max, T_min=T_min)
    P = f["T"].shape[0]
    g4 = np.zeros((P, 4))
    g4[:, :3] = _d64(d_color).reshape(P, 3)
    gA = np.zeros(P) if d_alpha is None else _d64(d_alpha).reshape(P).copy()
    if d_acc_depth is not None:
        g4[:, 3] += _d64(d_acc_depth).reshape(P)
    if d_expected_depth is not None:
        dE = _d64(d_expected_depth).reshape(P)
        a = f["alpha"]
        ok = a > 0.0
        inv = np.where(ok, 1.0 / np.where(ok, a, 1.0), 0.0)
        g4[:, 3] += dE * inv
        gA += -dE * f["expected_depth"] * inv
    bg4 = None if bg is None else np.concatenate([_d64(bg), [0.0]])
    g2 = render_splats_bwd(f["splats"], f["colors"], cam.width, cam.height, g4, d_alpha=gA, pixels=pixels, bg=bg4,
                           alpha_min=alpha_min, alpha_max=alpha_max, T_min=T_min)
    d_sh, d_means_sh = sh_bwd(scene, cam, g2["d_colors"][:, :3])
    g3 = project_bwd(scene, cam, g2["d_means2d"], g2["d_conics"], g2["d_opacities"], d_depths=g2["d_colors"][:, 3],
                     eps2d=eps2d, near=near, antialiased=antialiased)
    return dict(d_means=g3["d_means"] + d_means_sh, d_quats=g3["d_quats"], d_log_scales=g3["d_log_scales"],
                d_opacity_logits=g3["d_opacity_logits"], d_sh=d_sh, forward=f)

"""Differentiable rasterization built on the libgs C ABI.

``rasterization(...)`` mirrors the paper's user call (Design section, Fig. 1):
Gaussians and C cameras in, images and alphas out, differentiable with respect to
means, quaternions, log-scales, opacity logits and SH coefficients (or raw
N-dimensional features).  Every stage runs in libgs kernels; PyTorch only provides
the device buffers, the stream and autograd.

Memory: the forward keeps, per pixel, only the final transmittance and the index of
the last contributor (App. D.2 replays the compositing from them), so the saved
state is O(pixels + Gaussians + intersections).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import torch

from . import _lib

__all__ = ["RasterSettings", "RasterState", "project", "sh_eval", "bin_sort", "tile_order", "rasterize_fwd",
           "forward_pass",
           "rasterization", "RasterizeGaussians"]


@dataclass
class RasterSettings:
    tile: int = 16
    batch_depth: int = 256
    antialiased: bool = False
    eps2d: float = 0.3
    near_plane: float = 0.01
    alpha_min: float = 1.0 / 255.0
    alpha_max: float = 0.99
    T_min: float = 1e-4
    background: tuple | None = None
    absgrad: bool = False
    pixels_per_thread: int = 0
    tile_schedule: bool = True  # hand the longest tile lists to the GPU first (gs_tile_order)
    bwd_batch_depth: int = 0        # backward compositing launch (0: as the forward's)
    bwd_pixels_per_thread: int = 0
    persistent: bool = False        # compositing as persistent launches over tile_schedule's order
    bwd_persistent: bool = False

    def params(self, colors_shared=False) -> _lib.GsParams:
        return _cached_params(self.tile, self.batch_depth, bool(self.antialiased), self.eps2d, self.near_plane,
                              self.alpha_min, self.alpha_max, self.T_min, self.pixels_per_thread,
                              bool(self.persistent and self.tile_schedule), bool(colors_shared))

    def params_bwd(self, colors_shared=False) -> _lib.GsParams:
        return _cached_params(self.tile, self.bwd_batch_depth or self.batch_depth, bool(self.antialiased), self.eps2d,
                              self.near_plane, self.alpha_min, self.alpha_max, self.T_min,
                              self.bwd_pixels_per_thread or self.pixels_per_thread,
                              bool(self.bwd_persistent and self.tile_schedule), bool(colors_shared))


_PARAMS: dict = {}


def _cached_params(*key) -> _lib.GsParams:
    """One launch-parameter struct per distinct setting (the calls only read it)."""
    p = _PARAMS.get(key)
    if p is None:
        tile, batch, aa, eps2d, near, amin, amax, tmin, ppt, persistent, shared = key
        p = _lib.make_params(tile, batch, aa, eps2d, near, amin, amax, tmin, ppt, persistent=persistent,
                             colors_shared=shared)
        if len(_PARAMS) < 256:
            _PARAMS[key] = p
    return p


@dataclass
class RasterState:
    """Reusable intersection buffers: grown (x1.25) when a frame needs more than they hold.

    With deferred checking (``rasterization(..., defer_sync=True)``) the forward does not wait
    for the intersection count: it is copied to host memory behind the frame and ``check()``
    (called after any later synchronisation, e.g. reading the loss) reports whether the frame
    fit; a frame that did not must be redone (the buffers have grown by then)."""
    capacity: int = 0
    values: torch.Tensor | None = None
    workspace: torch.Tensor | None = None
    tile_order: torch.Tensor | None = None
    ws_key: tuple = field(default_factory=tuple)
    pending: tuple | None = None  # (pinned K copy, event, cams, N, params, device) of a deferred frame
    redone: int = 0

    def check(self) -> bool:
        """True if the last deferred frame's lists fit; otherwise grows the buffers and returns False."""
        if self.pending is None:
            return True
        K_host, ev, cams, N, params, dev = self.pending
        self.pending = None
        ev.synchronize()
        K = int(K_host.item())
        if K <= self.capacity:
            return True
        self.ensure(cams, N, params, K, dev)
        self.redone += 1
        return False

    def ensure(self, cams, N, params, K, device):
        if K > _lib.GS_MAX_INTERSECTIONS:
            raise _lib.GsError(_lib.GS_ERR_CAPACITY, "RasterState",
                               f"{K} intersections exceed GS_MAX_INTERSECTIONS (int32 list positions): "
                               "use a larger tile or fewer cameras per call")
        if K > self.capacity or self.values is None:
            self.capacity = min(max(int(K * 1.25) + 1024, 1 << 16), _lib.GS_MAX_INTERSECTIONS)
            self.values = torch.empty(self.capacity, dtype=torch.int32, device=device)
            self.ws_key = ()
        key = (cams.C, N, self.capacity, params.tile)
        if key != self.ws_key:
            nbytes = _lib.gs_tile_bin_sort_workspace(cams, N, params, self.capacity)
            self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=device)
            self.ws_key = key


def _splat_buffers(C, N, dev):
    CN = C * N
    f = torch.empty(7 * CN, device=dev)  # means2d | depths | conics | opacities, one allocation
    i = torch.empty(2 * CN, dtype=torch.int32, device=dev)  # radii | tiles touched
    return dict(means2d=f[:2 * CN].view(C, N, 2), depths=f[2 * CN:3 * CN].view(C, N),
                conics=f[3 * CN:6 * CN].view(C, N, 3), opacities=f[6 * CN:].view(C, N),
                radii=i[:CN].view(C, N), tiles_touched=i[CN:].view(C, N))


def project(cams, means, quats, log_scales, opacity_logits, params):
    out = _splat_buffers(cams.C, means.shape[0], means.device)
    _lib.gs_project(cams, means, quats, log_scales, opacity_logits, params, out["means2d"], out["depths"],
                    out["conics"], out["radii"], out["tiles_touched"], out["opacities"])
    return out


def project_sh(cams, means, quats, log_scales, opacity_logits, params, sh_degree, sh):
    """The splats and their SH colours [C,N,3] from one kernel."""
    out = _splat_buffers(cams.C, means.shape[0], means.device)
    colors = torch.empty(cams.C, means.shape[0], 3, device=means.device)
    _lib.gs_project_sh_eval(cams, params, sh_degree, sh, means, quats, log_scales, opacity_logits, out["means2d"],
                            out["depths"], out["conics"], out["radii"], out["tiles_touched"], out["opacities"],
                            colors)
    return out, colors


def sh_eval(cams, sh_degree, sh, means, radii, depths=None, out=None):
    """SH colours [C,N,3]; with ``depths``, (r, g, b, z) rows [C,N,4] for depth rendering (App. A)."""
    ch = 3 if depths is None else 4
    colors = torch.empty(cams.C, means.shape[0], ch, device=means.device) if out is None else out
    if depths is None:
        _lib.gs_sh_eval(cams, sh_degree, sh, means, radii, colors)
    else:
        _lib.gs_sh_eval_depth(cams, sh_degree, sh, means, radii, depths, colors)
    return colors


def bin_sort(cams, N, params, means2d, depths, radii, state: RasterState | None = None, want_keys=False,
             sync=True):
    """Intersection list and tile ranges.  With ``sync`` K is read back to the host (one sync) and the
    buffers grown until the list fits; without it the sort runs once at the current capacity and the
    caller checks ``K_out`` later (the compositing needs only the device-side ranges)."""
    dev = means2d.device
    state = state or RasterState()
    if state.values is None:
        state.ensure(cams, N, params, max(4 * cams.C * N, 1 << 16), dev)
    else:
        state.ensure(cams, N, params, 0, dev)
    T = cams.num_tiles(params.tile)
    ranges = torch.empty(T, 2, dtype=torch.int32, device=dev)
    K_out = torch.zeros(1, dtype=torch.int64, device=dev)
    if not sync and not want_keys:
        _lib.gs_tile_bin_sort(cams, N, params, means2d, depths, radii, state.capacity, None, state.values, ranges,
                              K_out, state.workspace)
        return dict(values=state.values, ranges=ranges, K=None, K_out=K_out, keys=None)
    for _ in range(2):
        keys = torch.empty(state.capacity, dtype=torch.int64, device=dev) if want_keys else None
        _lib.gs_tile_bin_sort(cams, N, params, means2d, depths, radii, state.capacity, keys, state.values, ranges,
                              K_out, state.workspace)
        K = int(K_out.item())
        if K <= state.capacity:
            break
        state.ensure(cams, N, params, K, dev)
    values = state.values[:K]
    return dict(values=values, ranges=ranges, K=K, K_out=K_out, keys=None if keys is None else keys[:K])


def tile_order(cams, params, ranges):
    """Launch order of the compositing kernels: longest tile lists first."""
    order = torch.empty(ranges.shape[0] + 4, dtype=torch.int32, device=ranges.device)  # + work counters
    _lib.gs_tile_order(cams, params, ranges, order)
    return order


def rasterize_fwd(cams, N, params, channels, ranges, values, radii, means2d, conics, opacities, colors, background,
                  count_blends=False, order=None):
    dev = means2d.device
    P = cams.num_pixels
    image = torch.empty(P, channels, device=dev)
    final_T = torch.empty(P, device=dev)
    last = torch.empty(P, dtype=torch.int32, device=dev)
    blends = torch.zeros(1, dtype=torch.int64, device=dev) if count_blends else None
    if values.numel() == 0:
        values = torch.empty(1, dtype=torch.int32, device=dev)
    _lib.gs_rasterize_fwd(cams, N, params, channels, ranges, values, radii, means2d, conics, opacities, colors,
                          background, image, final_T, last, blends, tile_order=order)
    return image, final_T, last, blends


_SIDE: dict = {}
SIDE_STREAM_MIN_PAIRS = 1 << 18  # (camera, Gaussian) pairs from which SH runs beside the sort


def _side_stream(main: torch.cuda.Stream) -> torch.cuda.Stream:
    """A side stream for work that overlaps the sort, one per launching stream (so frames on
    different streams never wait on each other's side work)."""
    key = main.cuda_stream
    st = _SIDE.get(key)
    if st is None:
        if len(_SIDE) >= 64:
            _SIDE.clear()
        st = _SIDE[key] = torch.cuda.Stream(device=main.device)
    return st


def forward_pass(cams, means, quats, log_scales, opacity_logits, sh=None, sh_degree=0, features=None,
                 settings: RasterSettings | None = None, state: RasterState | None = None, count_blends=False,
                 depth=False, defer_sync=False):
    """Project, colour, bin/sort and composite.  Returns a dict of every intermediate.  With
    ``depth`` (SH colours only) the image gains a fourth channel, the accumulated depth."""
    settings = settings or RasterSettings()
    params = settings.params()
    N = means.shape[0]
    side = None
    if features is not None:
        sp, colors = project(cams, means, quats, log_scales, opacity_logits, params), features
    elif not depth:  # projection and colours in one kernel
        sp, colors = project_sh(cams, means, quats, log_scales, opacity_logits, params, sh_degree, sh)
    elif cams.C * N >= SIDE_STREAM_MIN_PAIRS:
        # depth rendering: SH colours and depths on a side stream while the bin/sort runs on
        # this one (both need only the projection; the compositing waits for both).  The
        # buffer is taken on this stream.
        sp = project(cams, means, quats, log_scales, opacity_logits, params)
        colors = torch.empty(cams.C, N, 4 if depth else 3, device=means.device)
        main = torch.cuda.current_stream(means.device)
        side = _side_stream(main)
        side.wait_stream(main)
        with torch.cuda.stream(side):
            sh_eval(cams, sh_degree, sh, means, sp["radii"], sp["depths"] if depth else None, out=colors)
    else:  # small frames: the stream switch costs more than the overlap gains
        sp = project(cams, means, quats, log_scales, opacity_logits, params)
        colors = sh_eval(cams, sh_degree, sh, means, sp["radii"], sp["depths"] if depth else None)
    ch = colors.shape[-1]
    state = state or RasterState()
    # the sort and the compositing are queued back to back; K is checked once the whole
    # forward is on the stream, and the (rare) frame whose list outgrew the buffers is redone
    for _ in range(3):
        bs = bin_sort(cams, N, params, sp["means2d"], sp["depths"], sp["radii"], state, sync=False)
        order = tile_order(cams, params, bs["ranges"]) if settings.tile_schedule else None
        if side is not None:
            torch.cuda.current_stream(means.device).wait_stream(side)
            side = None
        # features [N, D] are shared by every camera: the kernels index their rows by Gaussian
        rparams = settings.params(colors_shared=True) if colors.dim() == 2 else params
        image, final_T, last, blends = rasterize_fwd(cams, N, rparams, ch, bs["ranges"], bs["values"], sp["radii"],
                                                     sp["means2d"], sp["conics"], sp["opacities"], colors,
                                                     settings.background, count_blends, order)
        if defer_sync:
            K_host = torch.empty(1, dtype=torch.int64, pin_memory=True)
            K_host.copy_(bs["K_out"], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record()
            state.pending = (K_host, ev, cams, N, params, means.device)
            return dict(sp, colors=colors, values=state.values, ranges=bs["ranges"], K=None, image=image,
                        final_T=final_T, last_contrib=last, blends=blends, params=params, tile_order=order)
        K = int(bs["K_out"].item())
        if K <= state.capacity:
            break
        state.ensure(cams, N, params, K, means.device)
    return dict(sp, colors=colors, values=state.values[:K], ranges=bs["ranges"], K=K, image=image,
                final_T=final_T, last_contrib=last, blends=blends, params=params, tile_order=order)


class RasterizeGaussians(torch.autograd.Function):
    """image [P, ch], alpha [P], radii, expected depth [P] (empty unless asked)
    = f(means, quats, log_scales, opacity_logits, sh | features).

    depth: 0 = colour only; 1 = a fourth channel with the accumulated depth (App. A);
    2 = as 1 and the expected depth (accumulated depth / alpha) as a fourth output."""

    @staticmethod
    def forward(ctx, means, quats, log_scales, opacity_logits, sh_or_features, cams, sh_degree, settings, state,
                depth=0, viewmats=None, defer_sync=False):
        use_sh = sh_degree is not None
        if depth and not use_sh:
            raise ValueError("depth rendering needs SH colours")
        feats = None
        if not use_sh:
            feats = sh_or_features.contiguous()  # [N, D] shared by the cameras, or [C, N, D]
        if depth and settings.background is not None:
            settings = RasterSettings(**{**settings.__dict__, "background": tuple(settings.background)[:3] + (0.0,)})
        out = forward_pass(cams, means, quats, log_scales, opacity_logits, sh=sh_or_features if use_sh else None,
                           sh_degree=sh_degree if use_sh else 0, features=feats, settings=settings, state=state,
                           depth=bool(depth), defer_sync=defer_sync)
        edepth = torch.empty(0, device=means.device)
        if depth == 2:
            edepth = torch.empty(cams.num_pixels, device=means.device)
            _lib.gs_expected_depth(out["image"], 3, out["final_T"], edepth)
        ctx.cams, ctx.settings, ctx.sh_degree, ctx.use_sh, ctx.depth = cams, settings, sh_degree, use_sh, depth
        ctx.feat_dim = None if use_sh else sh_or_features.dim()
        ctx.tile_order = out["tile_order"]
        ctx.save_for_backward(means, quats, log_scales, opacity_logits, sh_or_features, out["radii"], out["means2d"],
                              out["conics"], out["opacities"], out["colors"], out["values"], out["ranges"],
                              out["final_T"], out["last_contrib"], out["image"] if depth == 2 else None)
        ctx.mark_non_differentiable(out["radii"])
        ctx.set_materialize_grads(False)  # outputs without a gradient (alpha, depth) arrive as None
        ctx.viewmats_like = viewmats  # the pose leaf, if any (its values are in cams)
        alpha = 1.0 - out["final_T"]
        return out["image"], alpha, out["radii"], edepth

    @staticmethod
    def backward(ctx, d_image, d_alpha, _d_radii, d_edepth):
        (means, quats, log_scales, logits, shf, radii, means2d, conics, opac, colors, values, ranges, final_T,
         last, image) = ctx.saved_tensors
        cams, settings = ctx.cams, ctx.settings
        params = settings.params()
        shared = colors.dim() == 2  # features [N, D]: their gradient is summed over the cameras in the kernel
        params_bwd = settings.params_bwd(colors_shared=shared)
        C, N = cams.C, means.shape[0]
        ch = colors.shape[-1]
        dev = means.device
        rows = N if shared else C * N
        g2d = torch.zeros(C * N * 6 + rows * ch, device=dev)  # one memset for all accumulated 2D gradients
        d_means2d = g2d[:C * N * 2].view(C, N, 2)
        d_conics = g2d[C * N * 2:C * N * 5].view(C, N, 3)
        d_opac = g2d[C * N * 5:C * N * 6].view(C, N)
        d_colors = g2d[C * N * 6:].view(N, ch) if shared else g2d[C * N * 6:].view(C, N, ch)
        absgrad = torch.zeros(C, N, 2, device=dev) if settings.absgrad else None
        d_image = d_image.contiguous() if d_image is not None else torch.zeros(cams.num_pixels, ch, device=dev)
        d_alpha = d_alpha.contiguous() if d_alpha is not None else None
        if ctx.depth == 2 and d_edepth is not None and d_edepth.numel():
            d_image = d_image.clone()
            d_alpha = d_alpha.clone() if d_alpha is not None else torch.zeros(cams.num_pixels, device=dev)
            _lib.gs_expected_depth_bwd(image, 3, final_T, d_edepth.contiguous(), d_image, d_alpha)
        vals = values if values.numel() else torch.empty(1, dtype=torch.int32, device=dev)
        _lib.gs_rasterize_bwd(cams, N, params_bwd, ch, ranges, vals, radii, means2d, conics, opac, colors,
                              settings.background, final_T, last, d_image, d_alpha, d_means2d, d_conics, d_opac,
                              d_colors, absgrad, tile_order=ctx.tile_order)
        if absgrad is not None:
            RasterizeGaussians.last_absgrad = absgrad
        d_means = torch.empty(N, 3, device=dev)
        d_depths = None
        want_pose = ctx.viewmats_like is not None and ctx.needs_input_grad[10]
        d_view = torch.zeros(C, 4, 4, device=dev) if want_pose else None
        if ctx.use_sh and C == 1 and not ctx.depth and d_view is None:
            # one camera: SH and projection backward in one kernel
            d_sh = torch.empty_like(shf)
            d_quats = torch.empty(N, 4, device=dev)
            d_log_scales = torch.empty(N, 3, device=dev)
            d_logits = torch.empty(N, device=dev)
            _lib.gs_sh_project_bwd(cams, params, ctx.sh_degree, shf, means, quats, log_scales, logits, radii, d_colors,
                                   d_means2d, d_conics, d_opac, d_sh, d_means, d_quats, d_log_scales, d_logits)
            return d_means, d_quats, d_log_scales, d_logits, d_sh, None, None, None, None, None, None, None
        if ctx.use_sh:
            d_sh = torch.empty_like(shf)
            if ctx.depth:
                d_depths = torch.empty(C, N, device=dev)
                _lib.gs_sh_eval_depth_bwd(cams, ctx.sh_degree, shf, means, radii, d_colors, d_sh, d_means, d_depths,
                                          d_viewmats=d_view)
            else:
                _lib.gs_sh_eval_bwd(cams, ctx.sh_degree, shf, means, radii, d_colors, d_sh, d_means,
                                    d_viewmats=d_view)
            d_feat = d_sh
        else:
            d_means.zero_()
            d_feat = d_colors  # [N, D] accumulated over the cameras by the kernel, or [C, N, D]
        d_quats = torch.empty(N, 4, device=dev)
        d_log_scales = torch.empty(N, 3, device=dev)
        d_logits = torch.empty(N, device=dev)
        _lib.gs_project_bwd(cams, means, quats, log_scales, logits, params, radii, d_means2d, d_conics, d_opac,
                            d_depths, d_means, d_quats, d_log_scales, d_logits, d_viewmats=d_view)
        if d_view is not None:
            d_view = d_view.to(ctx.viewmats_like.device).reshape(ctx.viewmats_like.shape)
        return d_means, d_quats, d_log_scales, d_logits, d_feat, None, None, None, None, None, d_view, None


RENDER_MODES = {"RGB": 0, "D": 1, "ED": 2, "RGB+D": 1, "RGB+ED": 2}


def rasterization(means, quats, log_scales, opacity_logits, sh=None, cameras=None, *, features=None,
                  sh_degree=None, settings: RasterSettings | None = None, state: RasterState | None = None,
                  render_mode: str = "RGB", viewmats=None, defer_sync: bool = False):
    """Render C cameras.  Returns (images, alphas, meta) with one [H, W, ch] / [H, W] tensor per camera.

    Pass SH coefficients ``sh`` [N, K, 3] (degree inferred from K) or N-dimensional
    ``features`` [N, D] / [C, N, D].  Parameters are the leaves of the paper's
    gradient-flow figure: log-scales and opacity logits.  ``render_mode`` (SH colours):
    "RGB"; "D" / "RGB+D" with the accumulated depth sum z alpha T; "ED" / "RGB+ED" with the
    expected depth, the accumulated depth over alpha (App. A).  ``viewmats`` [C,4,4]
    (world->camera, any device) replaces the cameras' poses; when it requires grad, the pose
    gradient (App. A) flows back to it.  ``defer_sync`` (needs ``state``): do not wait for the
    intersection count; call ``state.check()`` after the next synchronisation and redo the frame
    when it returns False.
    """
    if cameras is None:
        raise ValueError("cameras are required")
    if render_mode not in RENDER_MODES:
        raise ValueError(f"render_mode must be one of {sorted(RENDER_MODES)}")
    if defer_sync and state is None:
        raise ValueError("defer_sync needs a RasterState to report through")
    depth = RENDER_MODES[render_mode]
    if viewmats is not None:
        vm = viewmats.detach().reshape(-1, 4, 4).cpu().numpy()
        base = list(cameras.cams) if isinstance(cameras, _lib.CameraArray) else list(cameras)
        if len(base) != vm.shape[0]:
            raise ValueError("viewmats must hold one 4x4 matrix per camera")
        cameras = [(*(c.as_tuple()[:2] if hasattr(c, "as_tuple") else c[:2]), vm[i],
                    *(c.as_tuple()[3:] if hasattr(c, "as_tuple") else c[3:])) for i, c in enumerate(base)]
    cams = cameras if isinstance(cameras, _lib.CameraArray) else _lib.CameraArray(cameras)
    settings = settings or RasterSettings()
    if features is None:
        if sh is None:
            raise ValueError("give sh or features")
        K = sh.shape[1]
        sh_degree = {1: 0, 4: 1, 9: 2, 16: 3}[K] if sh_degree is None else sh_degree
        img, alpha, radii, edepth = RasterizeGaussians.apply(means, quats, log_scales, opacity_logits, sh, cams,
                                                             sh_degree, settings, state, depth, viewmats,
                                                             defer_sync)
    else:
        if depth:
            raise ValueError("depth render modes need SH colours")
        img, alpha, radii, edepth = RasterizeGaussians.apply(means, quats, log_scales, opacity_logits, features,
                                                             cams, None, settings, state, 0, viewmats, defer_sync)
    if depth == 2:
        img = torch.cat([img[:, :3], edepth[:, None]], dim=1)
    if render_mode in ("D", "ED"):
        img = img[:, 3:4]
    images, alphas = [], []
    for (w, h), off in zip(cams.sizes, cams.pixel_offsets()):
        images.append(img[off:off + w * h].view(h, w, -1))
        alphas.append(alpha[off:off + w * h].view(h, w))
    return images, alphas, dict(radii=radii, cameras=cams)

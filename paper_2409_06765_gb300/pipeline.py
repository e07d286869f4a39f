"""Preallocated frame pipeline over the C ABI: every buffer of a forward (+ backward) pass of
C cameras over one resident scene, sized once, reused every frame, and replayable as CUDA
graphs.

One frame is project -> SH -> bin/sort (+ tile order) -> composite (App. C.2), and the
backward composite -> SH backward -> projection backward (App. D).  The intersection count K
is data dependent; the pipeline sizes its buffers from a real frame and keeps a margin, and
``frame_overflowed()`` tells (after a sync) whether a later frame needed more.  No call in
a frame synchronises the host, so the stages before and after the two compositing kernels
can be captured as CUDA graphs (``capture_graphs``), which removes the launch gaps of their
~30 short kernels; the compositing kernels themselves are launched directly so that events
can bracket them.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from . import _lib

__all__ = ["Schedule", "DeviceScene", "FramePipeline"]


@dataclass(frozen=True)
class Schedule:
    """Launch parameters of the pipeline; the rendered result does not depend on them.

    The tile size fixes the intersection lists for both compositing kernels; each kernel has
    its own batch depth and pixels per thread (bwd_* = 0: the same as the forward's)."""
    tile: int = 16
    batch_depth: int = 128
    pixels_per_thread: int = 2
    tile_order: bool = True
    bwd_batch_depth: int = 0
    bwd_pixels_per_thread: int = 0
    persistent: bool = False      # forward compositing as one persistent launch (needs tile_order)
    bwd_persistent: bool = False  # backward likewise
    fused_bwd: bool = True        # one camera: SH and projection backward as one kernel
    fused_fwd: bool = True        # projection and SH colours as one kernel

    def params(self) -> _lib.GsParams:
        return _lib.make_params(tile=self.tile, batch_depth=self.batch_depth, pixels_per_thread=self.pixels_per_thread,
                                persistent=self.persistent and self.tile_order)

    def params_bwd(self) -> _lib.GsParams:
        return _lib.make_params(tile=self.tile, batch_depth=self.bwd_batch_depth or self.batch_depth,
                                pixels_per_thread=self.bwd_pixels_per_thread or self.pixels_per_thread,
                                persistent=self.bwd_persistent and self.tile_order)

    def as_dict(self):
        return dict(tile=self.tile, batch_depth=self.batch_depth, pixels_per_thread=self.pixels_per_thread,
                    bwd_batch_depth=self.bwd_batch_depth or self.batch_depth,
                    bwd_pixels_per_thread=self.bwd_pixels_per_thread or self.pixels_per_thread,
                    tile_order=self.tile_order, persistent=self.persistent, bwd_persistent=self.bwd_persistent,
                    fused_bwd=self.fused_bwd, fused_fwd=self.fused_fwd)


class DeviceScene:
    """A scene's parameters resident on the device (float32, contiguous)."""

    def __init__(self, means, quats, log_scales, opacity_logits, sh, sh_degree):
        self.means, self.quats, self.log_scales = means, quats, log_scales
        self.opacity_logits, self.sh, self.sh_degree = opacity_logits, sh, int(sh_degree)
        self.n = int(means.shape[0])

    @classmethod
    def from_host(cls, scene, device="cuda"):
        t = lambda a: torch.as_tensor(np.ascontiguousarray(a, np.float32), device=device)
        return cls(t(scene.means), t(scene.quats), t(scene.log_scales), t(scene.opacity_logits), t(scene.sh),
                   scene.sh_degree)

    @property
    def nbytes(self) -> int:
        return sum(x.numel() * 4 for x in (self.means, self.quats, self.log_scales, self.opacity_logits, self.sh))


class FramePipeline:
    """Buffers and launches of one frame of C cameras over one DeviceScene."""

    def __init__(self, scene: DeviceScene, cams, schedule: Schedule = Schedule(), backward: bool = True,
                 capacity: int | None = None, margin: float = 1.1, side_stream: torch.cuda.Stream | None = None):
        self.scene = scene
        self.cams = cams if isinstance(cams, _lib.CameraArray) else _lib.CameraArray(cams)
        self.schedule = schedule
        self.params = schedule.params()
        self.params_bwd = schedule.params_bwd()
        self.with_backward = backward
        C, N = self.cams.C, scene.n
        self.C, self.N = C, N
        dev = scene.means.device
        self.device = dev
        f = lambda *s: torch.empty(*s, device=dev)
        i = lambda *s: torch.empty(*s, dtype=torch.int32, device=dev)
        self.means2d, self.depths, self.conics = f(C, N, 2), f(C, N), f(C, N, 3)
        self.radii, self.tiles, self.opac, self.colors = i(C, N), i(C, N), f(C, N), f(C, N, 3)
        self.P = self.cams.num_pixels
        self.T = self.cams.num_tiles(schedule.tile)
        self.image, self.final_T, self.last = f(self.P, 3), f(self.P), i(self.P)
        self.ranges = i(self.T, 2)
        self.order = i(self.T + 4) if schedule.tile_order else None  # order, then the work counters
        self.K_out = torch.zeros(1, dtype=torch.int64, device=dev)
        if backward:
            # 2D gradients in one allocation so that one memset clears them
            self.g2d = torch.zeros(C * N * 9, device=dev)
            o = 0
            self.d_means2d = self.g2d[o:o + C * N * 2].view(C, N, 2); o += C * N * 2
            self.d_conics = self.g2d[o:o + C * N * 3].view(C, N, 3); o += C * N * 3
            self.d_opac = self.g2d[o:o + C * N].view(C, N); o += C * N
            self.d_colors = self.g2d[o:o + C * N * 3].view(C, N, 3)
            self.d_sh, self.d_means = torch.empty_like(scene.sh), f(N, 3)
            self.d_quats, self.d_log_scales, self.d_logits = f(N, 4), f(N, 3), f(N)
            self.d_image = torch.zeros(self.P, 3, device=dev)
        self.g_pre = self.g_post = None
        # SH colours overlap the bin/sort.  (torch hands out streams round-robin from a small
        # pool, so callers running several pipelines at once pass a side stream of their own:
        # a side stream shared with another frame's main stream would chain the two frames.)
        self.side = side_stream if side_stream is not None else torch.cuda.Stream(dev)
        self.margin = margin
        self.K = None
        if capacity is None:
            self.capacity = 1 << 20
            self._alloc_sort()
            self.size_from_frame()
        else:
            self.capacity = int(capacity)
            self._alloc_sort()

    # -- buffers ---------------------------------------------------------------------------
    def _alloc_sort(self):
        self.values = torch.empty(max(self.capacity, 1), dtype=torch.int32, device=self.device)
        nbytes = _lib.gs_tile_bin_sort_workspace(self.cams, self.N, self.params, self.capacity)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.g_pre = self.g_post = None  # graphs hold the old pointers

    def size_from_frame(self):
        """Run the pre-compositing stages once and grow the intersection buffers to fit K."""
        for _ in range(2):
            self._pre()
            torch.cuda.synchronize(self.device)
            K = int(self.K_out.item())
            if K <= self.capacity:
                self.K = K
                return K
            if K > _lib.GS_MAX_INTERSECTIONS:
                raise _lib.GsError(_lib.GS_ERR_CAPACITY, "FramePipeline",
                                   f"{K} intersections exceed GS_MAX_INTERSECTIONS (int32 list positions): "
                                   "use a larger tile or fewer cameras per call")
            self.capacity = min(int(K * self.margin) + 1024, _lib.GS_MAX_INTERSECTIONS)
            self._alloc_sort()
        raise RuntimeError("intersection count did not settle")

    def frame_overflowed(self) -> bool:
        """After a synchronise: did the last frame need more intersections than the buffers hold?"""
        K = int(self.K_out.item())
        self.K = K
        return K > self.capacity

    @property
    def device_bytes(self) -> int:
        """Bytes of every buffer this pipeline owns (the scene's parameters excluded)."""
        total = 0
        for v in self.__dict__.values():
            if isinstance(v, torch.Tensor) and v.device.type == "cuda" and v._base is None:
                total += v.numel() * v.element_size()
        return total

    # -- stages ----------------------------------------------------------------------------
    @property
    def fused_fwd(self) -> bool:
        return self.schedule.fused_fwd

    def _pre(self):
        # project, then SH colours (and the zeroing of the 2D gradient buffer) on a side stream
        # while the bin/sort runs on this one: the SH kernel streams coefficients from HBM while
        # the sort's many short, latency-bound kernels leave bandwidth idle; both only need the
        # projection, and the compositing waits for both.  With fused_fwd (the default):
        # projection and colours as one kernel before the sort.
        s, L = self.scene, _lib
        main = torch.cuda.current_stream(self.device)
        if self.fused_fwd:
            L.gs_project_sh_eval(self.cams, self.params, s.sh_degree, s.sh, s.means, s.quats, s.log_scales,
                                 s.opacity_logits, self.means2d, self.depths, self.conics, self.radii, self.tiles,
                                 self.opac, self.colors)
        else:
            L.gs_project(self.cams, s.means, s.quats, s.log_scales, s.opacity_logits, self.params, self.means2d,
                         self.depths, self.conics, self.radii, self.tiles, self.opac)
        side_work = not self.fused_fwd or self.with_backward
        if side_work:
            self.side.wait_stream(main)
            with torch.cuda.stream(self.side):
                if not self.fused_fwd:
                    L.gs_sh_eval(self.cams, s.sh_degree, s.sh, s.means, self.radii, self.colors)
                if self.with_backward:
                    self.g2d.zero_()  # the 2D gradients the compositing backward accumulates into
        L.gs_tile_bin_sort(self.cams, self.N, self.params, self.means2d, self.depths, self.radii, self.capacity, None,
                           self.values, self.ranges, self.K_out, self.workspace)
        if self.order is not None:
            L.gs_tile_order(self.cams, self.params, self.ranges, self.order)
        if side_work:
            main.wait_stream(self.side)

    def _raster_fwd(self, count=None):
        _lib.gs_rasterize_fwd(self.cams, self.N, self.params, 3, self.ranges, self.values, self.radii, self.means2d,
                              self.conics, self.opac, self.colors, None, self.image, self.final_T, self.last, count,
                              tile_order=self.order)

    def _raster_bwd(self):
        _lib.gs_rasterize_bwd(self.cams, self.N, self.params_bwd, 3, self.ranges, self.values, self.radii, self.means2d,
                              self.conics, self.opac, self.colors, None, self.final_T, self.last, self.d_image, None,
                              self.d_means2d, self.d_conics, self.d_opac, self.d_colors, None, tile_order=self.order)

    @property
    def fused_bwd(self) -> bool:
        return self.C == 1 and self.schedule.fused_bwd

    def _post(self):
        s, L = self.scene, _lib
        if self.fused_bwd:
            L.gs_sh_project_bwd(self.cams, self.params, s.sh_degree, s.sh, s.means, s.quats, s.log_scales,
                                s.opacity_logits, self.radii, self.d_colors, self.d_means2d, self.d_conics, self.d_opac,
                                self.d_sh, self.d_means, self.d_quats, self.d_log_scales, self.d_logits)
            return
        L.gs_sh_eval_bwd(self.cams, s.sh_degree, s.sh, s.means, self.radii, self.d_colors, self.d_sh, self.d_means)
        L.gs_project_bwd(self.cams, s.means, s.quats, s.log_scales, s.opacity_logits, self.params, self.radii,
                         self.d_means2d, self.d_conics, self.d_opac, None, self.d_means, self.d_quats,
                         self.d_log_scales, self.d_logits)

    # -- graphs ----------------------------------------------------------------------------
    def capture_graphs(self):
        """Capture the stages before and after the compositing kernels as CUDA graphs."""
        side = torch.cuda.Stream(self.device)
        side.wait_stream(torch.cuda.current_stream(self.device))
        with torch.cuda.stream(side):  # warm-up on the capture stream
            self._pre()
            if self.with_backward:
                self._post()
        torch.cuda.current_stream(self.device).wait_stream(side)
        torch.cuda.synchronize(self.device)
        n0 = _lib.gs_kernel_launches()
        self.g_pre = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.g_pre):
            self._pre()
        if self.with_backward:
            self.g_post = torch.cuda.CUDAGraph()
            with torch.cuda.graph(self.g_post):
                self._post()
        torch.cuda.synchronize(self.device)
        self.graph_kernels = _lib.gs_kernel_launches() - n0

    # -- public steps ----------------------------------------------------------------------
    def forward(self, events=None, count=None, graphs=False):
        if graphs and self.g_pre is None:
            self.capture_graphs()
        if graphs:
            self.g_pre.replay()
        else:
            self._pre()
        if events:
            events[0].record()
        self._raster_fwd(count)
        if events:
            events[1].record()

    def backward(self, events=None, graphs=False):
        if not self.with_backward:
            raise RuntimeError("pipeline built without backward buffers")
        if events:
            events[0].record()
        self._raster_bwd()
        if events:
            events[1].record()
        if graphs:
            self.g_post.replay()
        else:
            self._post()

    def step(self, graphs=False):
        self.forward(graphs=graphs)
        if self.with_backward:
            self.backward(graphs=graphs)

    def count_blends(self) -> int:
        cnt = torch.zeros(1, dtype=torch.int64, device=self.device)
        self.forward(count=cnt)
        torch.cuda.synchronize(self.device)
        return int(cnt.item())

    def set_loss_gradient(self, target):
        """Upstream gradient of the mean L1 loss at the current image (held fixed while timing)."""
        self.d_image.copy_(torch.sign(self.image - target) / self.image.numel())

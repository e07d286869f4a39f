"""Render serving with continuous batching over resident scenes.

Several scenes' Gaussians stay resident on the device.  Forward-only render requests
(scene, camera) arrive over time; the server

* admits an arrived request into its scene's queue,
* forms a batch from whatever has arrived: the scene whose oldest request has waited
  longest first (up to ``max_views`` cameras of any mix of sizes, and by default at most 2048
  tiles per scene group so that its sort stays one counting pass), then, with ``max_groups`` > 1,
  the next-oldest scenes while the batch has room.  Each scene group of the batch is one
  multi-camera call (C > 1, per-camera tile lists, one launch per stage); the groups of a
  batch run back to back on one stream and retire together,
* launches the batch on a free CUDA stream of a small pool, so batches overlap on the
  device, as long as the device memory the batch needs (its buffers, sized from the
  request sizes) fits in the free-HBM budget left by the batches in flight; otherwise the
  batch waits until enough in-flight work retires,
* retires a batch when its stream's event completes: the images (already copied to
  pinned host memory on the batch's stream) are handed back and the batch's memory is
  returned to the budget.  A scene group whose intersection lists outgrew their estimate
  is rendered again with the exact size (at most ``max_retries`` times, admitted against
  the memory budget like a new batch).

The unbatched single-view path is the same loop with one view per batch.  A camera's image
does not depend on the batch it was rendered in (its tile lists hold only its own
Gaussians, in the same order), so batching changes latency, never pixels.

``plan_batch`` holds the batching decision as a pure function so that it can be tested
without a GPU.
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np
import torch

from . import _lib, synth
from .pipeline import DeviceScene, FramePipeline, Schedule

__all__ = ["Request", "Result", "ResidentScenes", "plan_batch", "batch_bytes", "Server", "poisson_trace",
           "latency_summary"]


@dataclass
class Request:
    rid: int
    scene: int
    camera: synth.Camera
    arrival: float  # seconds from the start of the trace


@dataclass
class Result:
    rid: int
    scene: int
    image: np.ndarray | None  # [H, W, 3] float32 (host); None when the server keeps no images
    arrival: float
    launched: float
    done: float
    batch_views: int
    batch: int = -1  # serial number of the batch that rendered it

    @property
    def latency(self) -> float:
        return self.done - self.arrival


# --------------------------------------------------------------------------------------
# batching decision (pure)
# --------------------------------------------------------------------------------------

def plan_batch(queues: dict, max_views: int, budget_free: int, estimate, group_ok=None, max_groups: int = 8):
    """Pick the next batch: a list of scene groups [(scene, requests), ...].

    queues: scene id -> list of queued requests (arrival order).  Scenes are visited in the
    order of their oldest request (longest wait first); each takes its queued requests in
    arrival order while the batch has fewer than ``max_views`` cameras, the estimated device
    bytes of all its groups (``estimate(scene, requests)`` per group) fit in ``budget_free``
    and ``group_ok(scene, requests)`` (when given) accepts the group.  A request that the
    group rule alone turns down is left for a later batch (it is taken first there).
    Returns None when nothing fits (the caller waits for in-flight work to retire): the
    oldest request of the oldest scene is never overtaken by younger ones.
    """
    order = sorted((q[0].arrival, sid) for sid, q in queues.items() if q)
    groups, views, used = [], 0, 0
    for _, sid in order:
        if views >= max_views or len(groups) >= max_groups:
            break
        take = []
        for req in queues[sid][:max_views - views]:
            if take and group_ok is not None and not group_ok(sid, take + [req]):
                break
            if used + estimate(sid, take + [req]) > budget_free:
                break
            take.append(req)
        if not take:
            break  # the next scene's oldest request does not fit: the batch ends here
        used += estimate(sid, take)
        groups.append((sid, take))
        views += len(take)
        nxt = queues[sid][len(take)] if len(take) < len(queues[sid]) else None
        if nxt is not None and views < max_views and (group_ok is None or group_ok(sid, take + [nxt])):
            break  # this scene's next request did not fit the budget
    return groups or None


# --------------------------------------------------------------------------------------
# resident scenes and per-batch memory
# --------------------------------------------------------------------------------------

class ResidentScenes:
    """Scenes kept on the device, admitted by free HBM, with an intersections-per-pixel rate
    per scene (measured on one calibration frame) to size a batch's buffers."""

    def __init__(self, device="cuda", reserve_bytes: int = 2 << 30):
        self.device = torch.device(device)
        self.reserve = reserve_bytes
        self.scenes: dict[int, DeviceScene] = {}
        self.k_rate: dict[int, float] = {}

    def add(self, sid: int, host_scene, calib_camera=None, schedule: Schedule = Schedule(), calib_poses: int = 4):
        need = host_scene.means.nbytes + host_scene.quats.nbytes + host_scene.log_scales.nbytes + \
            host_scene.opacity_logits.nbytes + host_scene.sh.nbytes
        free, _ = torch.cuda.mem_get_info(self.device)
        if need + self.reserve > free:
            raise MemoryError(f"scene {sid} needs {need} bytes, {free - self.reserve} free")
        ds = DeviceScene.from_host(host_scene, device=self.device)
        self.scenes[sid] = ds
        # intersections per pixel: the largest over a few poses (the server raises it further
        # whenever a batch overflows its estimate)
        cams = [calib_camera] if calib_camera else synth.sphere_cameras(1234 + sid, [(1280, 720)] * calib_poses)
        rate = 0.0
        for cam in cams:
            pipe = FramePipeline(ds, [cam], schedule, backward=False)
            rate = max(rate, max(pipe.K, 1) / float(cam.width * cam.height))
            del pipe
        self.k_rate[sid] = rate
        return ds


def batch_bytes(scene: DeviceScene, cams, schedule: Schedule, capacity: int) -> int:
    """Device bytes a forward-only FramePipeline of these cameras allocates."""
    ca = cams if isinstance(cams, _lib.CameraArray) else _lib.CameraArray(cams)
    C, N = ca.C, scene.n
    P, T = ca.num_pixels, ca.num_tiles(schedule.tile)
    per_pair = 8 + 4 + 12 + 4 + 4 + 4 + 12  # means2d, depth, conic, radius, tiles, opacity, colour
    ws = _lib.gs_tile_bin_sort_workspace(ca, N, schedule.params(), capacity)
    return C * N * per_pair + P * (12 + 4 + 4) + T * 12 + 4 * capacity + ws + 8


# --------------------------------------------------------------------------------------
# the server
# --------------------------------------------------------------------------------------

@dataclass
class _Group:
    sid: int
    reqs: list
    pipe: FramePipeline
    capacity: int
    nbytes: int
    host_off: int          # first float of this group's images in the batch's pinned buffer
    k_slot: int            # index of this group's intersection count in the batch's count buffer
    offsets: list = field(default_factory=list)


@dataclass
class _Batch:
    groups: list
    stream: torch.cuda.Stream
    event: torch.cuda.Event
    host_img: torch.Tensor
    host_k: torch.Tensor
    nbytes: int
    launched: float
    serial: int = -1

    @property
    def views(self) -> int:
        return sum(len(g.reqs) for g in self.groups)


class Server:
    """Continuous-batching render server (forward only) over ResidentScenes."""

    def __init__(self, store: ResidentScenes, schedule: Schedule = Schedule(), max_views: int = 8, streams: int = 4,
                 budget_bytes: int | None = None, k_margin: float = 1.5, max_retries: int = 3,
                 max_group_tiles: int | None = 2048, max_groups: int = 1):
        self.store = store
        self.schedule = schedule
        self.max_views = max(1, min(int(max_views), _lib.GS_MAX_CAMERAS))
        self.streams = [torch.cuda.Stream(store.device) for _ in range(max(1, streams))]
        # one side stream per stream, from the high-priority pool: torch hands out pooled
        # streams round-robin, and a side stream that is another batch's stream would chain
        # the two batches
        self.sides = {s.cuda_stream: torch.cuda.Stream(store.device, priority=-1) for s in self.streams}
        free, _ = torch.cuda.mem_get_info(store.device)
        self.budget = budget_bytes if budget_bytes is not None else max(0, free - store.reserve)
        self.k_margin = k_margin
        self.max_retries = int(max_retries)
        # a scene group's views share one sort: up to 2048 tiles it is the single counting pass
        # over whole tile ids, beyond that LSD passes over materialised lists, which cost more
        # than the group saves by sharing the scene's parameter and coefficient reads; so by
        # default a group stays within 2048 tiles (a single view above it still renders, alone).
        # At saturation, 4 streams, mixed sizes: 1472 frames/s capped, 1386 uncapped, 1392-1406
        # one view per batch; 640x480 only: 1880, 1858 and 1518-1528.  None lifts the cap.
        self.max_group_tiles = max_group_tiles
        # scene groups per batch: groups of different scenes share no GPU work (each is its own
        # call), so by default a batch is one scene's views; more groups only pack the launches
        self.max_groups = max(1, int(max_groups))
        self.overflows = 0
        self.batches = 0
        self.groups = 0
        self.waits_for_memory = 0
        # pinned host buffers per stream (a stream carries one batch at a time): allocating
        # page-locked memory per batch costs milliseconds and stalls the loop
        self._pinned = {}

    # capacity of a group's intersection buffers from the scene's intersections per pixel
    def _capacity(self, sid, reqs, hint=0):
        px = sum(r.camera.width * r.camera.height for r in reqs)
        est = int(px * self.store.k_rate[sid] * self.k_margin) + 65536
        return min(max(est, int(hint)), _lib.GS_MAX_INTERSECTIONS)

    def _group_ok(self, sid, reqs):
        if self.max_group_tiles is None:
            return True
        t = self.schedule.tile
        tiles = sum(((r.camera.width + t - 1) // t) * ((r.camera.height + t - 1) // t) for r in reqs)
        return tiles <= self.max_group_tiles

    def _estimate(self, sid, reqs, hint=0):
        if not reqs:
            return 0
        cams = [r.camera for r in reqs]
        return batch_bytes(self.store.scenes[sid], cams, self.schedule, self._capacity(sid, reqs, hint))

    def _launch(self, groups, stream, now, hints=None):
        """Render the scene groups [(scene, requests), ...] back to back on `stream`."""
        hints = hints or [0] * len(groups)
        pix = [sum(r.camera.width * r.camera.height for r in reqs) for _, reqs in groups]
        host_img, host_k = self._host_buffers(stream, 3 * sum(pix), len(groups))
        out, off, nbytes = [], 0, 0
        with torch.cuda.stream(stream):
            for k, ((sid, reqs), hint) in enumerate(zip(groups, hints)):
                scene = self.store.scenes[sid]
                cams = [r.camera for r in reqs]
                cap = self._capacity(sid, reqs, hint)
                nb = batch_bytes(scene, cams, self.schedule, cap)
                pipe = FramePipeline(scene, cams, self.schedule, backward=False, capacity=cap,
                                     side_stream=self.sides[stream.cuda_stream])
                pipe.forward()
                n = pipe.image.numel()
                host_img[off:off + n].copy_(pipe.image.view(-1), non_blocking=True)
                host_k[k:k + 1].copy_(pipe.K_out, non_blocking=True)
                out.append(_Group(sid, reqs, pipe, cap, nb, off, k, offsets=pipe.cams.pixel_offsets()))
                off += n
                nbytes += nb
            ev = torch.cuda.Event()
            ev.record(stream)
        self.batches += 1
        self.groups += len(groups)
        return _Batch(out, stream, ev, host_img, host_k, nbytes, now, self.batches)

    def _host_buffers(self, stream, floats, groups):
        """The stream's pinned image buffer (grown when a batch needs more) and count slots."""
        img, k = self._pinned.get(stream.cuda_stream, (None, None))
        if img is None or img.numel() < floats:  # grow geometrically: few page-locked allocations
            img = torch.empty(max(floats, 2 * (img.numel() if img is not None else 0), 1 << 20), dtype=torch.float32,
                              pin_memory=True)
        if k is None or k.numel() < groups:
            k = torch.empty(max(groups, _lib.GS_MAX_CAMERAS), dtype=torch.int64, pin_memory=True)
        self._pinned[stream.cuda_stream] = (img, k)
        return img, k

    def serve(self, requests, realtime=True, poll_sleep=50e-6, keep_images=True, on_image=None):
        """Serve a trace; returns the results in completion order.  With realtime=False every
        request counts as arrived at once (a saturation run: the queues start full).

        Every image reaches page-locked host memory.  With ``keep_images`` each result holds a
        copy of its image; without, ``on_image(result, view)`` (when given) sees each image as a
        view into the stream's host buffer, valid only during the call, and results hold None
        (a long trace of 1080p images would otherwise fill host memory)."""
        pending = deque(sorted(requests, key=lambda r: r.arrival))
        queues: dict[int, list] = {sid: [] for sid in self.store.scenes}
        free_streams = list(self.streams)
        inflight: list[_Batch] = []
        reserved = 0
        results = []
        retry: list = []  # (scene, requests, capacity hint, attempts) of groups whose lists outgrew their buffers
        t0 = time.perf_counter()
        clock = lambda: time.perf_counter() - t0
        while pending or inflight or retry or any(queues.values()):
            now = clock()
            while pending and (not realtime or pending[0].arrival <= now):
                r = pending.popleft()
                queues[r.scene].append(r)
            progressed = False
            # retire finished batches
            for b in list(inflight):
                if not b.event.query():
                    continue
                inflight.remove(b)
                free_streams.append(b.stream)
                reserved -= b.nbytes
                done = clock()
                img = b.host_img.numpy()
                for g in b.groups:
                    K = int(b.host_k[g.k_slot].item())
                    px = sum(r.camera.width * r.camera.height for r in g.reqs)
                    if K > 0:  # learn the scene's intersections per pixel from every group
                        self.store.k_rate[g.sid] = max(self.store.k_rate[g.sid], K / px)
                    if K > g.capacity:
                        self.overflows += 1
                        attempts = getattr(g, "attempts", 0) + 1
                        if attempts > self.max_retries:
                            raise RuntimeError(f"scene {g.sid}: intersection lists still outgrew their buffers after "
                                               f"{self.max_retries} retries")
                        retry.append((g.sid, g.reqs, int(K * 1.1) + 1024, attempts))
                        continue
                    for r, off in zip(g.reqs, g.offsets):
                        P = r.camera.width * r.camera.height
                        o = g.host_off + 3 * off
                        view = img[o:o + 3 * P].reshape(r.camera.height, r.camera.width, 3)
                        res = Result(r.rid, r.scene, view.copy() if keep_images else None, r.arrival, b.launched,
                                     done, b.views, b.serial)
                        if on_image is not None:
                            on_image(res, view)
                        results.append(res)
                del b
                progressed = True
            # launch: overflowed groups first (each alone, admitted by memory), then new batches
            while free_streams and retry:
                sid, reqs, hint, attempts = retry[0]
                need = self._estimate(sid, reqs, hint)
                if need > self.budget - reserved:
                    if not inflight:
                        raise MemoryError(f"scene {sid}: a retried group needs {need} bytes, the budget is "
                                          f"{self.budget - reserved}")
                    break  # wait for in-flight work to retire
                retry.pop(0)
                b = self._launch([(sid, reqs)], free_streams.pop(0), now, [hint])
                b.groups[0].attempts = attempts
                reserved += b.nbytes
                inflight.append(b)
                progressed = True
            while free_streams and not retry:
                plan = plan_batch(queues, self.max_views, self.budget - reserved, self._estimate, self._group_ok,
                                  self.max_groups)
                if plan is None:
                    if any(queues.values()):
                        self.waits_for_memory += 1 if inflight else 0
                        if not inflight:
                            raise MemoryError("a single request does not fit in the memory budget")
                    break
                for sid, reqs in plan:
                    for r in reqs:
                        queues[sid].remove(r)
                b = self._launch(plan, free_streams.pop(0), now)
                reserved += b.nbytes
                inflight.append(b)
                progressed = True
            if not progressed:
                if realtime and (pending or not inflight):
                    time.sleep(poll_sleep)
                elif inflight:
                    inflight[0].event.synchronize()
        for s in self.streams:
            s.synchronize()
        return results


# --------------------------------------------------------------------------------------
# traces and statistics
# --------------------------------------------------------------------------------------

SERVING_SIZES = [(640, 480), (1280, 720), (1920, 1080)]


def poisson_trace(rate_hz: float, duration_s: float, n_scenes: int, seed: int, sizes=SERVING_SIZES, start_s=0.0):
    """Requests arriving as a Poisson process: uniform scene, random pose on the radius-6
    sphere, size uniform over ``sizes``."""
    rng = np.random.default_rng(seed)
    t, rid, out = start_s, 0, []
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t >= start_s + duration_s:
            break
        w, h = sizes[int(rng.integers(0, len(sizes)))]
        cam = synth.sphere_cameras(int(rng.integers(0, 2**31 - 1)), [(w, h)])[0]
        out.append(Request(rid, int(rng.integers(0, n_scenes)), cam, t))
        rid += 1
    return out


def latency_summary(results, skip_before_s=0.0):
    lat = np.array([r.latency for r in results if r.arrival >= skip_before_s]) * 1000.0
    if lat.size == 0:
        return {"requests": 0}
    kept = [r for r in results if r.arrival >= skip_before_s]
    span = max(r.done for r in kept) - min(r.arrival for r in kept)
    wait = np.array([r.launched - r.arrival for r in kept]) * 1000.0
    service = np.array([r.done - r.launched for r in kept]) * 1000.0
    return {"requests": int(lat.size), "p50_ms": float(np.percentile(lat, 50)), "p90_ms": float(np.percentile(lat, 90)),
            "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()), "max_ms": float(lat.max()),
            "queue_wait_p50_ms": float(np.percentile(wait, 50)), "queue_wait_p99_ms": float(np.percentile(wait, 99)),
            "batch_time_p50_ms": float(np.percentile(service, 50)), "batch_time_p99_ms": float(np.percentile(service, 99)),
            "frames_per_s": float(lat.size / span) if span > 0 else None,
            "mean_views_per_batch": float(len(kept) / len({r.batch for r in kept})),
            "mean_scenes_per_batch": float(len({(r.batch, r.scene) for r in kept}) / len({r.batch for r in kept}))}

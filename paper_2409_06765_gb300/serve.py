"""Render serving with continuous batching over resident scenes.

Several scenes' Gaussians stay resident on the device.  Forward-only render requests
(scene, camera) arrive over time; the server

* admits an arrived request into its scene's queue,
* forms a batch from whatever has arrived for one scene (up to ``max_views`` cameras of
  any mix of sizes) -- one multi-camera call renders them together (C > 1, per-camera
  tile lists, one launch per stage),
* launches the batch on a free CUDA stream of a small pool, so batches of different
  scenes overlap on the device, as long as the device memory the batch needs (its
  buffers, sized from the request sizes) fits in the free-HBM budget left by the batches
  in flight; otherwise the batch waits until enough in-flight work retires,
* retires a batch when its stream's event completes: the images (already copied to
  pinned host memory on the batch's stream) are handed back and the batch's memory is
  returned to the budget.

The unbatched single-view path is the same loop with one stream and one view per batch.
A camera's image does not depend on the batch it was rendered in (its tile lists hold
only its own Gaussians, in the same order), so batching changes latency, never pixels.

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
    image: np.ndarray  # [H, W, 3] float32 (host)
    arrival: float
    launched: float
    done: float
    batch_views: int

    @property
    def latency(self) -> float:
        return self.done - self.arrival


# --------------------------------------------------------------------------------------
# batching decision (pure)
# --------------------------------------------------------------------------------------

def plan_batch(queues: dict, max_views: int, budget_free: int, estimate):
    """Pick the next batch.

    queues: scene id -> list of queued requests (arrival order).  The scene whose oldest
    request has waited longest goes first; its batch takes queued requests in arrival order
    while the batch has fewer than ``max_views`` cameras and its estimated device bytes
    (``estimate(scene, requests)``) fit in ``budget_free``.  Returns (scene, requests) or
    None when nothing fits (the caller waits for in-flight work to retire).
    """
    order = sorted((q[0].arrival, sid) for sid, q in queues.items() if q)
    for _, sid in order:
        q = queues[sid]
        take = []
        for req in q[:max_views]:
            if estimate(sid, take + [req]) > budget_free:
                break
            take.append(req)
        if take:
            return sid, take
        # the oldest request of this scene does not fit: do not let younger ones overtake it
        return None
    return None


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
class _Batch:
    sid: int
    reqs: list
    pipe: FramePipeline
    stream: torch.cuda.Stream
    event: torch.cuda.Event
    host_img: torch.Tensor
    host_k: torch.Tensor
    nbytes: int
    capacity: int
    launched: float
    offsets: list = field(default_factory=list)


class Server:
    """Continuous-batching render server (forward only) over ResidentScenes."""

    def __init__(self, store: ResidentScenes, schedule: Schedule = Schedule(), max_views: int = 8, streams: int = 4,
                 budget_bytes: int | None = None, k_margin: float = 1.5):
        self.store = store
        self.schedule = schedule
        self.max_views = max(1, min(int(max_views), _lib.GS_MAX_CAMERAS))
        self.streams = [torch.cuda.Stream(store.device) for _ in range(max(1, streams))]
        free, _ = torch.cuda.mem_get_info(store.device)
        self.budget = budget_bytes if budget_bytes is not None else max(0, free - store.reserve)
        self.k_margin = k_margin
        self.overflows = 0
        self.batches = 0
        self.waits_for_memory = 0
        # pinned host buffers per stream (a stream carries one batch at a time): allocating
        # page-locked memory per batch costs milliseconds and stalls the loop
        self._pinned = {}

    # capacity of a batch's intersection buffers from the scene's intersections per pixel
    def _capacity(self, sid, reqs, hint=0):
        px = sum(r.camera.width * r.camera.height for r in reqs)
        est = int(px * self.store.k_rate[sid] * self.k_margin) + 65536
        return max(est, int(hint))

    def _estimate(self, sid, reqs):
        if not reqs:
            return 0
        cams = [r.camera for r in reqs]
        return batch_bytes(self.store.scenes[sid], cams, self.schedule, self._capacity(sid, reqs))

    def _launch(self, sid, reqs, stream, now, hint=0):
        scene = self.store.scenes[sid]
        cams = [r.camera for r in reqs]
        cap = self._capacity(sid, reqs, hint)
        nbytes = batch_bytes(scene, cams, self.schedule, cap)
        with torch.cuda.stream(stream):
            pipe = FramePipeline(scene, cams, self.schedule, backward=False, capacity=cap)
            pipe.forward()
            host_img, host_k = self._host_buffers(stream, pipe.image.shape)
            host_img.copy_(pipe.image, non_blocking=True)
            host_k.copy_(pipe.K_out, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(stream)
        self.batches += 1
        return _Batch(sid, reqs, pipe, stream, ev, host_img, host_k, nbytes, cap, now,
                      offsets=pipe.cams.pixel_offsets())

    def _host_buffers(self, stream, shape):
        """The stream's pinned image buffer (grown when a batch needs more) and count slot."""
        n = 1
        for d in shape:
            n *= int(d)
        img, k = self._pinned.get(stream.cuda_stream, (None, None))
        if img is None or img.numel() < n:  # grow geometrically: few page-locked allocations
            img = torch.empty(max(n, 2 * (img.numel() if img is not None else 0), 1 << 20), dtype=torch.float32,
                              pin_memory=True)
            k = k if k is not None else torch.empty(1, dtype=torch.int64, pin_memory=True)
            self._pinned[stream.cuda_stream] = (img, k)
        return img[:n].view(shape), k

    def serve(self, requests, realtime=True, poll_sleep=50e-6):
        """Serve a trace; returns the results in completion order.  With realtime=False every
        request counts as arrived at once (a saturation run: the queues start full)."""
        pending = deque(sorted(requests, key=lambda r: r.arrival))
        queues: dict[int, list] = {sid: [] for sid in self.store.scenes}
        free_streams = list(self.streams)
        inflight: list[_Batch] = []
        reserved = 0
        results = []
        retry: list = []  # (sid, reqs, capacity hint) of batches whose buffers overflowed
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
                K = int(b.host_k.item())
                px = sum(r.camera.width * r.camera.height for r in b.reqs)
                if K > 0:  # learn the scene's intersections per pixel from every batch
                    self.store.k_rate[b.sid] = max(self.store.k_rate[b.sid], K / px)
                if K < 0 or K > b.capacity:
                    self.overflows += 1
                    retry.append((b.sid, b.reqs, int(max(K, b.capacity) * 1.1) + 1024))
                else:
                    img = b.host_img.numpy()
                    for r, off in zip(b.reqs, b.offsets):
                        P = r.camera.width * r.camera.height
                        results.append(Result(r.rid, r.scene, img[off:off + P].reshape(r.camera.height,
                                                                                       r.camera.width, 3).copy(),
                                              r.arrival, b.launched, done, len(b.reqs)))
                del b
                progressed = True
            # launch: overflowed batches first, then new batches while streams and memory allow
            while free_streams and retry:
                sid, reqs, hint = retry.pop(0)
                st = free_streams.pop(0)
                b = self._launch(sid, reqs, st, now, hint)
                reserved += b.nbytes
                inflight.append(b)
                progressed = True
            while free_streams:
                plan = plan_batch(queues, self.max_views, self.budget - reserved, self._estimate)
                if plan is None:
                    if any(queues.values()):
                        self.waits_for_memory += 1 if inflight else 0
                        if not inflight:
                            raise MemoryError("a single request does not fit in the memory budget")
                    break
                sid, reqs = plan
                for r in reqs:
                    queues[sid].remove(r)
                st = free_streams.pop(0)
                b = self._launch(sid, reqs, st, now)
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
            "mean_views_per_batch": float(np.mean([r.batch_views for r in kept]))}

"""Launch-schedule autotuner for the frame pipeline.

The paper exposes the tile size and the per-tile batch as tunable block sizes; here they
are the tile edge t in {8, 16, 32}, the batch depth (Gaussians staged in shared memory per
round) in {64, 128, 256}, and the pixels each compositing thread owns.  The support rule is
per pixel, so every schedule renders bit-identical images: tuning changes speed only.

``tune`` builds a FramePipeline per candidate, replays it as CUDA graphs and keeps the
fastest mean step time.  Candidates that cannot run (intersection buffers beyond the int32
index range or device memory) are recorded as failed and skipped.  Results are cached per
workload signature (device, scene size, SH degree, camera sizes, forward-only or not).
"""
from __future__ import annotations

import gc
import json
import os
from dataclasses import dataclass, field

import torch

from .pipeline import DeviceScene, FramePipeline, Schedule

__all__ = ["TILE_SHAPES", "BATCH_DEPTHS", "candidates", "TuneResult", "tune", "signature"]

# (tile, pixels per thread) shapes the compositing kernels are compiled for
TILE_SHAPES = [(8, 1), (16, 1), (16, 2), (32, 2), (32, 4)]
BATCH_DEPTHS = [64, 128, 256]


def candidates(tile_order=True):
    return [Schedule(tile=t, batch_depth=b, pixels_per_thread=p, tile_order=tile_order)
            for (t, p) in TILE_SHAPES for b in BATCH_DEPTHS]


@dataclass
class TuneResult:
    best: Schedule
    best_ms: float
    table: list = field(default_factory=list)  # (schedule dict, ms or None, note)

    def as_dict(self):
        return {"best": self.best.as_dict(), "best_ms": self.best_ms,
                "table": [{"schedule": s, "ms": ms, "note": note} for s, ms, note in self.table]}


_CACHE: dict = {}


def signature(scene: DeviceScene, cams, backward: bool):
    name = torch.cuda.get_device_name(scene.means.device)
    sizes = tuple(cams.sizes) if hasattr(cams, "sizes") else tuple((c.width, c.height) for c in cams)
    return (name, scene.n, scene.sh_degree, sizes, bool(backward))


def _time_schedule(scene, cams, sched, backward, steps, warmup):
    pipe = FramePipeline(scene, cams, sched, backward=backward)
    try:
        if backward:
            pipe.forward()
            pipe.d_image.normal_()
        pipe.capture_graphs()
        for _ in range(warmup):
            pipe.step(graphs=True)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(steps):
            pipe.step(graphs=True)
        b.record()
        torch.cuda.synchronize()
        if pipe.frame_overflowed():
            return None, "intersection buffers overflowed while timing"
        return a.elapsed_time(b) / steps, ""
    finally:
        del pipe


def tune(scene: DeviceScene, cams, backward=True, schedules=None, steps=5, warmup=2, use_cache=True,
         cache_file=None, log=None) -> TuneResult:
    """Time every candidate schedule on this workload and return the fastest."""
    key = signature(scene, cams, backward)
    if use_cache and key in _CACHE:
        return _CACHE[key]
    schedules = schedules or candidates()
    table = []
    best, best_ms = None, float("inf")
    for sched in schedules:
        try:
            ms, note = _time_schedule(scene, cams, sched, backward, steps, warmup)
        except (RuntimeError, torch.OutOfMemoryError) as exc:  # GsError is a RuntimeError
            ms, note = None, f"failed: {str(exc).splitlines()[0][:120]}"
        gc.collect()
        torch.cuda.empty_cache()
        table.append((sched.as_dict(), ms, note))
        if log:
            log(f"  tile {sched.tile:2d} ppt {sched.pixels_per_thread} batch {sched.batch_depth:3d}: "
                + (f"{ms:.3f} ms" if ms is not None else note))
        if ms is not None and ms < best_ms:
            best, best_ms = sched, ms
    if best is None:
        raise RuntimeError("no schedule could run this workload")
    res = TuneResult(best, best_ms, table)
    _CACHE[key] = res
    if cache_file:
        entries = {}
        if os.path.exists(cache_file):
            with open(cache_file) as fh:
                entries = json.load(fh)
        entries[repr(key)] = res.as_dict()
        with open(cache_file, "w") as fh:
            json.dump(entries, fh, indent=1)
    return res

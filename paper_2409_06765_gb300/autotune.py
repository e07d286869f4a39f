"""Launch-schedule autotuner for the frame pipeline.

The paper exposes the tile size and the per-tile batch as tunable block sizes; here they
are the tile edge t in {8, 16, 32}, and for each compositing kernel separately the batch
depth (Gaussians staged in shared memory per round, 64..1024), the pixels each thread owns,
and the launch form (one CTA per tile, or one persistent launch of as many CTAs as fit that
take tiles heaviest first).  The support rule is per pixel, so every schedule renders
bit-identical images: tuning changes speed only.

For each tile size ``tune`` builds one FramePipeline (the tile size fixes the intersection
lists), times the stages before and after compositing as CUDA-graph replays, and times
every (pixels per thread, batch depth, launch form) of the forward and of the backward
compositing kernel on the same lists; the schedule of a tile size is its fastest forward plus its
fastest backward, and the fastest total over tile sizes wins.  Tile sizes that cannot run
(intersection lists beyond the int32 index range, device memory) are recorded as failed.
Results are cached per workload signature (device, scene size, SH degree, camera sizes,
forward-only or not).
"""
from __future__ import annotations

import gc
import json
import os
from dataclasses import dataclass, field

import torch

from . import _lib
from .pipeline import DeviceScene, FramePipeline, Schedule

__all__ = ["TILE_SHAPES", "BATCH_DEPTHS", "TuneResult", "tune", "signature"]

# pixels per thread the compositing kernels are compiled for, per tile size
TILE_SHAPES = {8: (1,), 16: (1, 2), 32: (2, 4)}
BATCH_DEPTHS = (64, 128, 256, 512, 1024)


@dataclass
class TuneResult:
    best: Schedule
    best_ms: float
    table: list = field(default_factory=list)  # dicts: tile, phase, ppt, batch, ms, note

    def as_dict(self):
        return {"best": self.best.as_dict(), "best_ms": self.best_ms, "table": self.table}


_CACHE: dict = {}


def signature(scene: DeviceScene, cams, backward: bool):
    name = torch.cuda.get_device_name(scene.means.device)
    sizes = tuple(cams.sizes) if hasattr(cams, "sizes") else tuple((c.width, c.height) for c in cams)
    return (name, scene.n, scene.sh_degree, sizes, bool(backward))


def _time(fn, reps, warmup=1):
    for _ in range(warmup):
        fn()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def _tune_tile(scene, cams, tile, backward, reps, table, log):
    pipe = FramePipeline(scene, cams, Schedule(tile=tile, batch_depth=128, pixels_per_thread=TILE_SHAPES[tile][0]),
                         backward=backward)
    try:
        pipe.forward()
        if backward:
            pipe.d_image.normal_(0.0, 1e-6)
        pipe.capture_graphs()
        ms_fixed = _time(pipe.g_pre.replay, reps)
        if backward:
            ms_fixed += _time(pipe.g_post.replay, reps)
        best = {}
        shapes = [(p, b, q) for p in TILE_SHAPES[tile] for b in BATCH_DEPTHS for q in (False, True)]
        for phase in (("fwd", "bwd") if backward else ("fwd",)):
            for ppt, batch, pers in shapes:
                params = _lib.make_params(tile=tile, batch_depth=batch, pixels_per_thread=ppt, persistent=pers)
                if phase == "fwd":
                    pipe.params = params
                    fn = pipe._raster_fwd
                else:
                    pipe.params_bwd = params

                    def fn():
                        pipe.g2d.zero_()
                        pipe._raster_bwd()
                try:
                    ms, note = _time(fn, reps), ""
                except RuntimeError as exc:
                    ms, note = None, f"failed: {str(exc).splitlines()[0][:100]}"
                table.append(dict(tile=tile, phase=phase, ppt=ppt, batch=batch, persistent=pers, ms=ms, note=note))
                if log:
                    log(f"  tile {tile:2d} {phase} ppt {ppt} batch {batch:4d}{' persistent' if pers else ''}: "
                        + (f"{ms:.3f} ms" if ms is not None else note))
                if ms is not None and (phase not in best or ms < best[phase][0]):
                    best[phase] = (ms, ppt, batch, pers)
        if pipe.frame_overflowed():
            raise RuntimeError("intersection buffers overflowed while tuning")
        total = ms_fixed + sum(v[0] for v in best.values())
        f = best["fwd"]
        b = best.get("bwd", f)
        sched = Schedule(tile=tile, batch_depth=f[2], pixels_per_thread=f[1], bwd_batch_depth=b[2],
                         bwd_pixels_per_thread=b[1], persistent=f[3], bwd_persistent=b[3])
        table.append(dict(tile=tile, phase="total", ms=total, fixed_ms=ms_fixed, schedule=sched.as_dict()))
        return sched, total
    finally:
        del pipe


def tune(scene: DeviceScene, cams, backward=True, tiles=(8, 16, 32), reps=5, use_cache=True, cache_file=None,
         log=None, tile_order=True) -> TuneResult:
    """Time every compiled schedule on this workload and return the fastest."""
    key = signature(scene, cams, backward)
    if use_cache and key in _CACHE:
        return _CACHE[key]
    table = []
    best, best_ms = None, float("inf")
    for tile in tiles:
        try:
            sched, ms = _tune_tile(scene, cams, tile, backward, reps, table, log)
        except (RuntimeError, torch.OutOfMemoryError) as exc:  # GsError is a RuntimeError
            table.append(dict(tile=tile, phase="total", ms=None, note=f"failed: {str(exc).splitlines()[0][:120]}"))
            if log:
                log(f"  tile {tile:2d}: {table[-1]['note']}")
            sched, ms = None, None
        gc.collect()
        torch.cuda.empty_cache()
        if ms is not None and ms < best_ms:
            best, best_ms = sched, ms
    if best is None:
        raise RuntimeError("no schedule could run this workload")
    if not tile_order:
        best = Schedule(**{**best.__dict__, "tile_order": False, "persistent": False, "bwd_persistent": False})
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

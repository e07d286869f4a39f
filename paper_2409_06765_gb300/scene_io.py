"""Scenes on disk: one directory of raw float32 ``.npy`` arrays per scene.

A serving process keeps several scenes resident (``serve.ResidentScenes``).  This module
stores a scene's parameters so that it can be loaded again without being regenerated:

    means.npy           [N, 3]            float32
    quats.npy           [N, 4] (w,x,y,z)  float32
    log_scales.npy      [N, 3]            float32
    opacity_logits.npy  [N]               float32
    sh.npy              [N, (d+1)^2, 3]   float32
    scene.json          {"format", "n", "sh_degree"}

Arrays are little-endian, C order, written with ``numpy.save`` (no pickling).  The
descriptor is written last, so a directory whose writing was interrupted has none and does
not load.  Loading checks every array's dtype and shape against the descriptor and raises
``ValueError`` on a mismatch; ``mmap=True`` maps the arrays read-only instead of reading
them, and the copy to the device (``DeviceScene.from_host``) then streams from the page
cache.  The returned ``synth.Scene`` goes straight to ``ResidentScenes.add``.
"""
from __future__ import annotations

import json
import os

import numpy as np

from .synth import Scene

__all__ = ["FORMAT", "save_scene", "load_scene"]

FORMAT = "gs-scene-npy-1"
_FIELDS = ("means", "quats", "log_scales", "opacity_logits", "sh")
_F32 = np.dtype("<f4")


def _shapes(n: int, sh_degree: int) -> dict:
    k = (sh_degree + 1) ** 2
    return {"means": (n, 3), "quats": (n, 4), "log_scales": (n, 3), "opacity_logits": (n,), "sh": (n, k, 3)}


def save_scene(scene: Scene, path: str) -> None:
    """Write ``scene`` into directory ``path`` (created if needed; existing files replaced)."""
    d = int(scene.sh_degree)
    if not 0 <= d <= 3:
        raise ValueError(f"SH degree must be in 0..3, got {d}")
    want = _shapes(scene.n, d)
    arrays = {}
    for f in _FIELDS:
        a = np.asarray(getattr(scene, f))
        if a.shape != want[f]:
            raise ValueError(f"{f} has shape {a.shape}, expected {want[f]}")
        arrays[f] = np.ascontiguousarray(a, dtype=_F32)
    os.makedirs(path, exist_ok=True)
    meta = os.path.join(path, "scene.json")
    if os.path.exists(meta):  # the arrays are about to change: the old descriptor no longer holds
        os.remove(meta)
    for f, a in arrays.items():
        np.save(os.path.join(path, f + ".npy"), a, allow_pickle=False)
    with open(meta, "w") as fh:
        json.dump({"format": FORMAT, "n": scene.n, "sh_degree": d}, fh)


def load_scene(path: str, mmap: bool = False, check_finite: bool = True) -> Scene:
    """Read the scene stored in directory ``path`` by ``save_scene``.

    ``check_finite`` rejects NaN or infinite parameters (it reads every value, so with
    ``mmap=True`` it touches the whole file once)."""
    with open(os.path.join(path, "scene.json")) as fh:
        meta = json.load(fh)
    if meta.get("format") != FORMAT:
        raise ValueError(f"{path}: unknown scene format {meta.get('format')!r}")
    n, d = int(meta["n"]), int(meta["sh_degree"])
    if n < 0 or not 0 <= d <= 3:
        raise ValueError(f"{path}: invalid descriptor n={n}, sh_degree={d}")
    want = _shapes(n, d)
    arrays = {}
    for f in _FIELDS:
        a = np.load(os.path.join(path, f + ".npy"), mmap_mode="r" if mmap else None, allow_pickle=False)
        if a.dtype != _F32:
            raise ValueError(f"{path}: {f} is {a.dtype}, expected float32")
        if a.shape != want[f]:
            raise ValueError(f"{path}: {f} has shape {a.shape}, expected {want[f]}")
        if check_finite and not np.isfinite(a).all():
            raise ValueError(f"{path}: {f} holds non-finite values")
        arrays[f] = a
    return Scene(arrays["means"], arrays["quats"], arrays["log_scales"], arrays["opacity_logits"], arrays["sh"], d)

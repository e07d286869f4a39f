"""Scenes saved as raw float32 .npy arrays load back bit for bit; damaged or mismatched
files are rejected with a clear error.  No GPU needed."""
import json
import os

import numpy as np
import pytest

from paper_2409_06765_gb300 import scene_io, synth

FIELDS = ("means", "quats", "log_scales", "opacity_logits", "sh")


def _same(a, b):
    assert a.sh_degree == b.sh_degree and a.n == b.n
    for f in FIELDS:
        x, y = getattr(a, f), getattr(b, f)
        assert x.dtype == y.dtype == np.float32 and x.shape == y.shape
        np.testing.assert_array_equal(x, y)


@pytest.mark.parametrize("deg", [0, 1, 3])
@pytest.mark.parametrize("mmap", [False, True])
def test_round_trip_is_bit_exact(tmp_path, deg, mmap):
    sc = synth.clustered_scene(3000, seed=deg, sh_degree=deg)
    scene_io.save_scene(sc, str(tmp_path / "s"))
    back = scene_io.load_scene(str(tmp_path / "s"), mmap=mmap)
    _same(sc, back)
    if mmap:
        assert isinstance(back.sh, np.memmap)


def test_empty_scene_round_trip(tmp_path):
    sc = synth.clustered_scene(0, seed=1, sh_degree=2)
    scene_io.save_scene(sc, str(tmp_path))
    _same(sc, scene_io.load_scene(str(tmp_path)))


def test_overwrite_replaces_the_scene(tmp_path):
    scene_io.save_scene(synth.clustered_scene(500, seed=1, sh_degree=3), str(tmp_path))
    sc = synth.clustered_scene(200, seed=2, sh_degree=0)
    scene_io.save_scene(sc, str(tmp_path))
    _same(sc, scene_io.load_scene(str(tmp_path)))


def test_interrupted_write_does_not_load(tmp_path):
    sc = synth.clustered_scene(100, seed=3, sh_degree=1)
    scene_io.save_scene(sc, str(tmp_path))
    os.remove(tmp_path / "scene.json")  # the descriptor is written last
    with pytest.raises(FileNotFoundError):
        scene_io.load_scene(str(tmp_path))


def test_mismatched_arrays_are_rejected(tmp_path):
    sc = synth.clustered_scene(100, seed=4, sh_degree=3)
    path = str(tmp_path)
    scene_io.save_scene(sc, path)
    np.save(os.path.join(path, "sh.npy"), sc.sh[:, :4].copy())  # degree-1 coefficients
    with pytest.raises(ValueError, match="sh has shape"):
        scene_io.load_scene(path)
    scene_io.save_scene(sc, path)
    np.save(os.path.join(path, "means.npy"), sc.means.astype(np.float64))
    with pytest.raises(ValueError, match="float32"):
        scene_io.load_scene(path)
    scene_io.save_scene(sc, path)
    bad = sc.opacity_logits.copy()
    bad[7] = np.nan
    np.save(os.path.join(path, "opacity_logits.npy"), bad)
    with pytest.raises(ValueError, match="non-finite"):
        scene_io.load_scene(path)
    assert scene_io.load_scene(path, check_finite=False).n == 100
    with open(os.path.join(path, "scene.json"), "w") as fh:
        json.dump({"format": "something-else", "n": 100, "sh_degree": 3}, fh)
    with pytest.raises(ValueError, match="format"):
        scene_io.load_scene(path)


def test_save_checks_the_scene(tmp_path):
    sc = synth.clustered_scene(10, seed=5, sh_degree=3)
    sc.sh = sc.sh[:, :9]  # degree-2 coefficients under a degree-3 label
    with pytest.raises(ValueError, match="sh has shape"):
        scene_io.save_scene(sc, str(tmp_path))
    assert not (tmp_path / "scene.json").exists()

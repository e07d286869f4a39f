"""The product path has no CPU fallback and never routes through the oracle.

The package computes only in libgs.so.  No module of it imports the FP64 oracle, loading
fails loudly when the library file is absent, and CPU tensors are rejected at the binding
instead of being rendered some other way.  No GPU needed.
"""
import ast
import os

import numpy as np
import pytest
import torch

from paper_2409_06765_gb300 import _build, _lib, raster, synth

PKG = os.path.dirname(os.path.abspath(_lib.__file__))


def _imported_modules(path):
    tree = ast.parse(open(path).read(), path)
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            yield from (a.name for a in node.names)
        elif isinstance(node, ast.ImportFrom) and node.module and node.level == 0:
            yield node.module


def test_no_package_module_imports_the_oracle():
    files = [os.path.join(d, f) for d, _, fs in os.walk(PKG) for f in fs if f.endswith(".py")]
    assert len(files) >= 8
    for path in files:
        bad = [m for m in _imported_modules(path) if m == "oracle" or m.startswith("oracle.")]
        assert not bad, f"{path} imports {bad}"
        assert "gs_oracle" not in open(path).read(), path


def test_missing_library_raises(monkeypatch, tmp_path):
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_build, "LIB", str(tmp_path / "libgs.so"))
    with pytest.raises(RuntimeError, match="libgs.so not found"):
        _lib.load(build_if_missing=False)


def test_cpu_tensors_are_rejected_not_rendered():
    sc, cam, _ = synth.tiny_scene()
    ca = _lib.CameraArray([cam])
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a, np.float32))
    with pytest.raises(ValueError, match="CUDA tensor"):
        raster.project(ca, t(sc.means), t(sc.quats), t(sc.log_scales), t(sc.opacity_logits), _lib.make_params())

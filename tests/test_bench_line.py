"""The benchmark's result line stays short enough for a consumer that keeps only the tail of
stdout, whatever the size of the full record (autotuner candidates, serving detail); no GPU."""
import io
import json
import os
import sys
from contextlib import redirect_stderr, redirect_stdout

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402

LINE_LIMIT = 1400  # bytes: the consumer keeps the last 1500 characters of stdout


def _full_record():
    cand = [{"tile": t, "phase": ph, "ppt": p, "batch": b, "persistent": pe, "ms": 1.2345678912345, "note": ""}
            for t in (8, 16, 32) for ph in ("fwd", "bwd") for p in (1, 2, 4) for b in (64, 128, 256, 512, 1024)
            for pe in (False, True)]
    stage = {"bound": "hbm", "bytes": 123456789, "bound_ms": 0.0123456789, "ms": 0.0456789, "frac": 0.27027027}
    serve_row = {"requests": 11981, "p50_ms": 2.965989267005753, "p90_ms": 8.914460455995865,
                 "p99_ms": 18.73840368200188, "mean_ms": 4.163428936550632, "max_ms": 27.073458233054293,
                 "frames_per_s": 197.91587791987695, "mean_views_per_batch": 1.0413932357395255,
                 "saturated_frames_per_s": 379.0436983697336, "saturated_mean_views_per_batch": 3.2,
                 "saturated_640x480_frames_per_s": 1612.345678, "saturated_640x480_mean_views_per_batch": 5.9123,
                 "streams": 4, "batches": 2407, "overflow_retries": 2}
    return {
        "metric": bench.METRIC, "value": 2.5e11, "unit": bench.UNIT, "n_gpus": 1, "steps": 20, "warmup": 5,
        "ms_per_step": 2.0912345, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic (seeded clustered Gaussians; no dataset)",
        "config": {"workload": "headline", "description": "x" * 120, "gaussians": 3000000, "sh_degree": 3,
                   "resolution": [1920, 1080], "views_per_gpu": 1, "tile": 32, "batch_depth": 512,
                   "pixels_per_thread": 4, "bwd_batch_depth": 1024, "bwd_pixels_per_thread": 4,
                   "persistent_launch": [False, False], "schedule_from": "autotuner", "cuda_graphs": True,
                   "tile_order": True, "intersections_K": 16912345, "blends_per_view": 522123456,
                   "l2": "inputs (708 MB of parameters) exceed L2; no flush", "parallelism": "replicas x1"},
        "ms_per_view_fwd_bwd": 2.0912345, "ms_per_view_fwd": 0.9123456, "blends_per_s_fwd": 5.72e11,
        "gpu_launches": 640, "gpu_launches_per_step": 32.0,
        "autotune": {"best": {"tile": 32}, "candidates": cand},
        "roofline": {"bound": "alu", "kernel": "rasterize_bwd", "achieved": 29876.54321, "peak": 40273.92,
                     "unit": "Gop/s", "frac": 0.741852, "traffic": 1234567890, "peak_source": "y" * 60,
                     "ops_per_blend": 45, "fwd": {"ms": 0.333, "gop_s": 31234.5, "frac": 0.7755},
                     "bwd": {"ms": 0.797, "gop_s": 29876.5, "frac": 0.7418}, "frac_at_sampled_clock": 0.7418,
                     "probe": {"ffma_gop_s": 39200.0, "ex2_gop_s": 10000.0, "frac_of_ffma_probe": 0.76}},
        "step_roofline": {"bound_ms": 1.43, "stages_ms": 2.09, "frac": 0.68,
                          "stages": {k: dict(stage) for k in ("project", "sh", "bin_sort", "rasterize_fwd",
                                                                        "rasterize_bwd", "sh_bwd", "project_bwd")}, "note": "z" * 150},
        "peaks": {"source": "measured", "hbm_gbs": 6764.0},
        "clocks": {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 12, "scope": "timed region",
                   "power_w_max": 640.0},
        "e2e": {"value": 2.16e11, "unit": bench.UNIT, "ms_per_step": 2.42, "h2d_bytes_per_step": 24883200,
                "d2h_bytes_per_step": 4, "api": "w" * 100, "redone_steps": 0},
        "cpu_baseline": {"value": 562629.84, "unit": bench.UNIT, "cores": 16, "kind": "oracle",
                         "ms_per_view_extrapolated": 967929.46, "sample": "s" * 230, "sample_blends": 123456},
        "serving_p99_ms": 18.7,
        "multiview": {"workload": "m" * 100, "ms_per_batch": 29.3, "views_per_s": 546.0, "blends_per_s": 3.1e11,
                      "speedup_vs_single_view": 1.32, "intersections_K": 123456789,
                      "schedule": {"tile": 32, "batch_depth": 512, "pixels_per_thread": 4, "bwd_batch_depth": 1024,
                                   "bwd_pixels_per_thread": 4},
                      "autotune": {"candidates": cand}},
        "memory": {"workload": "q" * 90, "ms_per_step": 9.6, "peak_allocated_bytes": 8.4e9,
                   "per_blend_state_would_need_bytes": 15.7e9},
        "serving": {"workload": "v" * 200, "seconds": 60.0, "rate": 200.0, "batched": dict(serve_row),
                    "single_view": dict(serve_row), "p99_ms": 18.7},
    }


def test_result_line_is_short_and_carries_the_contract_fields():
    full = _full_record()
    out, err = io.StringIO(), io.StringIO()
    with redirect_stdout(out), redirect_stderr(err):
        bench.emit(full)
    lines = out.getvalue().splitlines()
    assert len(lines) == 1
    assert len(lines[0].encode()) <= LINE_LIMIT, len(lines[0])
    line = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "gpu_launches", "roofline", "cpu_baseline",
                "e2e", "clocks"):
        assert key in line, key
    assert line["value"] == full["value"] and line["config"]["workload"] == "headline"
    for key in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert key in line["roofline"]
    assert set(line["e2e"]) >= {"value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"}
    assert set(line["cpu_baseline"]) >= {"value", "unit", "cores", "kind", "sample"}
    assert line["serving"]["batch"][1] > 0 and "multiview" in line and "memory" in line
    # the whole record is still there, on stderr
    detail = [ln for ln in err.getvalue().splitlines() if ln.startswith("detail ")]
    assert json.loads(detail[0][len("detail "):]) == json.loads(json.dumps(full))


def test_failed_rows_are_reported_in_the_line():
    full = _full_record()
    full["serving"] = {"error": "RuntimeError: out of memory"}
    full["multiview"] = {"error": "RuntimeError: x"}
    line = bench.summary_line(full)
    assert line["serving"] == {"error": "RuntimeError: out of memory"}
    assert line["multiview"] == {"error": "RuntimeError: x"}
    assert len(json.dumps(line, separators=(",", ":"))) <= LINE_LIMIT

"""The benchmark's reference arm (the FP64 oracle on the host cores) prints one JSON line
with the fields a consumer of ``bench.py`` reads, on a small workload; no GPU needed."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench(*args, env=None):
    return subprocess.run([sys.executable, "bench.py", *args], cwd=ROOT, capture_output=True, text=True, timeout=600,
                          env=dict(os.environ, **(env or {})))


def test_reference_line_has_the_contract_fields():
    r = _bench("--impl", "reference", "--workload", "tiny", "--steps", "2", "--warmup", "3", "--ref-budget", "5")
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference"
    for key in ("metric", "unit", "data", "dtype", "scaling"):
        assert isinstance(line[key], str) and line[key]
    assert line["value"] > 0 and line["ms_per_step"] > 0
    assert (line["n_gpus"], line["steps"], line["warmup"]) == (1, 2, 3)
    assert line["higher_is_better"] is True and line["vs_baseline"] is None
    assert line["config"]["workload"] == "tiny"
    cpu = line["cpu_baseline"]
    assert cpu["kind"] == "oracle" and cpu["cores"] >= 1 and cpu["value"] == line["value"]
    assert cpu["unit"] == line["unit"] and "extrapolated" in cpu["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["gpu_launches"] == 0


def test_reference_arm_runs_on_rank_0_only():
    r = _bench("--impl", "reference", "--workload", "tiny", "--steps", "1", "--warmup", "3", "--ref-budget", "2",
               env={"RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert not [ln for ln in r.stdout.splitlines() if ln.startswith("{")]


def test_fewer_than_three_warmup_steps_are_refused():
    r = _bench("--impl", "reference", "--workload", "tiny", "--steps", "1", "--warmup", "2")
    assert r.returncode != 0 and "--warmup" in (r.stderr + r.stdout)


def test_multiview_workload_is_the_sixteen_view_batch_and_not_a_reference_workload():
    """``--workload multiview`` times the 16-view batch (four views of each of the four sizes) as its
    step; the reference arm, whose oracle sample is one view, refuses it."""
    import bench
    scene, cams, desc = bench.build_workload("multiview", 0)
    sizes = [(c.width, c.height) for c in cams]
    assert sizes == bench.MULTIVIEW_SIZES and len(sizes) == 16
    assert sorted(set(sizes)) == [(640, 480), (1280, 720), (1920, 1080), (2560, 1440)]
    assert all(sizes.count(s) == 4 for s in set(sizes))
    assert scene.n == 3_000_000 and scene.sh_degree == 3
    r = _bench("--impl", "reference", "--workload", "multiview", "--steps", "1", "--warmup", "3")
    assert r.returncode != 0 and "one view" in (r.stderr + r.stdout)

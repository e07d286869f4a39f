"""Benchmark of the differentiable tile-based Gaussian rasterizer on one GB300.

Workload (default): 3,000,000 clustered Gaussians with SH degree 3 (the scene
distributions of the 1M-Gaussian training-step configuration, scaled to 3M) seen
by one 1920x1080 camera on the radius-6 sphere; a step is one forward + backward
pass of the whole rasterizer (project, SH, bin + sort, composite, composite
backward, SH backward, projection backward) through the C ABI with all inputs
resident in HBM.  The upstream image gradient is the L1-loss gradient of the first
rendered frame, held fixed.  Inputs (708 MB of Gaussian parameters) exceed the
129 MB L2, so no explicit flush is needed between steps.

Metric: Gaussian-pixel blends per second for forward + backward, where the blend
count B is the number of (pixel, Gaussian) pairs whose alpha the forward evaluates
(the pixel lies in the Gaussian's 3-sigma box and has not terminated), counted by
the instrumented forward once before timing; ms per view is reported beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
    python -m torch.distributed.run --nproc-per-node N bench.py --gpus N ...

With N > 1 every rank renders its own camera of the same scene (replicas, weak
scaling, no collective on the data path).  ``--impl reference`` times the FP64 CPU
oracle on a bounded pixel sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "fwd+bwd ms/view and Gaussian-pixel blends/s, 3M Gaussians @1080p; serving p99 ms"
UNIT = "blends/s"

# Algorithmic work per evaluated blend (FP32 lane operations), read off the arithmetic of
# App. C.2 / App. D.1 as implemented (an FMA counts as one operation, MUFU ops separate):
#   forward : box test 4, delta 2, sigma 6, exp scale 1, alpha 2 (mul, min), skip test 1,
#             T(1-alpha) 2, stop test 1, weight 1, colour 3 FMA, bookkeeping 2     -> 25 ops + 1 MUFU
#   backward: forward part up to alpha 16, 1/(1-alpha) 1 MUFU + 1, T 1, weight 1, gc 3,
#             dcol 3, dalpha 3, S update 1, clamp 1, dop 1, dsigma 2, dmean 6, dconic 7 -> 47 ops + 2 MUFU
FWD_OPS_PER_BLEND = 25
BWD_OPS_PER_BLEND = 47


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            return json.load(fh), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while the timed region runs."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.file = None

    def __enter__(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.file,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.proc is None or self.file is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.file.flush()
        rows = []
        with open(self.file.name) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.file.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "power_w_max": max((num(r[3]) or 0) for r in rows)}


def build_workload(name: str, rank: int):
    from paper_2409_06765_gb300 import synth
    if name == "headline":
        scene = synth.clustered_scene(3_000_000, 3)
        cams = synth.sphere_cameras(1003 + 7919 * rank, [(1920, 1080)])
        desc = "3M clustered Gaussians, SH degree 3, one 1920x1080 view (f=0.848W) on the radius-6 sphere"
    elif name == "training_step":
        scene, cam, _ = synth.training_step_workload()
        if rank:
            cam = synth.sphere_cameras(2000 + rank, [(1297, 840)])[0]
        cams = [cam]
        desc = "1M clustered Gaussians, SH degree 3, one 1297x840 view, f=1100"
    elif name == "tiny":
        scene, cam, _ = synth.tiny_scene()
        cams = [cam]
        desc = "1,000 Gaussians, SH degree 0, one 64x64 view"
    else:
        raise SystemExit(f"unknown workload {name}")
    return scene, cams, desc


class KernelPath:
    """Preallocated buffers and one fwd+bwd step issued through the C ABI (no host sync)."""

    def __init__(self, scene, cams, tile=16, batch=256, ppt=0):
        import torch
        from paper_2409_06765_gb300 import _lib
        self.torch, self.L = torch, _lib
        dev = "cuda"
        t = lambda a: torch.as_tensor(np.ascontiguousarray(a, np.float32), device=dev)
        self.means, self.quats, self.log_scales = t(scene.means), t(scene.quats), t(scene.log_scales)
        self.logits, self.sh, self.deg = t(scene.opacity_logits), t(scene.sh), scene.sh_degree
        self.cams = _lib.CameraArray(cams)
        self.params = _lib.make_params(tile=tile, batch_depth=batch, pixels_per_thread=ppt)
        C, N = self.cams.C, scene.n
        self.C, self.N = C, N
        f = lambda *s: torch.empty(*s, device=dev)
        i = lambda *s: torch.empty(*s, dtype=torch.int32, device=dev)
        self.means2d, self.depths, self.conics = f(C, N, 2), f(C, N), f(C, N, 3)
        self.radii, self.tiles, self.opac, self.colors = i(C, N), i(C, N), f(C, N), f(C, N, 3)
        P = self.cams.num_pixels
        self.P = P
        self.image, self.final_T, self.last = f(P, 3), f(P), i(P)
        self.ranges = i(self.cams.num_tiles(tile), 2)
        self.K_out = torch.zeros(1, dtype=torch.int64, device=dev)
        # 2D gradient buffers in one allocation so that one memset clears them
        self.g2d = torch.zeros(C * N * 9, device=dev)
        o = 0
        self.d_means2d = self.g2d[o:o + C * N * 2].view(C, N, 2); o += C * N * 2
        self.d_conics = self.g2d[o:o + C * N * 3].view(C, N, 3); o += C * N * 3
        self.d_opac = self.g2d[o:o + C * N].view(C, N); o += C * N
        self.d_colors = self.g2d[o:o + C * N * 3].view(C, N, 3)
        self.d_sh, self.d_means = torch.empty_like(self.sh), f(N, 3)
        self.d_quats, self.d_log_scales, self.d_logits = f(N, 4), f(N, 3), f(N)
        self.d_image = torch.zeros(P, 3, device=dev)
        # size the intersection buffers from one real frame (K is data dependent)
        self.capacity = 1 << 20
        self._alloc_sort()
        self.forward()
        torch.cuda.synchronize()
        K = int(self.K_out.item())
        if K > self.capacity:
            self.capacity = int(K * 1.1) + 1024
            self._alloc_sort()
            self.forward()
            torch.cuda.synchronize()
        self.K = int(self.K_out.item())
        if not 0 <= self.K <= self.capacity:
            raise RuntimeError(f"bin/sort returned K = {self.K} for capacity {self.capacity}")

    def _alloc_sort(self):
        torch = self.torch
        self.values = torch.empty(self.capacity, dtype=torch.int32, device="cuda")
        nbytes = self.L.gs_tile_bin_sort_workspace(self.cams, self.N, self.params, self.capacity)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device="cuda")

    def set_loss_gradient(self, target):
        """Upstream gradient of the mean L1 loss at the current image (held fixed while timing)."""
        torch = self.torch
        self.d_image.copy_(torch.sign(self.image - target) / self.image.numel())

    # The step in four parts: the two compositing kernels are launched directly (bracketed by
    # CUDA events for the roofline); the stages before and after them, some twenty short
    # launches, can be replayed as CUDA graphs (capture_graphs) to cut launch gaps.
    def _pre(self):
        L = self.L
        L.gs_project(self.cams, self.means, self.quats, self.log_scales, self.logits, self.params, self.means2d,
                     self.depths, self.conics, self.radii, self.tiles, self.opac)
        L.gs_sh_eval(self.cams, self.deg, self.sh, self.means, self.radii, self.colors)
        L.gs_tile_bin_sort(self.cams, self.N, self.params, self.means2d, self.depths, self.radii, self.capacity,
                           None, self.values, self.ranges, self.K_out, self.workspace)

    def _raster_fwd(self, count=None):
        self.L.gs_rasterize_fwd(self.cams, self.N, self.params, 3, self.ranges, self.values, self.radii,
                                self.means2d, self.conics, self.opac, self.colors, None, self.image, self.final_T,
                                self.last, count)

    def _raster_bwd(self):
        self.L.gs_rasterize_bwd(self.cams, self.N, self.params, 3, self.ranges, self.values, self.radii,
                                self.means2d, self.conics, self.opac, self.colors, None, self.final_T, self.last,
                                self.d_image, None, self.d_means2d, self.d_conics, self.d_opac, self.d_colors, None)

    def _post(self):
        L = self.L
        L.gs_sh_eval_bwd(self.cams, self.deg, self.sh, self.means, self.radii, self.d_colors, self.d_sh, self.d_means)
        L.gs_project_bwd(self.cams, self.means, self.quats, self.log_scales, self.logits, self.params, self.radii,
                         self.d_means2d, self.d_conics, self.d_opac, None, self.d_means, self.d_quats,
                         self.d_log_scales, self.d_logits)

    def capture_graphs(self):
        """Capture the stages around the compositing kernels as CUDA graphs (no host sync inside)."""
        torch = self.torch
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):  # warm the capture stream once
            self.g2d.zero_()
            self._pre()
            self._post()
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        n0 = self.L.gs_kernel_launches()
        self.g_pre, self.g_post = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.g_pre):
            self.g2d.zero_()  # the 2D gradients the compositing backward accumulates into
            self._pre()
        with torch.cuda.graph(self.g_post):
            self._post()
        torch.cuda.synchronize()
        self.graph_kernels = self.L.gs_kernel_launches() - n0  # kernel nodes of both graphs

    def forward(self, events=None, count=None, graphs=False):
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
        if not graphs:
            self.g2d.zero_()
        if events:
            events[0].record()
        self._raster_bwd()
        if events:
            events[1].record()
        if graphs:
            self.g_post.replay()
        else:
            self._post()

    def count_blends(self):
        torch = self.torch
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        self.forward(count=cnt)
        torch.cuda.synchronize()
        return int(cnt.item())


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2409_06765_gb300 import _lib, raster

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    scene, cams, desc = build_workload(args.workload, rank)
    kp = KernelPath(scene, cams, tile=args.tile, batch=args.batch, ppt=args.ppt)
    rng = np.random.default_rng(5 + rank)
    target_np = rng.uniform(0.0, 1.0, (kp.P, 3)).astype(np.float32)
    target = torch.as_tensor(target_np, device="cuda")
    kp.set_loss_gradient(target)
    blends = kp.count_blends()

    def barrier():
        if world > 1:
            dist.barrier()

    # kernels launched by one step (counted eagerly; graph replays launch the same kernels)
    n0 = _lib.gs_kernel_launches()
    kp.forward()
    kp.backward()
    torch.cuda.synchronize()
    launches_per_step = _lib.gs_kernel_launches() - n0
    graphs = not args.no_graph
    if graphs:
        kp.capture_graphs()
    # warm-up
    for _ in range(args.warmup):
        kp.forward(graphs=graphs)
        kp.backward(graphs=graphs)
    torch.cuda.synchronize()

    ev = lambda: torch.cuda.Event(enable_timing=True)
    fwd_ev = [(ev(), ev()) for _ in range(args.steps)]
    bwd_ev = [(ev(), ev()) for _ in range(args.steps)]
    start, stop = ev(), ev()
    with ClockSampler(local) as clocks:
        barrier()
        torch.cuda.synchronize()
        start.record()
        for k in range(args.steps):
            kp.forward(events=fwd_ev[k], graphs=graphs)
            kp.backward(events=bwd_ev[k], graphs=graphs)
        stop.record()
        torch.cuda.synchronize()
        barrier()
    launches = launches_per_step * args.steps
    ms_total = start.elapsed_time(stop)
    ms_step = ms_total / args.steps
    t_fwd_raster = float(np.mean([a.elapsed_time(b) for a, b in fwd_ev]))
    t_bwd_raster = float(np.mean([a.elapsed_time(b) for a, b in bwd_ev]))
    if world > 1:
        t = torch.tensor([ms_step, float(blends)], device="cuda", dtype=torch.float64)
        mx = t.clone()
        dist.all_reduce(mx, op=dist.ReduceOp.MAX)
        sm = t.clone()
        dist.all_reduce(sm, op=dist.ReduceOp.SUM)
        ms_step_job, blends_job = float(mx[0]), float(sm[1])
    else:
        ms_step_job, blends_job = ms_step, float(blends)
    value = blends_job / (ms_step_job / 1000.0)

    # forward-only timing (separate loop, same buffers)
    torch.cuda.synchronize()
    s2, e2 = ev(), ev()
    s2.record()
    for _ in range(args.steps):
        kp.forward(graphs=graphs)
    e2.record()
    torch.cuda.synchronize()
    ms_fwd = s2.elapsed_time(e2) / args.steps

    # end to end through the public API: target image H2D from pinned memory every step,
    # loss D2H every step, Gaussians resident (they are the trainable parameters)
    e2e = None
    if not args.no_e2e:
        leaves = [x.detach().clone().requires_grad_(True) for x in (kp.means, kp.quats, kp.log_scales, kp.logits,
                                                                     kp.sh)]
        settings = raster.RasterSettings(tile=args.tile, batch_depth=args.batch, pixels_per_thread=args.ppt)
        state = raster.RasterState()
        host_target = torch.as_tensor(target_np).pin_memory()
        dev_target = torch.empty_like(target)
        cam_arr = _lib.CameraArray(cams)

        def e2e_step():
            dev_target.copy_(host_target, non_blocking=True)
            imgs, alphas, _ = raster.rasterization(*leaves, cameras=cam_arr, settings=settings, state=state)
            loss = (imgs[0].reshape(-1, 3) - dev_target).abs().mean()
            loss.backward()
            return float(loss.item())

        for _ in range(max(2, args.warmup)):
            e2e_step()
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        torch.cuda.synchronize()
        barrier()
        e2e_ms = (time.perf_counter() - t0) * 1000.0 / args.steps
        if world > 1:
            t = torch.tensor([e2e_ms], device="cuda", dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_ms = float(t[0])
        e2e = {"value": blends_job / (e2e_ms / 1000.0), "unit": UNIT, "ms_per_step": e2e_ms,
               "h2d_bytes_per_step": int(host_target.numel() * 4), "d2h_bytes_per_step": 4,
               "api": "paper_2409_06765_gb300.raster.rasterization + L1 loss backward"}

    peaks, peak_kind = _peaks()
    clk = clocks.summary()
    sm_count = torch.cuda.get_device_properties(0).multi_processor_count
    f_max = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    alu_peak = sm_count * 128 * f_max  # FP32 lane operations / s at the maximum SM clock
    bwd_ach = blends * BWD_OPS_PER_BLEND / (t_bwd_raster / 1000.0)
    fwd_ach = blends * FWD_OPS_PER_BLEND / (t_fwd_raster / 1000.0)
    dominant = "rasterize_bwd" if t_bwd_raster >= t_fwd_raster else "rasterize_fwd"
    ach = bwd_ach if dominant == "rasterize_bwd" else fwd_ach
    traffic = None
    prof = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(prof):
        with open(prof) as fh:
            tr = json.load(fh)
        if tr.get("workload") == args.workload and dominant in tr.get("kernels", {}):
            traffic = tr["kernels"][dominant]
    roofline = {"bound": "alu", "kernel": dominant, "achieved": ach / 1e9, "peak": alu_peak / 1e9,
                "unit": "Gop/s", "frac": ach / alu_peak, "traffic": traffic,
                "peak_source": f"{sm_count} SMs x 128 FP32 lanes x {f_max / 1e6:.0f} MHz (max SM clock)",
                "work": f"{BWD_OPS_PER_BLEND if dominant == 'rasterize_bwd' else FWD_OPS_PER_BLEND} FP32 ops per blend",
                "fwd": {"ms": t_fwd_raster, "gop_s": fwd_ach / 1e9, "frac": fwd_ach / alu_peak},
                "bwd": {"ms": t_bwd_raster, "gop_s": bwd_ach / 1e9, "frac": bwd_ach / alu_peak}}
    if clk.get("sm_mhz"):
        roofline["frac_at_sampled_clock"] = ach / (sm_count * 128 * clk["sm_mhz"] * 1e6)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(scene, cams[0], target_np, args.cpu_pixels, kp_blends=blends)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_step_job, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic (seeded clustered Gaussians; no dataset)",
        "config": {"workload": args.workload, "description": desc, "gaussians": scene.n, "sh_degree": scene.sh_degree,
                   "resolution": [cams[0].width, cams[0].height], "views_per_gpu": len(cams), "tile": args.tile,
                   "batch_depth": args.batch, "pixels_per_thread": args.ppt,
                   "cuda_graphs": graphs, "intersections_K": kp.K, "blends_per_view": blends,
                   "l2": "inputs (708 MB of parameters) exceed L2; no flush", "parallelism": f"replicas x{world}"},
        "ms_per_view_fwd_bwd": ms_step_job, "ms_per_view_fwd": ms_fwd,
        "blends_per_s_fwd": blends / (ms_fwd / 1000.0),
        "gpu_launches": int(launches), "gpu_launches_per_step": launches / args.steps,
        "roofline": roofline, "peaks": {"source": peak_kind, "hbm_gbs": peaks.get("hbm_gbs")},
        "clocks": clk, "e2e": e2e, "cpu_baseline": cpu,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def oracle_setup(scene, cam):
    """Full-view FP64 projection and colours, needed as input by the per-pixel oracle stages."""
    import oracle
    sp = oracle.project(scene, cam)
    colors, _ = oracle.sh_colors(scene, cam)
    return sp, colors


def cpu_baseline(scene, cam, target_np, pixels, gauss_sample=100_000, setup=None, kp_blends=None, seed=99):
    """The FP64 oracle, as it stands, on a bounded sample of one view, extrapolated to the view.

    Per-Gaussian stages (projection, SH, their backward) run on a seeded subset of
    ``gauss_sample`` Gaussians and scale linearly in N.  Per-pixel stages (brute-force
    compositing over all depth-sorted Gaussians, forward and backward) run on a seeded
    pixel sample; the one-off cost of a call (its depth sort) is timed with a one-pixel
    call and the rest scales linearly in pixels.
    """
    import oracle
    from paper_2409_06765_gb300 import synth
    P = cam.width * cam.height
    N = scene.n
    rng = np.random.default_rng(seed)
    G = min(gauss_sample, N)
    idx = np.sort(rng.choice(N, G, replace=False))
    sub = synth.Scene(scene.means[idx], scene.quats[idx], scene.log_scales[idx], scene.opacity_logits[idx],
                      scene.sh[idx], scene.sh_degree)
    t0 = time.perf_counter()
    oracle.project(sub, cam)
    oracle.sh_colors(sub, cam)
    oracle.sh_bwd(sub, cam, np.full((G, 3), 1e-3))
    oracle.project_bwd(sub, cam, np.full((G, 2), 1e-3), np.full((G, 3), 1e-3), np.full(G, 1e-3))
    t_gauss = (time.perf_counter() - t0) * N / G
    sp, colors = setup if setup is not None else oracle_setup(scene, cam)
    pix = synth.sample_pixels(cam.width, cam.height, pixels, seed=seed)

    def pixel_stages(pp):
        t = time.perf_counter()
        r = oracle.render_splats(sp, colors, cam.width, cam.height, pixels=pp)
        d_img = np.sign(r["color"] - target_np[pp]) / (P * 3)
        oracle.render_splats_bwd(sp, colors, cam.width, cam.height, d_img, pixels=pp)
        return time.perf_counter() - t, r
    t_one, _ = pixel_stages(pix[:1])
    t_many, r = pixel_stages(pix)
    per_pixel = max(t_many - t_one, 0.0) / max(len(pix) - 1, 1)
    t_view = t_gauss + max(t_one - per_pixel, 0.0) + per_pixel * P
    sample_blends = int(r["blends"].sum())
    blends_view = kp_blends if kp_blends is not None else sample_blends * P / len(pix)
    return {"value": blends_view / t_view, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "ms_per_view_extrapolated": t_view * 1000.0,
            "sample": f"per-Gaussian stages on {G} of {N} Gaussians (x{N / G:.1f}); per-pixel fwd+bwd on {len(pix)} "
                      f"of {P} pixels (seed {seed}), {per_pixel * 1e3:.3f} ms/pixel, extrapolated linearly",
            "sample_blends": sample_blends}


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    scene, cams, desc = build_workload(args.workload, 0)
    cam = cams[0]
    rng = np.random.default_rng(5)
    target_np = rng.uniform(0.0, 1.0, (cam.width * cam.height, 3)).astype(np.float32)
    setup = oracle_setup(scene, cam)
    results = []
    for k in range(args.warmup + args.steps):
        r = cpu_baseline(scene, cam, target_np, args.ref_pixels, gauss_sample=50_000, setup=setup, seed=99 + k)
        if k >= args.warmup:
            results.append(r)
    t_view = float(np.mean([r["ms_per_view_extrapolated"] for r in results]))
    value = float(np.mean([r["value"] for r in results]))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_view, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded clustered Gaussians)",
            "config": {"workload": args.workload, "description": desc, "gaussians": scene.n},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": results[0]["cores"], "kind": "oracle",
                             "sample": results[0]["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="headline", choices=["headline", "training_step", "tiny"])
    ap.add_argument("--tile", type=int, default=16)
    ap.add_argument("--batch", type=int, default=256)
    ap.add_argument("--ppt", type=int, default=0, help="pixels per compositing thread (0 = library default)")
    ap.add_argument("--cpu-pixels", type=int, default=1024)
    ap.add_argument("--ref-pixels", type=int, default=128)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-graph", action="store_true", help="launch every stage directly instead of graph replays")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

#!/usr/bin/env python
"""Benchmark of the motion-blurred differentiable renderer on one GB300 (or N replicas).

Workload (the rotation scene of the plain-vs-fast comparison): icosphere subdiv 4 (2562 v, 5120 f)
with a degree-6 spherical-harmonic radial displacement (seeded), one full turn about a seeded axis
per exposure, T = 64 sub-frames, 256 x 256, 12 linear segments.  One step = forward render +
adjoint (dL/dimage fixed, seeded) with the fast solver -- every step of the hot path.  Synthetic
inputs stand in for the paper's ShapeNet scenes.

Headline: pixel x sub-frame samples/s of the fast solver's forward + backward.  Also reported:
forward+backward iterations/s, the plain per-sub-frame solver's numbers on the same GPU and the
fast/plain speedup, the roofline of the dominant raster kernel, the end-to-end number through
the C ABI with host buffers, and the FP64 oracle timed on the host cores (CPU baseline).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mbr|reference]
Under torchrun (N > 1) every rank renders its own replica (no collective on the data path);
timing is the max over ranks and the value is the aggregate.
"""
import argparse
import datetime
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "pixel x sub-frame samples/s, fast solver forward+backward"
UNIT = "samples/s"
WORKLOAD = ("rotation: icosphere subdiv 4 + SH degree 6 (2562 v, 5120 f), one turn about a seeded axis, "
            "T=64, 256x256, 12 segments; step = forward + adjoint")
CPU_WINDOW = (64, 64, 128, 128)   # bounded oracle sample for the CPU baseline (~20 s on one core)
REF_WINDOW = (96, 96, 64, 64)     # per-step oracle sample of the reference arm (all host cores)


def ref_window(steps):
    """The reference arm's per-step window: REF_WINDOW up to 200 steps, fewer rows beyond (at least
    16), so that a long --steps run still ends within a few minutes."""
    x0, y0, w, h = REF_WINDOW
    return (x0, y0, w, h if steps <= 200 else max(16, h * 200 // steps))
# DRAM bytes (read + write) per launch from the ncu captures summarised in profiles/ (tiles 8x8,
# this workload), by (kernel, sub-frames per thread); to be refreshed whenever the kernels change
# Pipe utilisation (% of active cycles) and issue-active share of the fast raster kernels at tiles
# 8x8, from one `ncu --set full` capture each on this workload (summaries in profiles/): the
# counter view of the roofline fraction next to the credited-flops view.
NCU_PIPES = {"raster_bwd_persistent": {"fma": 19.7, "alu": 27.3, "xu": 4.5, "lsu": 22.2, "issue_active": 43.0},
             "raster_fwd_persistent": {"fma": 20.0, "alu": 32.3, "xu": 8.2, "lsu": 21.7, "issue_active": 49.8}}
NCU_DRAM_BYTES = {("raster_bwd_persistent", 1): 34.93e6, ("raster_fwd_persistent", 1): 18.18e6,
                  ("raster_bwd_persistent", 2): 33.98e6, ("raster_fwd_persistent", 2): 16.90e6}


def _dist_env():
    return int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0"))


class Replicas:
    """Bookkeeping of an N-process run: one independent replica of the whole step per GPU, no
    data-path collective.  The barrier brackets the timed region and each rank's elapsed time is
    reduced with MAX, so the whole-job throughput is N x (units of one replica) / (slowest rank's
    time).  ``backend`` is "nccl" for the GPU run (tensors on ``device``) and "gloo" on CPU."""

    def __init__(self, world, rank, backend=None, device="cpu"):
        self.world, self.rank, self.device = world, rank, device
        self.dist = None
        if world > 1:
            import torch.distributed as dist
            if backend == "nccl":
                dist.init_process_group("nccl", device_id=device)
            else:
                dist.init_process_group(backend)
            self.dist = dist

    def barrier(self, sync=None):
        if self.dist is not None:
            self.dist.barrier()
        if sync is not None:
            sync()

    def max(self, x):
        if self.dist is None:
            return x
        import torch
        t = torch.tensor([x], dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def job_rate(self, units_per_replica, seconds):
        """Whole-job throughput: all replicas' units over the slowest rank's time."""
        return self.world * units_per_replica / seconds

    def close(self):
        if self.dist is not None:
            self.dist.barrier()
            self.dist.destroy_process_group()
            self.dist = None


def _clock_sampler():
    """nvidia-smi sampling the clocks and throttle reasons every 200 ms into a temporary file;
    returns once the first sample is written (or after 5 s), so that the timed region that follows
    is covered from its start."""
    try:
        f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        p = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms", "200"],
                             stdout=f, stderr=subprocess.DEVNULL)
        t_end = time.time() + 5.0
        while time.time() < t_end and p.poll() is None and os.path.getsize(f.name) == 0:
            time.sleep(0.02)
        return p, f.name
    except Exception:
        return None, None


def _sample_time(stamp):
    try:
        return datetime.datetime.strptime(stamp, "%Y/%m/%d %H:%M:%S.%f").timestamp()
    except ValueError:
        return None


def _clock_summary(proc, path, index, t0=None, t1=None):
    """Median SM clock, maximum SM clock and the throttle reasons seen by the samples taken between
    t0 and t1 (time.time() around the timed region); all samples if none falls inside."""
    if proc is None:
        return None
    proc.terminate()
    try:
        proc.wait(timeout=5)
    except Exception:
        proc.kill()
    rows = []
    try:
        for line in open(path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 10 and parts[1] == str(index):
                rows.append(parts)
        os.unlink(path)
    except Exception:
        return None
    if not rows:
        return None
    inside = [r for r in rows if t0 is not None and (_sample_time(r[0]) or 0.0) >= t0 and
              (_sample_time(r[0]) or 0.0) <= t1]
    use = inside or rows
    sm = [float(r[2]) for r in use if r[2].replace(".", "", 1).isdigit()]
    mx = [float(r[3]) for r in use if r[3].replace(".", "", 1).isdigit()]
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    reasons = sorted({names[i] for r in use for i in range(4) if r[6 + i].lower() == "active"})
    return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
            "reasons": reasons, "samples": len(use), "samples_in_timed_region": len(inside),
            "timed_region_s": None if t0 is None else round(t1 - t0, 3)}


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def _oracle_strip(job):
    """One worker's share of an oracle timing: fast-mode forward + backward of rows [r0, r1) of the
    window (x0, y0, w, h) of the rotation workload.  The loss gradient is the same seeded array for
    any split, so the strips together do exactly the window's work."""
    x0, y0, w, h, r0, r1 = job
    import numpy as np

    import oracle
    import scenes
    sc = scenes.config2()
    G = np.random.default_rng(7).normal(size=(h, w, 4))[r0:r1]
    win = (x0, y0 + r0, w, r1 - r0)
    t = time.perf_counter()
    oracle.render(sc, "fast", window=win)
    oracle.render_backward(sc, G, "fast", window=win)
    return time.perf_counter() - t


class OraclePool:
    """The FP64 oracle, as it stands, on all host cores: one single-threaded worker process per
    core (started with spawn, before any GPU work of this process), a window split into row
    strips across them."""

    def __init__(self, cores=None):
        import multiprocessing as mp
        import oracle
        oracle.build()
        self.cores = cores or os.cpu_count() or 1
        self.pool = mp.get_context("spawn").Pool(self.cores)
        self.pool.map(_oracle_strip, [(0, 0, 1, 1, 0, 1)] * self.cores)  # import and load in every worker

    def run(self, window):
        x0, y0, w, h = window
        n = min(self.cores, h)
        cuts = [round(h * i / n) for i in range(n + 1)]
        t = time.perf_counter()
        self.pool.map(_oracle_strip, [(x0, y0, w, h, cuts[i], cuts[i + 1]) for i in range(n)])
        return time.perf_counter() - t

    def close(self):
        self.pool.close()
        self.pool.join()


def run_reference(args):
    """Reference arm: the FP64 oracle (as it stands) on the host cores, each step a bounded window
    of the same workload, forward + backward of the fast solver's definition, split across one
    worker process per core."""
    world, rank, _ = _dist_env()
    if rank != 0:
        return 0
    import scenes
    pool = OraclePool()
    T = scenes.config2()["T"]
    win = ref_window(args.steps)
    x0, y0, w, h = win
    for _ in range(args.warmup):
        pool.run(win)
    dt = sum(pool.run(win) for _ in range(args.steps))
    pool.close()
    samples = w * h * T * args.steps
    value = samples / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": f"{w}x{h} pixel window at ({x0},{y0}) per step",
                       "parallelism": f"{pool.cores} host processes (one per core), row strips of the window"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": pool.cores, "kind": "oracle",
                             "sample": f"{w}x{h} window x {T} sub-frames per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def cpu_baseline(pool):
    """The oracle on the host cores: a window of the workload on every core (row strips), and the
    same window on one core."""
    import scenes
    T = scenes.config2()["T"]
    x0, y0, w, h = CPU_WINDOW
    dt_all = pool.run(CPU_WINDOW)
    dt_one = _oracle_strip((x0, y0, w, h, 0, h))
    n = w * h * T
    return {"value": n / dt_all, "unit": UNIT, "cores": pool.cores, "kind": "oracle",
            "sample": f"fast-mode forward+backward of a {w}x{h} window at ({x0},{y0}) of the same workload, "
                      f"all {T} sub-frames, {pool.cores} worker processes (row strips), {dt_all:.1f} s",
            "single_core": {"value": n / dt_one, "cores": 1, "seconds": dt_one}}


def extra_workloads(mbr, scenes, torch, np, world):
    """Context lines for the other workloads (same metric; not the headline): an 8-view shape-recovery
    iteration (c3), a 32-object batch (c4) and the 1024^2 / 100k-face / T=256 render (c5)."""
    from paper_2602_07860_gb300.recovery import ViewBatch
    out = {}

    def timeit(fn, reps):
        fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / reps * 1e3

    # c3: one iteration of the recovery loop's renders (8 views, forward + adjoint, batched)
    views_sc, template = scenes.config3()
    s0 = views_sc[0]
    dev = "cuda"
    tv = torch.as_tensor(np.asarray(template, np.float32), device=dev).contiguous()
    tf = torch.as_tensor(np.asarray(s0["faces"], np.int32), device=dev).contiguous()
    ta = torch.as_tensor(np.asarray(s0["albedo"], np.float32), device=dev).contiguous()
    views = [(mbr.motion_from_dict(s["motion"]), mbr.camera_from_dict(s["camera"])) for s in views_sc]
    vb = ViewBatch(tv, tf, ta, views, s0["T"], s0["H"], s0["W"], "fast")
    g = torch.randn((len(views), s0["H"], s0["W"], 4), device=dev, generator=torch.Generator(dev).manual_seed(5))
    ms = timeit(lambda: (vb.forward(), vb.backward(g)), 5)
    n = len(views) * s0["H"] * s0["W"] * s0["T"]
    out["c3_recovery_iteration"] = {"ms": ms, "samples_per_s": world * n / (ms / 1e3), "views": len(views),
                                    "workload": "8 views (4 translations, 4 rotations), 2562 v, T=64, 256x256"}
    # c4: 32 objects of mixed size in one batched forward + adjoint
    items, n = [], 0
    ctx = mbr.Context()
    for s in scenes.config4():
        vv, ff, aa = mbr.mesh_tensors(s)
        n += s["H"] * s["W"] * s["T"]
        items.append(dict(verts=vv, faces=ff, albedo=aa, motion=mbr.motion_from_dict(s["motion"]),
                          camera=mbr.camera_from_dict(s["camera"]), T=s["T"], H=s["H"], W=s["W"], solver="fast",
                          image=torch.zeros((s["H"], s["W"], 4), device=dev),
                          dl_dimage=torch.ones((s["H"], s["W"], 4), device=dev),
                          dl_dverts=torch.zeros_like(vv), dl_dalbedo=torch.zeros_like(aa)))
    ms = timeit(lambda: ctx.render_batch(items, True), 3)
    out["c4_batch_32_objects"] = {"ms": ms, "samples_per_s": world * n / (ms / 1e3), "samples": n,
                                  "workload": "32 objects, subdiv 2-5, T in {16..256}, 128-512 px, one graph replay"}
    # c5: the large render, both solvers
    s = scenes.config5()
    vv, ff, aa = mbr.mesh_tensors(s)
    mo, ca = mbr.motion_from_dict(s["motion"]), mbr.camera_from_dict(s["camera"])
    T, H, W = s["T"], s["H"], s["W"]
    G5 = torch.ones((H, W, 4), device=dev)
    ctx5 = mbr.Context()
    c5 = {"workload": f"surface of revolution {ff.shape[0]} faces, 8 turns, T=256, 1024x1024, 96 segments"}
    for solver in ("fast", "plain"):
        ms = timeit(lambda: (ctx5.render_blur(vv, ff, aa, mo, ca, T, H, W, solver),
                             ctx5.render_blur_backward(vv, ff, aa, mo, ca, T, H, W, G5, solver, reuse_forward=True)), 2)
        c5[solver] = {"fwdbwd_ms": ms, "samples_per_s": world * H * W * T / (ms / 1e3)}
    out["c5_large"] = c5
    # segmentation analysis on the benchmark workload: linear segments of the fast solver vs the
    # exact per-sub-frame render (plain): time and image error
    import dataclasses
    s2 = scenes.config2()
    v2, f2, a2 = mbr.mesh_tensors(s2)
    mo2, ca2 = mbr.motion_from_dict(s2["motion"]), mbr.camera_from_dict(s2["camera"])
    T2, H2, W2 = s2["T"], s2["H"], s2["W"]
    G2 = torch.ones((H2, W2, 4), device=dev)
    ctx2 = mbr.Context()
    exact = ctx2.render_blur(v2, f2, a2, mo2, ca2, T2, H2, W2, "plain").clone()
    sweep = {}
    for S in (6, 12, 24, 48):
        m = dataclasses.replace(mo2, segments=S)
        img = ctx2.render_blur(v2, f2, a2, m, ca2, T2, H2, W2, "fast")
        err = (img - exact).abs()
        ms = timeit(lambda: (ctx2.render_blur(v2, f2, a2, m, ca2, T2, H2, W2, "fast"),
                             ctx2.render_blur_backward(v2, f2, a2, m, ca2, T2, H2, W2, G2, "fast",
                                                       reuse_forward=True)), 5)
        sweep[str(S)] = {"fwdbwd_ms": ms, "mean_abs_err_vs_exact": float(err.mean()), "max_abs_err_vs_exact": float(err.max())}
    out["segment_sweep"] = sweep
    # the paper's translational recovery setting: 16 views of 128^2 per iteration from a 1352-vertex
    # template (Eq. loss-img, Adam (0.01, 0.5, 0.99)), T = 16
    from paper_2602_07860_gb300.recovery import ViewBatch as _VB, recover_translational
    rng = np.random.default_rng(21)
    tv, tf = scenes.sh_sphere(4, 6, 0.08, rng)
    views = []
    for i in range(40):
        cam = mbr.camera_from_dict(scenes.camera(scenes.look_at(scenes.orbit_eye(4.0, 9.0 * i, 20.0 * ((i % 3) - 1)))))
        views.append((mbr.motion_from_dict(scenes.translate(scenes.random_unit(rng) * rng.uniform(0.5, 2.0))), cam))
    tt = lambda x, dt=torch.float32: torch.as_tensor(np.asarray(x), dtype=dt, device=dev).contiguous()
    alb = tt(scenes.random_albedo(len(tv), rng))
    tgt = torch.cat([_VB(tt(tv), tt(tf, torch.int32), alb, views[i:i + 8], 16, 128, 128, "fast").forward().clone()
                     for i in range(0, 40, 8)])
    sv, sf = scenes.uv_sphere()
    iters = 20
    recover_translational(tt(sv), tt(sf, torch.int32), torch.full((len(sv), 3), 0.5, device=dev), views, tgt, 16, 128,
                          128, iters=2)  # warm-up (plans and captures)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, _, hist = recover_translational(tt(sv), tt(sf, torch.int32), torch.full((len(sv), 3), 0.5, device=dev), views,
                                       tgt, 16, 128, 128, iters=iters)
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) / iters * 1e3
    out["translational_recovery_iteration"] = {
        "ms": ms, "samples_per_s": world * 16 * 128 * 128 * 16 / (ms / 1e3),
        "workload": "16 of 40 translation-blurred views, 128x128, T=16, 1352-vertex UV-sphere template, "
                    "L1 + smoothness + Laplacian, Adam (0.01, 0.5, 0.99); includes loss terms and optimiser",
        "image_loss_first_last": [hist[0][0], hist[-1][0]]}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    # 600 timed steps take about 0.65 s: three or more clock samples at the sampler's 200 ms
    ap.add_argument("--steps", type=int, default=600)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mbr", choices=["mbr", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra-workloads", action="store_true")
    ap.add_argument("--tile", type=int, default=0, help="fixed tile edge (with --spt): skip the autotuner")
    ap.add_argument("--spt", type=int, default=0)
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    world, rank, _ = _dist_env()
    # the oracle's worker processes start before this process touches the GPU
    cpu_pool = OraclePool() if rank == 0 and world == 1 and not args.no_cpu_baseline else None

    import numpy as np
    import torch

    import paper_2602_07860_gb300 as mbr
    import scenes
    from paper_2602_07860_gb300 import roofline

    world, rank, local = _dist_env()
    torch.cuda.set_device(local)
    reps = Replicas(world, rank, "nccl", torch.device("cuda", local))

    def barrier():
        reps.barrier(torch.cuda.synchronize)

    max_over_ranks = reps.max

    ctx = mbr.Context()
    sc = scenes.config2()
    T, H, W = sc["T"], sc["H"], sc["W"]
    v, f, a = mbr.mesh_tensors(sc)
    mo, ca = mbr.motion_from_dict(sc["motion"]), mbr.camera_from_dict(sc["camera"])
    G = torch.as_tensor(np.random.default_rng(11).normal(size=(H, W, 4)).astype(np.float32), device="cuda")
    # tile shape and sub-frames per group from the library's autotuner (untimed), kept on ctx
    tune_item = dict(verts=v, faces=f, albedo=a, motion=mo, camera=ca, T=T, H=H, W=W, solver="fast",
                     image=torch.zeros((H, W, 4), device="cuda"), dl_dimage=G, dl_dverts=torch.zeros_like(v),
                     dl_dalbedo=torch.zeros_like(a))
    if args.tile and args.spt:
        tile, ctx_spt = args.tile, args.spt
        ctx.set_tuning(tile, ctx_spt, 0)
    else:
        tile, ctx_spt, _ = ctx.autotune([tune_item], True)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")  # > 129 MB L2
    n_samples = H * W * T

    def step(solver, bwd=True):
        # forward, then the adjoint as the autograd path runs it (reusing the forward's front half)
        ctx.render_blur(v, f, a, mo, ca, T, H, W, solver)
        if bwd:
            ctx.render_blur_backward(v, f, a, mo, ca, T, H, W, G, solver, reuse_forward=True)

    def timed(solver, bwd, steps, warmup, t_region=None):
        for _ in range(warmup):
            step(solver, bwd)
        barrier()
        if t_region is not None:
            t_region[0] = time.time()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for e0, e1 in ev:
            flush.zero_()
            e0.record()
            step(solver, bwd)
            e1.record()
        barrier()
        if t_region is not None:
            t_region[1] = time.time()
        return sum(e0.elapsed_time(e1) for e0, e1 in ev)

    # ---- headline: fast solver forward + backward, raster kernels timed by events in the library
    l0 = ctx.stats()["launches"]
    ctx.set_profiling(True)
    proc, path = _clock_sampler() if rank == 0 else (None, None)
    t_region = [0.0, 0.0]
    total_ms = timed("fast", True, args.steps, args.warmup, t_region)
    clocks = _clock_summary(proc, path, local, *t_region) if rank == 0 else None
    st = ctx.stats()
    ctx.set_profiling(False)
    launches = (st["launches"] - l0) * args.steps // (args.steps + args.warmup)
    total_ms = max_over_ranks(total_ms)
    ms_per_step = total_ms / args.steps
    value = reps.job_rate(n_samples * args.steps, total_ms / 1e3)

    # ---- roofline of the dominant raster kernel (FP32 ALU bound); work units counted by the GPU
    # path itself (mbr_count_work), flops per unit from the formulas (roofline.py)
    fwd_ms = st["raster_fwd_ms"] / max(1, st["raster_fwd_count"])
    bwd_ms = st["raster_bwd_ms"] / max(1, st["raster_bwd_count"])
    num_sms = torch.cuda.get_device_properties(local).multi_processor_count
    peak = roofline.fp32_peak_tflops(num_sms)

    def kernel_roofs(solver, f_ms, b_ms):
        d = ctx.count_work(v, f, a, mo, ca, T, H, W, solver, detail=True)
        n_box, n_soft, n_cov = d["n_box"], d["n_soft"], d["n_cov"]
        fw = roofline.fwd_flops(solver, n_box, n_soft, n_cov, n_samples)
        bw = roofline.bwd_flops(solver, n_box, n_soft, n_cov, n_samples)
        units = dict(d, n_sample=n_samples)
        return fw, bw, units, fw / (f_ms / 1e3) / 1e12, bw / (b_ms / 1e3) / 1e12

    fwf, bwf, units, fwd_tf, bwd_tf = kernel_roofs("fast", fwd_ms, bwd_ms)
    backward_dominant = bwd_ms >= fwd_ms
    kern = "raster_bwd_persistent" if backward_dominant else "raster_fwd_persistent"
    achieved = bwd_tf if backward_dominant else fwd_tf
    traffic = NCU_DRAM_BYTES.get((kern, ctx_spt)) if tile == 8 else None
    roof = {"bound": "alu", "kernel": kern, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": traffic,
            "traffic_note": f"DRAM bytes per launch from ncu (profiles/), tiles 8x8, spt {ctx_spt}",
            "peak_note": f"{num_sms} SMs x 128 FP32 lanes x 2 flops x 2070 MHz (derived from unit counts "
                         "and the maximum SM clock; no measured FP32 peak)",
            "work": roofline.describe("fast", units["n_box"], units["n_soft"], units["n_cov"], n_samples,
                                      backward_dominant),
            "flops_per_launch": bwf if backward_dominant else fwf,
            "kernel_ms": bwd_ms if backward_dominant else fwd_ms, "raster_fwd_ms": fwd_ms, "raster_bwd_ms": bwd_ms,
            "fwd_frac": fwd_tf / peak, "bwd_frac": bwd_tf / peak, "units": units,
            "ncu_pipes_pct": NCU_PIPES.get(kern) if tile == 8 else None}

    # ---- plain per-sub-frame solver and forward-only numbers on the same GPU
    k2 = max(3, args.steps // 2)
    ctx.set_profiling(True)
    plain_fb = max_over_ranks(timed("plain", True, k2, 2)) / k2
    pst = ctx.stats()
    ctx.set_profiling(False)
    p_fwd = pst["raster_fwd_ms"] / max(1, pst["raster_fwd_count"])
    p_bwd = pst["raster_bwd_ms"] / max(1, pst["raster_bwd_count"])
    _, _, p_units, p_fwd_tf, p_bwd_tf = kernel_roofs("plain", p_fwd, p_bwd)
    fast_f = max_over_ranks(timed("fast", False, k2, 2)) / k2
    plain_f = max_over_ranks(timed("plain", False, k2, 2)) / k2
    extras = {
        "fast_fwdbwd_iters_per_s": 1e3 / ms_per_step,
        "plain_fwdbwd_ms": plain_fb, "plain_fwdbwd_samples_per_s": world * n_samples / (plain_fb / 1e3),
        "plain_fwdbwd_iters_per_s": 1e3 / plain_fb,
        "fast_fwd_ms": fast_f, "fast_fwd_samples_per_s": world * n_samples / (fast_f / 1e3),
        "plain_fwd_ms": plain_f, "plain_fwd_samples_per_s": world * n_samples / (plain_f / 1e3),
        "speedup_fast_over_plain_fwdbwd": plain_fb / ms_per_step,
        "speedup_fast_over_plain_fwd": plain_f / fast_f,
        "plain_raster_fwd_ms": p_fwd, "plain_raster_bwd_ms": p_bwd,
        "plain_fwd_frac": p_fwd_tf / peak, "plain_bwd_frac": p_bwd_tf / peak, "plain_units": p_units,
        "tuning": {"tile": tile, "spt": ctx_spt, "splits": "auto",
                   "chosen_by": "command line" if (args.tile and args.spt) else "mbr_autotune"},
        "paper_context": "paper: up to 4.57x fwd+grad speedup vs SoftRas on one RTX 4090 (different workload)",
    }

    # ---- end to end through the C ABI with host buffers (pinned), copies inside the timed region
    hv, hf, ha, hG = v.cpu().pin_memory(), f.cpu().pin_memory(), a.cpu().pin_memory(), G.cpu().pin_memory()
    out_img = torch.empty((H, W, 4), dtype=torch.float32).pin_memory()
    out_gv = torch.empty_like(hv).pin_memory()
    out_ga = torch.empty_like(ha).pin_memory()
    dv, df, da, dG = torch.empty_like(v), torch.empty_like(f), torch.empty_like(a), torch.empty_like(G)

    def e2e_step():
        dv.copy_(hv, non_blocking=True)
        df.copy_(hf, non_blocking=True)
        da.copy_(ha, non_blocking=True)
        dG.copy_(hG, non_blocking=True)
        img = ctx.render_blur(dv, df, da, mo, ca, T, H, W, "fast")
        gv, ga = ctx.render_blur_backward(dv, df, da, mo, ca, T, H, W, dG, "fast", reuse_forward=True)
        out_img.copy_(img, non_blocking=True)
        out_gv.copy_(gv, non_blocking=True)
        out_ga.copy_(ga, non_blocking=True)

    for _ in range(2):
        e2e_step()
    barrier()
    t0 = time.perf_counter()
    for _ in range(k2):
        e2e_step()
        torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    barrier()
    # untimed: the overlapped read-back delivered the image of the step
    check = ctx.render_blur(v, f, a, mo, ca, T, H, W, "fast").cpu()
    if not torch.allclose(out_img, check, atol=1e-6, rtol=0.0):
        raise RuntimeError("end-to-end step: the image read back differs from a fresh render")
    h2d = sum(t.numel() * t.element_size() for t in (hv, hf, ha, hG))
    d2h = sum(t.numel() * t.element_size() for t in (out_img, out_gv, out_ga))
    e2e = {"value": world * n_samples * k2 / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": d2h, "ms_per_step": 1e3 * e2e_s / k2}

    if not args.no_extra_workloads:
        extras.update(extra_workloads(mbr, scenes, torch, np, world))

    cpu = None
    if cpu_pool is not None:
        cpu = cpu_baseline(cpu_pool)
        cpu_pool.close()

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD, "solver": "fast", "l2": "flushed between steps (256 MiB write)",
                           "step": "mbr_render_blur + mbr_render_blur_backward_reuse (the autograd path)",
                           "parallelism": f"{world} independent replica(s)"},
                "clocks": clocks, "e2e": e2e, "gpu_launches": int(launches), "roofline": roof,
                "cpu_baseline": cpu, "extras": extras}
        print(json.dumps(line), flush=True)
    reps.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())

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
# Counters of the dominant raster kernels from one ncu capture each (summaries in profiles/): DRAM
# bytes per launch and pipe utilisation (% of active cycles).  They describe the kernels as they were
# compiled when captured: the entry is attached to the bench line only if the current kernel
# sources hash to CAPTURED["sources"] and the run uses the captured tile / samples-per-group;
# otherwise the line carries null.
CAPTURED = {
    "sources": "df90c844e7d43555", "tile": 8, "spt": 2,
    "kernels": {
        # profiles/raster_bwd_persistent_c2_fast.md
        "raster_bwd_persistent": {"dram_bytes": 33804288 + 762624,
                                  "pipes_pct": {"fma": 30.7, "alu": 33.9, "xu": 6.4, "lsu": 23.0, "issue_active": 59.7}},
        # profiles/raster_fwd_persistent_c2_fast.md
        "raster_fwd_persistent": {"dram_bytes": 17357568 + 233216,
                                  "pipes_pct": {"fma": 32.3, "alu": 44.1, "xu": 10.0, "lsu": 28.4, "issue_active": 72.9}},
    },
}


def kernel_sources_sha():
    """sha256 (first 16 hex digits) of the CUDA sources the library is built from."""
    import hashlib
    d = os.path.join(ROOT, "paper_2602_07860_gb300", "csrc")
    h = hashlib.sha256()
    for name in sorted(os.listdir(d)):
        if name.endswith((".cu", ".cuh", ".h")):
            h.update(name.encode())
            h.update(open(os.path.join(d, name), "rb").read())
    return h.hexdigest()[:16]


def captured_counters(kernel, tile, spt):
    """The captured counters of ``kernel`` if they still describe this build and configuration."""
    if CAPTURED["sources"] != kernel_sources_sha() or (CAPTURED["tile"], CAPTURED["spt"]) != (tile, spt):
        return None
    return CAPTURED["kernels"].get(kernel)


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


def _clock_summary(proc, path, index, t0=None, t1=None, keep_rows=False):
    """Median SM clock, maximum SM clock and the throttle reasons seen by the samples taken between
    t0 and t1 (time.time() around the timed region); all samples if none falls inside.  With
    keep_rows: (summary, all rows of this GPU) so that other intervals can be summarised too."""
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
    summary = _summarise_rows(rows, t0, t1)
    return (summary, rows) if keep_rows else summary


def _summarise_rows(rows, t0, t1):
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

    # c3: the shape-recovery run to its end: 8 blurred views (4 translations, 4 rotations) of the
    # SH-8 target, 256^2, T = 64; Adam (lr 1e-3) on the undisplaced sphere's vertices for 500
    # iterations, L2 image loss + 0.1 Laplacian; every iteration one graph replay of the 8-view
    # forward batch and one of the adjoint batch
    from paper_2602_07860_gb300.recovery import recover_shape
    views_sc, template = scenes.config3()
    s0 = views_sc[0]
    dev = "cuda"
    tt = lambda x, dt=torch.float32: torch.as_tensor(np.asarray(x), dtype=dt, device=dev).contiguous()
    tgt_v = tt(s0["verts"])
    tf = tt(s0["faces"], torch.int32)
    ta = tt(s0["albedo"])
    views = [(mbr.motion_from_dict(s["motion"]), mbr.camera_from_dict(s["camera"])) for s in views_sc]
    targets = ViewBatch(tgt_v, tf, ta, views, s0["T"], s0["H"], s0["W"], "fast").forward().clone()
    tv = tt(template)
    vb = ViewBatch(tv.clone(), tf, ta, views, s0["T"], s0["H"], s0["W"], "fast")
    g = torch.randn((len(views), s0["H"], s0["W"], 4), device=dev, generator=torch.Generator(dev).manual_seed(5))
    ms = timeit(lambda: (vb.forward(), vb.backward(g)), 5)
    n = len(views) * s0["H"] * s0["W"] * s0["T"]
    out["c3_recovery_iteration"] = {"ms": ms, "samples_per_s": world * n / (ms / 1e3), "views": len(views),
                                    "workload": "8 views (4 translations, 4 rotations), 2562 v, T=64, 256x256"}
    iters, marks, track = 500, (0, 100, 250, 499), {}

    def on_iter(it, v, img_loss):
        if it in marks:
            track[it] = (float(img_loss), float((v - tgt_v).norm(dim=1).mean()))

    # untimed warm-up: the loop's one-time costs (the batch plans and graph captures, and PyTorch's
    # first use of the optimiser's and the loss terms' kernels, which a fresh process may have to
    # compile for this GPU) stay out of the per-iteration time
    recover_shape(tv, tf, ta, views, targets, s0["T"], s0["H"], s0["W"], iters=2, lr=1e-3, lap_weight=0.1,
                  solver="fast")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    v_final, hist = recover_shape(tv, tf, ta, views, targets, s0["T"], s0["H"], s0["W"], iters=iters, lr=1e-3,
                                  lap_weight=0.1, solver="fast", on_iter=on_iter)
    torch.cuda.synchronize()
    run_s = time.perf_counter() - t0
    out["c3_recovery_run"] = {
        "iterations": iters, "seconds": run_s, "ms_per_iteration": 1e3 * run_s / iters,
        "image_loss": {str(k): track[k][0] for k in marks},
        "mean_vertex_distance_to_target": {str(k): track[k][1] for k in marks},
        "final_mean_vertex_distance_to_target": float((v_final - tgt_v).norm(dim=1).mean()),
        "workload": "8 views, 256x256, T=64, Adam lr 1e-3, L2 image loss + 0.1 Laplacian, from the undisplaced "
                    "subdiv-4 sphere towards the SH-8 target (same topology: per-vertex distance)",
        "includes": "renders, adjoint, loss terms, optimiser, one host read of the loss per iteration"}
    # c4: 32 objects of mixed size in one batched forward + adjoint, tiles chosen by the autotuner
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
    tile4, spt4, tune_ms = ctx.autotune(items, True)
    ms = timeit(lambda: ctx.render_batch(items, True), 3)
    out["c4_batch_32_objects"] = {"ms": ms, "samples_per_s": world * n / (ms / 1e3), "samples": n,
                                  "tuning": {"tile": tile4, "spt": spt4, "autotune_best_ms": tune_ms,
                                             "chosen_by": "mbr_autotune"},
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
    # the adjoint's per-sample state, kept (5 bytes per sample, written by the forward) or
    # recomputed by the adjoint (mbr_set_state_budget 0), on c2 and c5; by default c2 keeps it and
    # c5 (1.34 GB of state, above the 1 GiB default budget) recomputes it
    modes = {}
    s2m = scenes.config2()
    v2m, f2m, a2m = mbr.mesh_tensors(s2m)
    cases = (("c2", (v2m, f2m, a2m, mbr.motion_from_dict(s2m["motion"]), mbr.camera_from_dict(s2m["camera"]),
                     s2m["T"], s2m["H"], s2m["W"]), 10),
             ("c5", (vv, ff, aa, mo, ca, T, H, W), 2))
    for label, (mv, mf, ma, mmo, mca, mT, mH, mW), reps in cases:
        mG = torch.ones((mH, mW, 4), device=dev)
        row = {"state_bytes_if_kept": mT * mH * mW * 5}
        for mode, budget in (("kept", 1 << 34), ("recomputed", 0)):
            cx = mbr.Context()
            cx.set_state_budget(budget)
            ms = timeit(lambda: (cx.render_blur(mv, mf, ma, mmo, mca, mT, mH, mW, "fast"),
                                 cx.render_blur_backward(mv, mf, ma, mmo, mca, mT, mH, mW, mG, "fast",
                                                         reuse_forward=True)), reps)
            row[mode] = {"fwdbwd_ms": ms, "samples_per_s": world * mT * mH * mW / (ms / 1e3)}
            cx.close()
        modes[label] = row
    out["adjoint_state_modes"] = modes
    # translation (one linear segment) at growing T: the plain solver places vertices, builds
    # records and bins per sub-frame, the fast solver per keyframe (2 slots); fwd+bwd ms per solver
    tsweep = {}
    for Tn in (64, 256, 1024):
        st_ = scenes.config2_translate(T=Tn)
        tv_, tf_, ta_ = mbr.mesh_tensors(st_)
        tmo, tca = mbr.motion_from_dict(st_["motion"]), mbr.camera_from_dict(st_["camera"])
        tG = torch.ones((st_["H"], st_["W"], 4), device=dev)
        row = {}
        for solver in ("fast", "plain"):
            cx = mbr.Context()
            cx.set_tuning(8, 2 if solver == "fast" else 1, 0)
            ms = timeit(lambda: (cx.render_blur(tv_, tf_, ta_, tmo, tca, Tn, st_["H"], st_["W"], solver),
                                 cx.render_blur_backward(tv_, tf_, ta_, tmo, tca, Tn, st_["H"], st_["W"], tG, solver,
                                                         reuse_forward=True)), 5)
            row[solver] = {"fwdbwd_ms": ms, "samples_per_s": world * Tn * st_["H"] * st_["W"] / (ms / 1e3)}
            cx.close()
        row["speedup_fast_over_plain_fwdbwd"] = row["plain"]["fwdbwd_ms"] / row["fast"]["fwdbwd_ms"]
        tsweep[str(Tn)] = row
    out["translate_T_sweep"] = tsweep
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
    # the rotation task through an SDF (NEXT-4): 5 views of a spinning SH-displaced sphere, the field on a
    # 33^3 grid starting from the paper's inclined ellipsoid, Adam (5e-4, 0.9, 0.999) as in the paper
    from paper_2602_07860_gb300.sdf import ellipsoid_sdf, extract_mesh, recover_rotational
    rsc = scenes.config_sdf_rotation()
    rctx = mbr.Context()
    rv, rf, ra = mbr.mesh_tensors(rsc[0])
    rviews = [(mbr.motion_from_dict(s["motion"]), mbr.camera_from_dict(s["camera"])) for s in rsc]
    rT, rH, rW = rsc[0]["T"], rsc[0]["H"], rsc[0]["W"]
    rtgt = torch.stack([rctx.render_blur(rv, rf, ra, mo, ca, rT, rH, rW, "fast").clone() for mo, ca in rviews])
    n_grid, lo = 32, (-1.1, -1.1, -1.1)
    hg = 2.2 / n_grid
    s0 = ellipsoid_sdf(n_grid, lo, hg)

    def gap(sdf):
        verts, _ = extract_mesh(sdf, lo, hg, rctx)
        return float(torch.cdist(verts, rv).min(dim=1).values.mean())

    r_iters = 300
    recover_rotational(s0, lo, hg, rviews, rtgt, rT, rH, rW, iters=3)  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sdf_end, rhist = recover_rotational(s0, lo, hg, rviews, rtgt, rT, rH, rW, iters=r_iters)
    torch.cuda.synchronize()
    r_ms = (time.perf_counter() - t0) / r_iters * 1e3
    out["sdf_rotational_recovery"] = {
        "iterations": r_iters, "ms_per_iteration": r_ms, "image_loss_first_last": [rhist[0][0], rhist[-1][0]],
        "faces_first_last": [rhist[0][2], rhist[-1][2]], "surface_gap_first_last": [gap(s0), gap(sdf_end)],
        "workload": f"5 views (elevations -40..40 deg), one turn about +y, T={rT}, {rH}x{rW}, fast solver; SDF grid "
                    f"{n_grid + 1}^3 from the inclined ellipsoid; Adam (5e-4, 0.9, 0.999); L1 image loss + SDF "
                    "regularisers; per iteration: extraction, 5 renders + adjoints, extraction adjoint"}
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

    class Scene:
        """Timing of one scene on ctx: forward (+ adjoint reusing the forward's front half, as the
        autograd path runs it), L2 flushed before every timed step, CUDA events around each step;
        the library's own events time the raster kernels."""

        def __init__(self, scd):
            self.sc = scd
            self.T, self.H, self.W = scd["T"], scd["H"], scd["W"]
            self.v, self.f, self.a = mbr.mesh_tensors(scd)
            self.mo, self.ca = mbr.motion_from_dict(scd["motion"]), mbr.camera_from_dict(scd["camera"])
            self.G = torch.as_tensor(np.random.default_rng(11).normal(size=(self.H, self.W, 4)).astype(np.float32),
                                     device="cuda")
            self.n = self.H * self.W * self.T

        def step(self, solver, bwd=True):
            ctx.render_blur(self.v, self.f, self.a, self.mo, self.ca, self.T, self.H, self.W, solver)
            if bwd:
                ctx.render_blur_backward(self.v, self.f, self.a, self.mo, self.ca, self.T, self.H, self.W, self.G,
                                         solver, reuse_forward=True)

        def timed(self, solver, bwd, steps, warmup, t_region=None):
            """(total ms over the timed steps, library stats of the timed steps)"""
            for _ in range(warmup):
                self.step(solver, bwd)
            barrier()
            ctx.set_profiling(True)
            if t_region is not None:
                t_region[0] = time.time()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
            for e0, e1 in ev:
                flush.zero_()
                e0.record()
                self.step(solver, bwd)
                e1.record()
            barrier()
            if t_region is not None:
                t_region[1] = time.time()
            st_ = ctx.stats()
            ctx.set_profiling(False)
            return max_over_ranks(sum(e0.elapsed_time(e1) for e0, e1 in ev)), st_

        def units(self, solver):
            d = ctx.count_work(self.v, self.f, self.a, self.mo, self.ca, self.T, self.H, self.W, solver, detail=True)
            return dict(d, n_sample=self.n)

        def fracs(self, solver, st_, peak_tf):
            """raster kernel ms, credited TFLOP/s and fraction of the measured peak, per direction"""
            u = self.units(solver)
            out = {"units": u}
            for key, fl_fn, cnt in (("fwd", roofline.fwd_flops, "raster_fwd"), ("bwd", roofline.bwd_flops, "raster_bwd")):
                if st_[cnt + "_count"]:
                    k_ms = st_[cnt + "_ms"] / st_[cnt + "_count"]
                    fl = fl_fn(solver, u["n_box"], u["n_soft"], u["n_cov"], self.n)
                    tf = fl / (k_ms / 1e3) / 1e12
                    out[key] = {"raster_ms": k_ms, "flops": fl, "tflops": tf, "frac": tf / peak_tf}
            return out

    main_scene = Scene(sc)
    main_scene.v, main_scene.f, main_scene.a, main_scene.G = v, f, a, G

    # ---- headline: fast solver forward + backward, raster kernels timed by events in the library
    l0 = ctx.stats()["launches"]
    proc, path = _clock_sampler() if rank == 0 else (None, None)
    t_region = [0.0, 0.0]
    total_ms, st = main_scene.timed("fast", True, args.steps, args.warmup, t_region)
    launches = (ctx.stats()["launches"] - l0) * args.steps // (args.steps + args.warmup)
    ms_per_step = total_ms / args.steps
    value = reps.job_rate(n_samples * args.steps, total_ms / 1e3)
    # ---- the roofline's denominator, measured now: FMA chains on every SM for about half a second
    t_peak = [time.time(), 0.0]
    peak, peak_flops, peak_ms = ctx.measure_fp32_peak(iters=20000, launches=25)
    t_peak[1] = time.time()
    clock_rows = _clock_summary(proc, path, local, *t_region, keep_rows=True) if rank == 0 else None
    clocks = clock_rows[0] if clock_rows else None
    peak_clocks = _summarise_rows(clock_rows[1], *t_peak) if clock_rows else None
    num_sms = torch.cuda.get_device_properties(local).multi_processor_count
    peak_derived = roofline.fp32_peak_tflops(num_sms)

    # ---- roofline of the dominant raster kernel (FP32 ALU bound); work units counted by the GPU
    # path itself (mbr_count_work), flops per unit from the formulas (roofline.py)
    rf = main_scene.fracs("fast", st, peak)
    units = rf["units"]
    fwd_ms, bwd_ms = rf["fwd"]["raster_ms"], rf["bwd"]["raster_ms"]
    backward_dominant = bwd_ms >= fwd_ms
    kern = "raster_bwd_persistent" if backward_dominant else "raster_fwd_persistent"
    dom = rf["bwd"] if backward_dominant else rf["fwd"]
    cap = captured_counters(kern, tile, ctx_spt)
    roof = {"bound": "alu", "kernel": kern, "achieved": dom["tflops"], "peak": peak, "unit": "TFLOP/s",
            "frac": dom["frac"], "traffic": cap["dram_bytes"] if cap else None,
            "traffic_note": (f"ncu DRAM bytes per launch, captured on these kernel sources at tile {tile}, "
                             f"spt {ctx_spt}" if cap else "null: no ncu capture of the current kernel sources "
                             "in this configuration"),
            "peak_measured": peak,
            "peak_note": (f"measured in this run: mbr_measure_fp32_peak, FMA chains on all {num_sms} SMs, "
                          f"{peak_flops:.3e} flops in {peak_ms:.0f} ms (CUDA events); clocks during it: "
                          f"{peak_clocks}"),
            "peak_derived": peak_derived, "frac_of_derived": dom["tflops"] / peak_derived,
            "peak_derived_note": f"{num_sms} SMs x 128 FP32 lanes x 2 flops x 2070 MHz",
            "work": roofline.describe("fast", units["n_box"], units["n_soft"], units["n_cov"], n_samples,
                                      backward_dominant),
            "flops_per_launch": dom["flops"], "kernel_ms": dom["raster_ms"],
            "raster_fwd_ms": fwd_ms, "raster_bwd_ms": bwd_ms,
            "fwd_frac": rf["fwd"]["frac"], "bwd_frac": rf["bwd"]["frac"], "units": units,
            "ncu_pipes_pct": cap["pipes_pct"] if cap else None, "n_split": st["n_split"], "groups": st["groups"]}

    # ---- plain per-sub-frame solver and forward-only numbers on the same GPU (rotation)
    k2 = max(3, args.steps // 2)
    plain_fb, pst = main_scene.timed("plain", True, k2, 2)
    plain_fb /= k2
    prf = main_scene.fracs("plain", pst, peak)
    fast_f, fst = main_scene.timed("fast", False, k2, 2)
    fast_f /= k2
    plain_f, _ = main_scene.timed("plain", False, k2, 2)
    plain_f /= k2
    extras = {
        "fast_fwdbwd_iters_per_s": 1e3 / ms_per_step,
        "plain_fwdbwd_ms": plain_fb, "plain_fwdbwd_samples_per_s": world * n_samples / (plain_fb / 1e3),
        "plain_fwdbwd_iters_per_s": 1e3 / plain_fb,
        "speedup_fast_over_plain_fwdbwd": plain_fb / ms_per_step,
        "c2_forward_plain_vs_fast": {
            "fast_ms": fast_f, "plain_ms": plain_f, "speedup_fast_over_plain": plain_f / fast_f,
            "fast_samples_per_s": world * n_samples / (fast_f / 1e3),
            "plain_samples_per_s": world * n_samples / (plain_f / 1e3),
            "fast_raster_ms": fst["raster_fwd_ms"] / max(1, fst["raster_fwd_count"])},
        "plain_raster_fwd_ms": prf["fwd"]["raster_ms"], "plain_raster_bwd_ms": prf["bwd"]["raster_ms"],
        "plain_fwd_frac": prf["fwd"]["frac"], "plain_bwd_frac": prf["bwd"]["frac"], "plain_units": prf["units"],
        "tuning": {"tile": tile, "spt": ctx_spt, "splits": "auto",
                   "chosen_by": "command line" if (args.tile and args.spt) else "mbr_autotune"},
        "paper_context": "paper: up to 4.57x fwd+grad speedup vs SoftRas on one RTX 4090 (different workload, "
                         "linear translation, Sec. 4.2)",
    }
    # ---- the translation scene at the headline's size (the paper's speed comparison uses linear
    # translation): same mesh, d = 1.5 perpendicular to the view, T = 64, 256^2, one segment
    tsc = Scene(scenes.config2_translate())
    tr = {"workload": "translation: the rotation workload's mesh moved by d = (1.5, 0, 0), T=64, 256x256, S=1"}
    for solver in ("fast", "plain"):
        fb_ms, fb_st = tsc.timed(solver, True, k2, 2)
        fb_ms /= k2
        fw_ms, fw_st = tsc.timed(solver, False, k2, 2)
        fw_ms /= k2
        fr = tsc.fracs(solver, fb_st, peak)
        tr[solver] = {"fwdbwd_ms": fb_ms, "fwdbwd_samples_per_s": world * tsc.n / (fb_ms / 1e3),
                      "fwdbwd_iters_per_s": 1e3 / fb_ms, "fwd_ms": fw_ms,
                      "fwd_samples_per_s": world * tsc.n / (fw_ms / 1e3),
                      "raster_fwd_ms": fr["fwd"]["raster_ms"], "raster_bwd_ms": fr["bwd"]["raster_ms"],
                      "fwd_frac": fr["fwd"]["frac"], "bwd_frac": fr["bwd"]["frac"], "units": fr["units"]}
    tr["speedup_fast_over_plain_fwdbwd"] = tr["plain"]["fwdbwd_ms"] / tr["fast"]["fwdbwd_ms"]
    tr["speedup_fast_over_plain_fwd"] = tr["plain"]["fwd_ms"] / tr["fast"]["fwd_ms"]
    extras["translate"] = tr
    # ---- config 1 (64^2, T = 16, translation): forward only, plain vs fast
    c1 = Scene(scenes.config1())
    c1r = {"workload": "icosphere subdiv 2 + jitter, d = (1.5, 0, 0), T=16, 64x64, forward only"}
    for solver in ("fast", "plain"):
        ms1, _ = c1.timed(solver, False, k2, 2)
        c1r[solver] = {"fwd_ms": ms1 / k2, "samples_per_s": world * c1.n / (ms1 / k2 / 1e3)}
    c1r["speedup_fast_over_plain_fwd"] = c1r["plain"]["fwd_ms"] / c1r["fast"]["fwd_ms"]
    extras["c1_forward"] = c1r

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

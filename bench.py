#!/usr/bin/env python3
"""Meshing-iteration throughput of the GB300 path on the million-point annulus.

Workload: annulus 0.3 <= r <= 1 on a 1024^2 FP32 SDF grid, adaptive sizing
h = 0.002 + 0.05|sdf| on a 512^2 grid, 10^6 points drawn by rejection
sampling with density proportional to 1/h^2 (seed 1), hybrid method
(DistMesh then CVD), FP64 positions.  One step = one meshing iteration
(bucketing, Voronoi cells, triangle emission and validity, quality, move,
point treatment) over all points.

    python bench.py [--gpus N --steps K --warmup W] [--impl reference] [--no-extras] [--no-sweep] [--no-cpu]

Prints one JSON line (rank 0).  N > 1 runs N independent replicas, one per
GPU (the meshes do not exchange data), and reports their aggregate.
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mpoints/s per meshing iteration at 1e6 pts; wall time to quality at 1e6 pts"
WORKLOAD = ("annulus r in [0.3,1], 1024^2 FP32 SDF, sizing 0.002+0.05|sdf| on 512^2, "
            "1e6 points ~ 1/h^2 (seed 1), hybrid DistMesh->CVD")
VORONOI_FLOP_PER_CELL = 2500.0  # algorithmic flops of one cell's clipping: ~30 distance tests, ~8 cuts, ~60 predicates
L2_FLUSH_BYTES = 256 << 20
# FP64 mode keeps every decision (emission, validity, predicates' filters,
# point treatment) in FP64 and evaluates the moves' sums in float-float
# (pairs of f32, ~48 bits); FP32 mode holds positions, forces and centroids in
# f32 with the same FP64/exact decisions
DTYPE = {0: "f64 decisions, float-float (2xf32) moves", 1: "f32 positions, f64/exact decisions"}
PRECISION = {0: "fp64 decisions, float-float moves", 1: "fp32 positions, fp64/exact predicates"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--points", type=int, default=1_000_000)
    ap.add_argument("--precision", type=int, default=0)
    ap.add_argument("--method", type=int, default=2)
    ap.add_argument("--no-extras", action="store_true", help="skip the legs beyond the headline iteration")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--n-opt", type=float, default=None, help="points per neighbour bucket (default 3.3)")
    ap.add_argument("--no-sweep", action="store_true",
                    help="skip the N sweep (annulus 1e4..1e7, square 1e6) and the 1e7-point star")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region: rows
    every 20 ms carry nvidia-smi's own timestamp, and only the rows inside
    the window marked by mark_start()/mark_stop() count (the rows nearest to
    it when the window is shorter than the sampling period)."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    PERIOD_MS = 20

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.f = None
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", str(self.PERIOD_MS)],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
            # nvidia-smi's start-up (driver queries) must be over before the
            # timed region: wait for its first rows (at most 10 s)
            t_end = time.time() + 10.0
            while time.time() < t_end and self.proc.poll() is None:
                if os.path.getsize(self.f.name) > 0 and open(self.f.name).read().count("\n") >= 3:
                    break
                time.sleep(0.05)
        except Exception:
            self.proc = None

    def mark_start(self):
        self.t0 = time.time()

    def mark_stop(self):
        self.t1 = time.time()

    @staticmethod
    def parse(rows, t0=None, t1=None):
        """Median SM clock, max clock and active throttle reasons of the rows
        (lists of fields) whose timestamp lies in [t0, t1]."""
        import datetime

        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        recs = []
        for r in rows:
            try:
                ts = datetime.datetime.strptime(r[0].strip(), "%Y/%m/%d %H:%M:%S.%f").timestamp()
                recs.append((ts, float(r[2]), float(r[3]),
                             [n for k, n in enumerate(names) if r[6 + k].strip().lower() == "active"]))
            except (ValueError, IndexError):
                continue
        if t0 is not None and t1 is not None and recs:
            inside = [x for x in recs if t0 <= x[0] <= t1]
            if not inside:  # a window shorter than the period: the nearest row on each side
                before = [x for x in recs if x[0] < t0]
                after = [x for x in recs if x[0] > t1]
                inside = before[-1:] + after[:1]
            recs = inside
        sm = [x[1] for x in recs]
        reasons = sorted({n for x in recs for n in x[3]})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(x[2] for x in recs) if recs else None,
                "reasons": reasons, "samples": len(sm)}

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(2 * self.PERIOD_MS / 1e3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.strip().split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        out = self.parse(rows, self.t0, self.t1)
        out["period_ms"] = self.PERIOD_MS
        return out


# ------------------------------------------------------------------ helpers
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return json.load(f)
    except Exception:
        return {}


def committed_profile(kernel_src, points=1_000_000):
    """DRAM bytes and warp instructions per launch of the Voronoi kernel from
    the committed ncu summary; both None if the kernel source changed since
    it was captured or the workload has another size."""
    import hashlib

    path = os.path.join(ROOT, "profiles", "voronoi_annulus_1e6.md")
    try:
        txt = open(path).read()
    except OSError:
        return None, None
    digest = hashlib.sha256(open(kernel_src, "rb").read()).hexdigest()[:16]
    tr, wi, hs = None, None, None
    for line in txt.splitlines():
        if line.startswith("traffic_bytes_per_launch:"):
            tr = float(line.split(":")[1])
        if line.startswith("warp_instructions_per_launch:"):
            wi = float(line.split(":")[1])
        if line.startswith("voronoi_cuh_sha256_16:"):
            hs = line.split(":")[1].strip()
    return (tr, wi) if hs == digest and points == 1_000_000 else (None, None)


def flush_l2(buf):
    buf.fill_(1)


def replica_value(points_per_rank, steps, local_seconds, dist=None, device="cpu"):
    """Aggregate throughput of independent replicas: all ranks' points x steps
    over the slowest rank's time (max over ranks).  Returns (Mpts/s, max s)."""
    import torch

    world = 1
    t = local_seconds
    if dist is not None and dist.is_initialized():
        world = dist.get_world_size()
        x = torch.tensor([local_seconds], dtype=torch.float64, device=device)
        dist.all_reduce(x, op=dist.ReduceOp.MAX)
        t = float(x.item())
    return points_per_rank * world * steps / t / 1e6, t


def oracle_sample_rate(wl, target_s, max_cells=None, threads=1, om=None):
    """Oracle per-cell iteration work (cell clipping, owned triangles with
    Tests 1-3, CVD centroid) on a random sample of cells sized to take about
    target_s seconds; threads > 1 spreads the cells over OpenMP threads.
    Returns (cells, seconds, oracle mesh)."""
    import oracle

    oracle.build()
    if om is None:
        om = oracle.OracleMesh(wl.sdf, wl.sizing, wl.points, method=wl.method)
    n = len(wl.points)
    rng = np.random.default_rng(123)

    def work(cells):
        if threads > 1:
            om.rebuild_sample_mt(cells, True, threads)
        else:
            om.rebuild_sample(cells, True)

    probe = rng.choice(n, min(n, 4000 * threads), replace=False)
    t = time.perf_counter()
    work(probe)
    per = (time.perf_counter() - t) / len(probe)
    cnt = int(min(n if max_cells is None else max_cells, max(len(probe), target_s / per)))
    cells = rng.choice(n, cnt, replace=False)
    t = time.perf_counter()
    work(cells)
    return cnt, time.perf_counter() - t, om


def oracle_iterations(wl, threads, steps, om=None):
    """Full oracle meshing iterations (om_step: bucketing, every cell's clip,
    emission with Tests 1-3, quality, hybrid switch, DistMesh forces or CVD
    centroids, point treatment) of the whole workload, the per-cell loops on
    `threads` OpenMP threads.  Returns (seconds per iteration list, oracle
    mesh); the mesh carries on along its own trajectory."""
    import oracle

    oracle.build()
    if om is None:
        om = oracle.OracleMesh(wl.sdf, wl.sizing, wl.points, method=wl.method)
    om.set_threads(threads)
    times = []
    for _ in range(steps):
        t = time.perf_counter()
        om.step()
        times.append(time.perf_counter() - t)
    return times, om


def run_reference(args, wl):
    """The oracle as the reference arm: each step is one full FP64 meshing
    iteration of the whole workload on all host cores."""
    world, rank, local = dist_env()
    if rank != 0:
        return
    threads = os.cpu_count() or 1
    _, om = oracle_iterations(wl, threads, args.warmup)
    times, om = oracle_iterations(wl, threads, args.steps, om)
    n = len(wl.points)
    v = n * args.steps / sum(times) / 1e6
    sample = (f"full meshing iterations of the {n}-point workload (FP64 oracle om_step: cells, emission with "
              f"Tests 1-3, quality, hybrid switch, move, point treatment), per-cell loops on {threads} OpenMP "
              f"threads, iterations {args.warmup + 1}..{args.warmup + args.steps} of the trajectory")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "Mpts/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "points": n},
            "cpu_baseline": {"value": v, "unit": "Mpts/s", "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "Mpts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def batched_leg(g, torch, stream, steps, flush):
    """256 independent star meshes stepped as one batch (one launch per
    stage, autotuned tiling) against the same meshes stepped one mesh handle
    after another, plus the batch's wall time until every mesh terminates."""
    import workloads as W

    wl = W.star_batch_workload(workers=min(16, os.cpu_count() or 1), precision=1)
    meshes = [(s, z, W.to_fp32_positions(p)) for s, z, p in wl.meshes]
    npts = wl.total_points
    t0 = time.perf_counter()
    b = g.MeshBatch(meshes, stream=stream.cuda_stream, autotune=True, precision=1, method=2)
    init_s = time.perf_counter() - t0
    tun = b.tuning()

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for k in range(steps):
            flush_l2(flush)
            evs[k][0].record(stream)
            fn()
            evs[k][1].record(stream)
        torch.cuda.synchronize()
        return sum(a.elapsed_time(c) for a, c in evs) / steps

    ms_b = timed(lambda: b.step_async(1))
    b.close()
    singles = [g.Mesh(s, z, p, precision=1, method=2, stream=stream.cuda_stream) for s, z, p in meshes]

    def step_all():
        for m in singles:
            m.step_async(1)

    ms_s = timed(step_all)
    for m in singles:
        m.close()
    q = g.MeshBatch(meshes, stream=stream.cuda_stream, autotune=False, precision=1, method=2)
    q.set_tuning(tun["n_opt"], tun["lanes"])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = q.step(2000)
    torch.cuda.synchronize()
    tq = time.perf_counter() - t0
    q.close()
    sizes = [len(m[2]) for m in meshes]
    return {"workload": f"{len(meshes)} random star polygons (50-300 vertices), 512^2 FP32 SDF each, sizing "
                        f"0.002+0.05|sdf|, points log-uniform in [1e3,1e5] (total {npts}), uniform seeding, "
                        f"hybrid, FP32 positions",
            "meshes": len(meshes), "points": npts, "min_points": min(sizes), "max_points": max(sizes),
            "value": npts / (ms_b / 1e3) / 1e6, "unit": "Mpts/s", "ms_per_step": ms_b,
            "one_mesh_at_a_time": {"value": npts / (ms_s / 1e3) / 1e6, "unit": "Mpts/s", "ms_per_step": ms_s},
            "tuning": {"n_opt": tun["n_opt"], "lanes": tun["lanes"],
                       "candidates_ms": [[c[0], c[1], c[2]] for c in tun["candidates"]],
                       "init_seconds_with_autotune": init_s},
            "time_to_quality": {"seconds": tq, "all_terminated": all(x["terminated"] for x in st),
                                "max_iterations": max(x["iterations"] for x in st),
                                "min_angle_deg_worst": min(x["min_angle_deg"] for x in st if x["n_tri"] > 0),
                                "max_alpha_worst": max(x["max_alpha"] for x in st)}}


def device_rate(g, torch, stream, flush, sdf, siz, pts, steps, **params):
    """Device time of `steps` iterations of a fresh mesh (L2 flushed before
    each), after 3 warm-up iterations; returns (Mpts/s, ms per step)."""
    m = g.Mesh(sdf, siz, pts, stream=stream.cuda_stream, **params)
    for _ in range(3):
        m.step_async(1)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        flush_l2(flush)
        evs[k][0].record(stream)
        m.step_async(1)
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in evs) / steps
    m.close()
    return len(pts) / (ms / 1e3) / 1e6, ms


def sweep_leg(g, torch, stream, steps, flush):
    """Throughput over problem sizes (the annulus at 1e4..1e7 points, FP64
    hybrid; the uniform square at 1e6) and the 1e7-point star polygon (FP32
    positions, hybrid) with its wall time to quality."""
    import workloads as W

    out = {"annulus_fp64_hybrid": []}
    for n in (10_000, 100_000, 10_000_000):
        wl = W.annulus_workload(n=n)
        v, ms = device_rate(g, torch, stream, flush, wl.sdf, wl.sizing, wl.points, steps, method=2)
        out["annulus_fp64_hybrid"].append({"points": n, "value": v, "unit": "Mpts/s", "ms_per_step": ms})
    wl = W.square_workload(1_000_000)
    v, ms = device_rate(g, torch, stream, flush, wl.sdf, wl.sizing, wl.points, steps, method=2)
    out["square_fp64_hybrid"] = {"points": 1_000_000, "value": v, "unit": "Mpts/s", "ms_per_step": ms}
    wl = W.star_workload(10_000_000, workers=min(16, os.cpu_count() or 1))
    p32 = W.to_fp32_positions(wl.points)
    v, ms = device_rate(g, torch, stream, flush, wl.sdf, wl.sizing, p32, steps, method=2, precision=1)
    m = g.Mesh(wl.sdf, wl.sizing, p32, method=2, precision=1, stream=stream.cuda_stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s = m.step(2000)
    torch.cuda.synchronize()
    tq = time.perf_counter() - t0
    m.close()
    out["star500_fp32_hybrid_1e7"] = {
        "workload": "star polygon, 500 vertices (radii U[0.4,1], seed 2), 4096^2 FP32 SDF, curvature-adaptive "
                    "sizing in [2e-4,1e-2] on 1024^2, 1e7 points ~ 1/h^2, FP32 positions, hybrid",
        "value": v, "unit": "Mpts/s", "ms_per_step": ms,
        "time_to_quality": {"seconds": tq, "iterations": s["iterations"], "terminated": bool(s["terminated"]),
                            "min_angle_deg": s["min_angle_deg"], "half_mean_alpha": s["half_mean_alpha"],
                            "max_alpha": s["max_alpha"], "n_tri": s["n_tri"]}}
    return out


def segment_sdf_leg(g, torch, stream):
    """The SDF of the benchmark star (500 clockwise segments) on its 4096^2
    grid, built on the device (mesh_segment_sdf_grid, into device memory;
    device time by CUDA events, best of 3) against the host builder of the
    workloads (a sampled nearest-segment search in numpy, all cores) and the
    oracle's brute force on a sample of nodes (one core)."""
    import workloads as W

    v = W.star_polygon(500, 0.4, 1.0, 2)
    n = 4096
    out = torch.empty((n, n), dtype=torch.float32, device="cuda")
    g.segment_sdf_grid(v, n, out=out, stream=stream.cuda_stream)  # warm-up
    best = None
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.segment_sdf_grid(v, n, out=out, stream=stream.cuda_stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    t0 = time.perf_counter()
    W.polygon_sdf_grid(v, n, workers=min(16, os.cpu_count() or 1))
    host_s = time.perf_counter() - t0
    import oracle

    oracle.build()
    rng = np.random.default_rng(0)
    px, py = rng.uniform(-1.1, 1.1, 20000), rng.uniform(-1.1, 1.1, 20000)
    t0 = time.perf_counter()
    oracle.segment_sdf(v, px, py)
    rate_or = 20000 / (time.perf_counter() - t0)
    return {"nodes": n * n, "segments": len(v), "device_ms": best, "device_mnodes_per_s": n * n / best / 1e3,
            "host_builder_seconds": host_s, "host_builder_workers": min(16, os.cpu_count() or 1),
            "oracle_mnodes_per_s_1_core": rate_or / 1e6,
            "note": "device time includes its scratch allocation and the cell candidate search"}


def adf_measure(g, torch, m, v, sg):
    """The mesh's adaptive distance field (Sec. 3.7: its boundary cells,
    E_tol = 0.1 geps_i, depth 10): build time, nodes, evaluation rate at 10^6
    points of the boundary cells (device buffers, CUDA events) and its error
    against the exact segment SDF at 10^5 of them, beside the error of the
    float32 grid the mesh samples."""
    import workloads as W

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    a = g.ADF.for_mesh(m, v, sg, fac_etol=0.1, max_depth=10)
    t_build = time.perf_counter() - t0
    nodes, levels = a.size()
    rng = np.random.default_rng(11)
    nx = sg.values.shape[1]
    d = (sg.x1 - sg.x0) / (nx - 1)
    c = a.cells[rng.integers(0, len(a.cells), 1_000_000)]
    p = np.stack([sg.x0 + (c % (nx - 1) + rng.random(len(c))) * d, sg.y0 + (c // (nx - 1) + rng.random(len(c))) * d],
                 1)
    pd = torch.from_numpy(p).cuda()
    out = torch.empty(len(p), dtype=torch.float64, device="cuda")
    a.eval(pd, out=out)  # warm-up
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    cur = torch.cuda.current_stream()
    e0.record(cur)
    a.eval(pd, out=out, stream=cur.cuda_stream)
    e1.record(cur)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    k = 100_000
    exact = g.segment_sdf_points(v, p[:k])
    adf = out[:k].cpu().numpy()
    grid = W._bilinear_np(sg, p[:k, 0], p[:k, 1])
    res = {"build_seconds": t_build, "boundary_cells": int(len(a.cells)), "nodes": int(nodes), "levels": int(levels),
           "tol_median": float(np.median(a.tol)), "eval_ms_1e6": ms, "eval_mpts_per_s": 1e3 / ms,
           "max_error": float(np.abs(adf - exact).max()), "mean_error": float(np.abs(adf - exact).mean()),
           "grid_max_error": float(np.abs(grid - exact).max()), "grid_mean_error": float(np.abs(grid - exact).mean())}
    a.close()
    return res


def polygon_leg(g, torch, stream):
    """From a polygon to a mesh with the initialisation pipeline (segment SDF,
    automatic sizing, dithered initial points): the benchmark star (500 clockwise segments) -> its SDF grid and
    automatic sizing field on 1024^2 (App. A, Sec. 3.3, Eq. 7, K = 0.1) ->
    10^6 dithered initial points (Sec. 3.5) -> hybrid meshing (FP32 positions)
    until termination.  Host clock around synchronous calls."""
    import workloads as W

    v = W.star_polygon(500, 0.4, 1.0, 2)
    n, box = 1024, (-1.1, -1.1, 1.1, 1.1)
    t0 = time.perf_counter()
    sdf, mu, counts = g.auto_sizing(v, 0.1, n, box)
    t_auto = time.perf_counter() - t0
    sg, zg = W.Grid(sdf, *box), W.Grid(mu, *box)
    t0 = time.perf_counter()
    pts = g.init_points(sg, zg, 1_000_000, seed=1)
    t_init = time.perf_counter() - t0
    out = {"auto_sizing_seconds": t_auto, "samples": counts["samples"], "medial_points": counts["medial"],
           "medial_kept": counts["kept"], "sizing_min": float(mu.min()), "sizing_max": float(mu.max()),
           "init_points_seconds": t_init, "points": len(pts)}
    try:
        m = g.Mesh(sg, zg, W.to_fp32_positions(pts), method=2, precision=1, stream=stream.cuda_stream)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s = m.step(2000)
        torch.cuda.synchronize()
        out.update({"meshing_seconds": time.perf_counter() - t0, "iterations": s["iterations"],
                    "terminated": bool(s["terminated"]), "min_angle_deg": s["min_angle_deg"],
                    "max_alpha": s["max_alpha"], "half_mean_alpha": s["half_mean_alpha"]})
        out["adf"] = adf_measure(g, torch, m, v, sg)
        m.close()
    except g.MeshError as e:
        out["meshing_error"] = str(e)
    return out


def distmesh_leg(g, torch, stream):
    """The DistMesh method (config 1's disk at 1e4 points and the annulus at
    1e6) to termination, re-triangulating every iteration and only after large
    movements (Algorithm 1, fac_retria = 0.1)."""
    import workloads as W

    out = {}
    for name, wl in (("disk_1e4", W.disk_workload(n=10000)), ("annulus_1e6", W.annulus_workload(n=1_000_000))):
        rec = {}
        for fac in (0.0, 0.1):
            m = g.Mesh(wl.sdf, wl.sizing, wl.points, method=0, fac_retria=fac, stream=stream.cuda_stream)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s = m.step(2000)
            torch.cuda.synchronize()
            rec[f"fac_retria_{fac}"] = {"seconds": time.perf_counter() - t0, "iterations": s["iterations"],
                                        "triangulations": s["triangulations"], "terminated": bool(s["terminated"]),
                                        "min_angle_deg": s["min_angle_deg"], "half_mean_alpha": s["half_mean_alpha"],
                                        "max_alpha": s["max_alpha"]}
            m.close()
        out[name] = rec
    return out


_STAR = {}


def star_1e6():
    """The star polygon with 10^6 points (2048^2 SDF, 512^2 sizing), built once."""
    import workloads as W

    if "w" not in _STAR:
        _STAR["w"] = W.star_workload(1_000_000, sdf_n=2048, siz_n=512, workers=min(16, os.cpu_count() or 1))
    return _STAR["w"]


def addition_leg(g, torch, stream):
    """Point addition (Sec. 3.6) against initialising all points, the paper's
    comparison on its complicated shape: the star with N_total = 10^6, hybrid,
    FP32 positions, from fac_init N_total = 2 x 10^5 seeds (the first points of
    the same density sample) or all 10^6, until termination.  Also the device
    time of one addition at that size (10^6 -> 1.6 x 10^6 points)."""
    import workloads as W

    star = star_1e6()
    p32 = W.to_fp32_positions(star.points)
    out = {}
    for name, pts, kw in (("point_addition", p32[:200_000], {"n_total": 1_000_000}), ("init_all", p32, {})):
        m = g.Mesh(star.sdf, star.sizing, pts, method=2, precision=1, stream=stream.cuda_stream, **kw)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        added = iters = 0
        seq = []
        for _ in range(200):
            s = m.step(20)
            iters += s["iterations"]
            if s["added"]:
                added += s["added"]
                seq.append([iters, s["n_points"]])
            if s["terminated"] or s["iterations"] == 0:
                break
        torch.cuda.synchronize()
        out[name] = {"seconds": time.perf_counter() - t0, "iterations": iters, "terminated": bool(s["terminated"]),
                     "n_points": s["n_points"], "points_added": added,
                     "iterations_and_n_after_calls_that_added": seq,
                     "min_angle_deg": s["min_angle_deg"], "max_alpha": s["max_alpha"],
                     "half_mean_alpha": s["half_mean_alpha"], "n_tri": s["n_tri"]}
        m.close()
    # one addition on its own: forced at the second iteration (T_add above any change)
    m = g.Mesh(star.sdf, star.sizing, p32, method=2, precision=1, n_total=1_600_000, T_add=1e9,
               stream=stream.cuda_stream)
    m.step(1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s = m.step(1)
    torch.cuda.synchronize()
    t_add = time.perf_counter() - t0
    t0 = time.perf_counter()
    m.step(1)
    torch.cuda.synchronize()
    out["one_addition"] = {"points_before": 1_000_000, "points_added": s["added"],
                           "seconds_addition_call": t_add, "seconds_next_iteration": time.perf_counter() - t0,
                           "note": "host clock around synchronous calls; the addition call includes its "
                                   "triangulating iteration, the selection and the graph re-capture"}
    m.close()
    return out


def learned_leg(g, stream):
    """The learned displacement model: trained on the device on trajectories of
    the disk (DistMesh, 1e4 points) and the benchmark annulus (hybrid, 1e6),
    then the wall time of the hybrid method with and without its proposals to
    the plain method's converged minimum angle minus 1 degree, on the annulus
    drawn with four seeds (the first is the benchmark's), and both forms run
    to termination on the 1e6-point star."""
    import workloads as W
    from paper_2309_13824_gb300 import learn

    disk = W.disk_workload(n=10000)
    anns = {sd: W.annulus_workload(n=1_000_000, seed=sd) for sd in (1, 2, 3, 4)}
    st = stream.cuda_stream
    t0 = time.perf_counter()
    net, loss, npairs = learn.train([(disk.sdf, disk.sizing, disk.points, 0, 0),
                                     (anns[1].sdf, anns[1].sizing, anns[1].points, 2, 0)], stream=st)
    out = {"training": {"pairs": npairs, "last_epoch_loss": loss, "seconds": time.perf_counter() - t0,
                        "trajectories": "disk 1e4 DistMesh FP64 (seed 0) + annulus 1e6 hybrid FP64 (seed 1), "
                                        "pairs every 11 iterations, horizon 10, 40+10 epochs Adam"},
           "policy": {"every": 5, "jump": 5.0, "min_angle_tol": 0.5, "max_proposals": 8,
                      "judge": "proposal branch kept only if it beats the plain iteration from the same state"}}

    def rec(t, s):
        if t is None:
            return dict(s)
        r = {"seconds": t, "iterations": s["iterations"], "target_reached": bool(s["target_reached"]),
             "min_angle_deg": s["min_angle_deg"], "half_mean_alpha": s["half_mean_alpha"],
             "max_alpha": s["max_alpha"], "mean_size_dev": s["mean_size_dev"]}
        if "accepted" in s:
            r.update({"proposals_kept": s["accepted"], "proposals_undone": s["rejected"]})
        return r

    def guarded(wl, pts, prec, **kw):
        try:
            return learn.time_to_quality(wl.sdf, wl.sizing, pts, precision=prec, stream=st, **kw)
        except g.MeshError as e:  # reported, not fatal to the benchmark
            return None, {"error": str(e)}

    seeds = []
    tot_p = tot_l = 0.0
    wins = 0
    for sd, wl in anns.items():
        tc, conv = guarded(wl, wl.points, 0)
        q = conv["min_angle_deg"] - 1.0
        tp, sp = guarded(wl, wl.points, 0, target=q)
        tl, sl = guarded(wl, wl.points, 0, net=net, target=q)
        seeds.append({"seed": sd, "target_min_angle_deg": q, "plain_converged": rec(tc, conv),
                      "plain_to_target": rec(tp, sp), "learned_to_target": rec(tl, sl)})
        if tp is not None and tl is not None:
            tot_p += tp
            tot_l += tl
            wins += tl < tp
    out["annulus_1e6_fp64"] = {"seeds": seeds, "plain_to_target_seconds_total": tot_p,
                               "learned_to_target_seconds_total": tot_l, "learned_faster_on": wins}
    star = star_1e6()
    p32 = W.to_fp32_positions(star.points)
    out["star500_1e6_fp32"] = {"plain_converged": rec(*guarded(star, p32, 1)),
                               "learned_converged": rec(*guarded(star, p32, 1, net=net))}
    out["batched_annuli_4x250k_fp64"] = batched_learned(g, net)
    return out


def batched_learned(g, net):
    """The batched form with the learned part at 10^6 points: four annuli of
    2.5 x 10^5 points (seeds 5-8) stepped as one batch; each mesh's target is
    the plain batch's converged minimum angle minus 1 degree; wall time (host
    clock around synchronous calls) of the plain batch and of the learned
    batch to every mesh's target."""
    import torch

    import workloads as W

    meshes = []
    for sd in (5, 6, 7, 8):
        wl = W.annulus_workload(n=250_000, seed=sd)
        meshes.append((wl.sdf, wl.sizing, wl.points))
    conv = g.MeshBatch(meshes, method=2, autotune=False).step(2000)
    targets = [c["min_angle_deg"] - 1.0 for c in conv]
    res = {"points": sum(len(m[2]) for m in meshes), "meshes": len(meshes),
           "targets_min_angle_deg": targets,
           "policy": {"every": 5, "jump": 5.0, "min_angle_tol": 0.5, "max_rounds": 8}}
    for name in ("plain", "learned"):
        b = g.MeshBatch(meshes, method=2, autotune=False)
        for k, q in enumerate(targets):
            b.set_quality_target(q, mesh=k)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = b.step(2000) if name == "plain" else b.step_learned(net, 2000, max_rounds=8)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        res[name] = {"seconds": dt, "all_reached": all(x["target_reached"] for x in st),
                     "iterations": [x["iterations"] for x in st],
                     "min_angle_deg": [x["min_angle_deg"] for x in st],
                     "max_alpha": [x["max_alpha"] for x in st]}
        if name == "learned":
            res[name]["proposals_kept"] = [x["accepted"] for x in st]
            res[name]["proposals_undone"] = [x["rejected"] for x in st]
        b.close()
    return res


def main():
    args = parse()
    world, rank, local = dist_env()
    import workloads as W

    wl = W.annulus_workload(n=args.points, method=args.method, precision=args.precision)
    if args.impl == "reference":
        return run_reference(args, wl)

    import torch

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_2309_13824_gb300 as g

    if not g.LIB_PATH.exists():
        g.build()
    g.lib()
    n = len(wl.points)
    pts = wl.points if args.precision == 0 else W.to_fp32_positions(wl.points)
    stream = torch.cuda.current_stream()
    kw = {} if args.n_opt is None else {"N_opt": args.n_opt}
    mesh = g.Mesh(wl.sdf, wl.sizing, pts, method=args.method, precision=args.precision,
                  stream=stream.cuda_stream, **kw)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    for _ in range(max(3, args.warmup)):
        mesh.step_async(1)
    torch.cuda.synchronize()

    # ---- timed region: K iterations, L2 flushed before each, device events
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.mark_start()
    for k in range(args.steps):
        flush_l2(flush)
        ev[k][0].record(stream)
        mesh.step_async(1)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    clocks.mark_stop()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_s = sum(step_ms) / 1e3
    step_stats = {"median_ms": float(np.median(step_ms)), "min_ms": float(min(step_ms)),
                  "max_ms": float(max(step_ms)), "mean_ms": float(np.mean(step_ms))}
    st = mesh.step(0)
    value, total_s = replica_value(n, args.steps, total_s, dist, device="cuda")

    # ---- per-stage device times (roofline of the dominant kernel)
    pm = g.Mesh(wl.sdf, wl.sizing, pts, method=args.method, precision=args.precision, stream=stream.cuda_stream,
                **kw)
    pm.profile(2)
    prof = pm.profile(args.steps)
    stage_ms = {k: v / args.steps for k, v in prof.items()}
    pm.close()
    t_vor = stage_ms["voronoi"] / 1e3
    peaks = measured_peaks()
    sm_count = torch.cuda.get_device_properties(local).multi_processor_count
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    alu_peak = sm_count * 128 * 2 * sm_mhz * 1e6 / 1e12  # FP32 FMA issue, TFLOP/s
    achieved = VORONOI_FLOP_PER_CELL * n / t_vor / 1e12
    pipe = g.mesh_measure_pipe_peaks()
    src = os.path.join(ROOT, "paper_2309_13824_gb300", "csrc", "voronoi.cuh")
    traffic, winst = committed_profile(src, n)
    roofline = {"bound": "alu", "kernel": "k_voronoi", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                "frac": achieved / alu_peak, "traffic": traffic,
                "peak_note": f"{sm_count} SMs x 128 FP32 lanes x 2 x {sm_mhz:.0f} MHz (unit counts and clocks)",
                "stage_ms": stage_ms, "measured_pipe_peaks": pipe}
    if winst:
        # the kernel is bound by instruction issue, not by FP32 arithmetic:
        # its ncu warp-instruction count against one instruction per
        # scheduler per clock (4 per SM), over the live Voronoi stage time
        ipk = sm_count * 4 * sm_mhz * 1e6
        roofline["issue"] = {"warp_instructions_per_launch": winst, "achieved_per_s": winst / t_vor,
                             "peak_per_s": ipk, "frac": winst / t_vor / ipk,
                             "note": "instructions of k_voronoi from the committed ncu capture; time of the whole "
                                     "Voronoi stage (the wider passes included)"}

    # ---- end to end through the C ABI: each step uploads the positions from
    # pinned host memory (the previous step's result), runs one iteration and
    # reads the moved positions back into pinned host memory
    e2e = None
    if rank == 0 or world > 1:
        em = g.Mesh(wl.sdf, wl.sizing, pts, method=args.method, precision=args.precision,
                    stream=stream.cuda_stream, **kw)
        dt_np = np.float64 if args.precision == 0 else np.float32
        bufs = [torch.from_numpy(np.ascontiguousarray(pts, dtype=dt_np)).pin_memory() for _ in range(2)]
        em.step(args.warmup)  # the same phase of the trajectory as the device-timed steps
        em.points(out=bufs[0])
        for k in range(2):
            em.set_state(bufs[k % 2].numpy())
            em.step(1)
            em.points(out=bufs[(k + 1) % 2])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(args.steps):
            em.set_state(bufs[k % 2].numpy())
            em.step(1)
            em.points(out=bufs[(k + 1) % 2])
        torch.cuda.synchronize()
        e_s = time.perf_counter() - t0
        nbytes = n * 2 * bufs[0].element_size()
        e2e = {"value": n * args.steps / e_s / 1e6, "unit": "Mpts/s", "h2d_bytes_per_step": nbytes,
               "d2h_bytes_per_step": nbytes}
        em.close()

    extras = {}
    if not args.no_sweep and not args.no_extras and rank == 0:
        extras["sweep"] = sweep_leg(g, torch, stream, args.steps, flush)
    if not args.no_extras and rank == 0:
        # wall time to quality: hybrid from the seeds until termination
        tq = g.Mesh(wl.sdf, wl.sizing, pts, method=2, precision=args.precision, stream=stream.cuda_stream, **kw)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s = tq.step(2000)
        torch.cuda.synchronize()
        extras["time_to_quality"] = {"seconds": time.perf_counter() - t0, "iterations": s["iterations"],
                                     "terminated": bool(s["terminated"]), "min_angle_deg": s["min_angle_deg"],
                                     "half_mean_alpha": s["half_mean_alpha"], "max_alpha": s["max_alpha"],
                                     "mean_size_dev": s["mean_size_dev"], "n_tri": s["n_tri"]}
        # the paper's table of the mesh at termination (quality report of the last rebuild)
        q = tq.quality()
        extras["time_to_quality"]["quality_report"] = {
            k: q[k] for k in ("median_alpha", "mean_alpha", "max_alpha", "std_alpha", "median_beta", "mean_beta",
                              "max_beta", "std_beta", "frac_alpha_lt_1_2", "frac_alpha_lt_2", "min_angle_deg",
                              "alpha_hist", "mean_size_dev", "p95_size_dev")}
        tq.close()
        # FP32-position mode on the same workload
        if args.precision == 0:
            p32 = W.to_fp32_positions(wl.points)
            fm = g.Mesh(wl.sdf, wl.sizing, p32, method=args.method, precision=1, stream=stream.cuda_stream, **kw)
            for _ in range(3):
                fm.step_async(1)
            evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for _ in range(args.steps)]
            for k in range(args.steps):
                flush_l2(flush)
                evs[k][0].record(stream)
                fm.step_async(1)
                evs[k][1].record(stream)
            torch.cuda.synchronize()
            ms32 = sum(a.elapsed_time(b) for a, b in evs)
            extras["fp32_positions"] = {"value": n * args.steps / (ms32 / 1e3) / 1e6, "unit": "Mpts/s",
                                        "ms_per_step": ms32 / args.steps}
            fm.close()
        extras["batched"] = batched_leg(g, torch, stream, args.steps, flush)
        extras["learned"] = learned_leg(g, stream)
        extras["distmesh"] = distmesh_leg(g, torch, stream)
        extras["point_addition"] = addition_leg(g, torch, stream)
        extras["segment_sdf"] = segment_sdf_leg(g, torch, stream)
        extras["from_polygon"] = polygon_leg(g, torch, stream)
    if rank == 0 and world == 1 and not args.no_cpu:
        # the oracle on the host cores beside the device numbers (N = 1 only)
        threads = os.cpu_count() or 1
        n = len(wl.points)
        tm, om = oracle_iterations(wl, threads, 3)
        t1, _ = oracle_iterations(wl, 1, 1, om)
        cnt, dt, _ = oracle_sample_rate(wl, 5.0, threads=threads)
        extras["cpu_baseline"] = {
            "value": n * len(tm) / sum(tm) / 1e6, "unit": "Mpts/s", "cores": threads, "kind": "oracle",
            "sample": f"3 full meshing iterations (1-3) of the {n}-point workload: FP64 oracle om_step, per-cell "
                      f"loops on {threads} OpenMP threads ({sum(tm):.1f} s)",
            "value_1_thread": n / t1[0] / 1e6,
            "sample_1_thread": f"iteration 4 of the same trajectory on one thread ({t1[0]:.1f} s)",
            "per_cell_only": {"value": cnt / dt / 1e6, "unit": "Mpts/s",
                              "sample": f"{cnt} random cells: clip, owned triangles with Tests 1-3, CVD centroid "
                                        f"(no bucketing, sorting, quality, forces or treatment), {threads} threads"}}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "Mpts/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[args.precision],
                "data": "synthetic", "step_ms": step_stats,
                "config": {"workload": WORKLOAD, "points": n, "method": ["dm", "cvd", "hybrid"][args.method],
                           "precision": PRECISION[args.precision],
                           "l2": "flushed before every timed step (256 MB write)",
                           "parallelism": f"replicas x{world}"},
                "roofline": roofline, "e2e": e2e, "clocks": clk,
                "gpu_launches": 18 * args.steps,  # 17 kernels of the iteration graph + the counter reset
                "last_step": {"method": st["method"], "switched": st["switched"], "n_tri": st["n_tri"],
                              "half_mean_alpha": st["half_mean_alpha"]}}
        line.update(extras)
        print(json.dumps(line), flush=True)
    mesh.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

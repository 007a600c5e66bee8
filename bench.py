#!/usr/bin/env python3
"""Benchmark: Phi + grad Phi evaluations and the batched Newton chart solve
on the graded-torus workload (30,720 triangles, Duffy 6x6 sources =
1,105,920 nodes, 1e6 targets within 3 sigma, order-8 charts = 1,105,920
chart nodes), one GB300.

A step = one Phi/grad-Phi evaluation at the 1e6 targets + one chart solve
(all Newton sweeps) to |Phi - 1/2| < 1e-12: mixed-precision sweeps, then
float-float sweeps (Phi to FP64 accuracy on the FP32 pipes).  value = target evaluations per second over the step
(the targets plus every active chart node of every sweep), with inputs
resident on the device.  e2e = the same through the C ABI with host buffers
(pinned), the copies inside the timed region.  The dominant kernel's
roofline is measured live with CUDA events recorded by the library on its
launch stream.  The CPU baseline is the FP64 oracle on a bounded target
sample on this host's cores.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FLOPS_FAR_PAIR = 31              # Laplace double layer, Phi + grad (1 rsqrt not counted)
FLOPS_NEAR_PAIR = 60             # full smoothed kernel, Phi + grad (erfc, exp, rsqrt not counted)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64", "ff"],
                    help="precision of the evaluation (ff: with --no-charts only)")
    ap.add_argument("--tol", type=float, default=1e-12)
    ap.add_argument("--targets", type=int, default=None,
                    help="targets (torus: 1e6, icosphere: 2e7)")
    ap.add_argument("--order", type=int, default=8)
    ap.add_argument("--small", action="store_true", help="small torus (quick check)")
    ap.add_argument("--cells", default=None,
                    help="torus cells NUxNV (default 240x64); e.g. 120x32 for a profiling case")
    ap.add_argument("--workload", default="torus",
                    choices=["torus", "ellipsoids", "serve", "icosphere", "geometry"],
                    help="torus: the default line; ellipsoids: 512 meshes in one batched, graph-captured "
                         "solve; serve: a Poisson request stream through the server")
    ap.add_argument("--requests", type=int, default=200)
    ap.add_argument("--rate", type=float, default=5.0)
    ap.add_argument("--tmax", type=float, default=1e4)
    ap.add_argument("--serve-seconds", type=float, default=0.0,
                    help="serve: cut the stream at this wall time (cancel what is still queued)")
    ap.add_argument("--tree-degree", type=int, default=0, help="treecode degree (0: library default)")
    ap.add_argument("--tree-theta", type=float, default=0.0, help="treecode opening parameter (0: default)")
    ap.add_argument("--ff-block", type=int, default=0,
                    help="targets per CTA of the float-float kernel (64 or 128; 0: library default)")
    ap.add_argument("--mixed-block", type=int, default=0,
                    help="targets per CTA of the mixed kernel (64, 128 or 256; 0: the autotuner's choice)")
    ap.add_argument("--newton-tree-degree", type=int, default=0,
                    help="treecode degree of the mixed Newton sweeps (0: library default 5; -1: the mesh's own)")
    ap.add_argument("--newton-tree-theta", type=float, default=0.0,
                    help="opening parameter of the mixed Newton sweeps' treecode (0: library default 0.5)")
    ap.add_argument("--tree-cluster", type=int, default=0,
                    help="targets per target cluster of the mixed treecode (0: library default 4096; -1: off)")
    ap.add_argument("--newton-cutoff", type=float, default=0.0,
                    help="near-field radius in sigma of the mixed Newton sweeps (0: library default 5.0)")
    ap.add_argument("--tree-grid", type=int, default=0,
                    help="proxy grids: 1 per-axis point counts (default), 2 full (degree + 1)^3")
    ap.add_argument("--sigma-x", action="store_true",
                    help="target-dependent sigma(x) (eq. sigma2, lambda 2.5) instead of per-triangle sigma")
    ap.add_argument("--no-charts", action="store_true", help="time the evaluation only")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-geometry", action="store_true",
                    help="skip the untimed Gauss flux and Gauss-Bonnet checks after the step (profiling runs)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--fp64-check", type=int, default=0,
                    help="icosphere: also compare with the FP64 direct sum on this many targets")
    ap.add_argument("--no-tune", action="store_true", help="ellipsoids: skip the batch autotuner")
    ap.add_argument("--no-unbatched", action="store_true", help="ellipsoids: skip the mesh-by-mesh comparison")
    ap.add_argument("--no-paths", action="store_true",
                    help="skip the float-float and FP64 path legs after the timed region")
    ap.add_argument("--replicas", action="store_true",
                    help="with several ranks: an independent torus per rank instead of one problem split")
    return ap.parse_args()


def _duffy_weights(n: int) -> np.ndarray:
    """Weights of the n x n Duffy-collapsed Gauss-Legendre rule on the
    reference triangle, in the library's node order (xi-major)."""
    g, wg = np.polynomial.legendre.leggauss(n)
    g, wg = 0.5 * (g + 1), 0.5 * wg
    xi = np.repeat(g, n)
    return np.repeat(wg, n) * np.tile(wg, n) * xi


def rank_seed(rank: int) -> int:
    """Seed of the graded torus and its targets on one rank with --replicas:
    every rank then solves its own independent problem (weak scaling, no
    data-path collective); rank 0's is the single-GPU workload.  Without
    --replicas all ranks share rank 0's problem, split into Morton ranges."""
    return 2 + 1009 * rank


def workload(args, rank: int = 0):
    import synth
    seed = rank_seed(rank)
    if args.small:
        w = synth.torus_c2(n_targets=min(args.targets or 50_000, 50_000), seed=seed, nu=60, nv=16)
    elif getattr(args, "cells", None):
        nu, nv = (int(v) for v in args.cells.lower().split("x"))
        w = synth.torus_c2(n_targets=args.targets or 1_000_000, seed=seed, nu=nu, nv=nv)
    else:
        w = synth.torus_c2(n_targets=args.targets or 1_000_000, seed=seed)
    return w


def reduce_over_ranks(dist, t_ms: float, units: int, device):
    """Whole-job timing across ranks: the slowest rank's time and the units
    all ranks processed.  With one process (dist None) this is the identity."""
    if dist is None:
        return t_ms, units
    import torch
    t = torch.tensor([t_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), int(round(u.item()))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.p = None
        fd, self.path = tempfile.mkstemp(prefix=f"lsm_clocks{index}_", suffix=".csv")
        os.close(fd)

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            try:
                os.unlink(self.path)
            except OSError:
                pass
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.fh.close()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in open(self.path):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        try:
            os.unlink(self.path)
        except OSError:
            pass
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(w, seconds: float, rule_n: int, sigma_x: bool = False, check=None):
    """The FP64 oracle (direct sum, all pairs) on a target sample, all host
    cores; with sigma_x, sigma(x) and its gradient are part of each evaluation.
    `check`: further targets at which the oracle's Phi is returned too (the
    precision paths' errors are measured there).  Returns (baseline, Phi at
    check or None)."""
    import oracle
    m = w["mesh"]
    if sigma_x:
        c, sj, dmax = oracle.sigma_sources(m.verts, m.tris)
        s0 = oracle.sigma0_default(dmax)
        y, nw, _ = oracle.sources(m.verts, m.tris, sj, rule_n, 0)

        def run(xx):
            sg, gs = oracle.sigma_x(c, sj, s0, xx)
            return oracle.phi_grad_sigx(y, nw, xx, sg, gs)
    else:
        y, nw, sg = oracle.sources(m.verts, m.tris, m.sigma, rule_n, 0)

        def run(xx):
            return oracle.phi_grad(y, nw, sg, xx)
    x = w["targets"]
    ncal = 8 * (os.cpu_count() or 1)
    t0 = time.perf_counter()
    run(x[:ncal])
    dt = time.perf_counter() - t0
    n = int(max(ncal, min(len(x), ncal * seconds / max(dt, 1e-6))))
    t0 = time.perf_counter()
    run(x[:n])
    dt = time.perf_counter() - t0
    phi_check = run(np.ascontiguousarray(check))[0] if check is not None and len(check) else None
    return ({"value": n / dt, "unit": "evals/s", "cores": os.cpu_count(), "kind": "oracle",
             "sample": f"{n} of {len(x)} targets, full FP64 direct sum over {len(y)} source nodes "
                       f"({dt:.1f} s)"}, phi_check)


def run_reference(args, rank, world):
    """The oracle as the reference arm: each step evaluates a bounded sample."""
    if rank != 0:
        return
    w = workload(args)
    import oracle
    m = w["mesh"]
    y, nw, sg = oracle.sources(m.verts, m.tris, m.sigma, w["rule"]["n"], 0)
    x = w["targets"]
    ncal = 8 * (os.cpu_count() or 1)
    t0 = time.perf_counter()
    oracle.phi_grad(y, nw, sg, x[:ncal])
    per = (time.perf_counter() - t0) / ncal
    n = int(max(ncal, min(len(x), 60.0 / max(per, 1e-9) / max(1, args.steps + args.warmup))))
    for _ in range(args.warmup):
        oracle.phi_grad(y, nw, sg, x[:n])
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.phi_grad(y, nw, sg, x[:n])
    dt = time.perf_counter() - t0
    val = n * args.steps / dt
    cb = {"value": val, "unit": "evals/s", "cores": os.cpu_count(), "kind": "oracle",
          "sample": f"{n} targets per step of {len(x)}, FP64 direct sum over {len(y)} nodes"}
    print(json.dumps({
        "impl": "reference", "metric": "phi_grad_evals_per_s", "value": val, "unit": "evals/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w["name"], "targets": len(x), "sources": len(y), "sample_targets": n},
        "cpu_baseline": cb,
        "e2e": {"value": val, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def bench_ellipsoids(args):
    """512 ellipsoids (200-5,000 triangles), order-6 charts, one batched solve
    per step: every Newton sweep is one captured CUDA graph over all meshes."""
    import torch
    import paper_1909_13356_gb300 as lsm
    import synth
    w = synth.ellipsoid_batch_c4()
    ctx = lsm.Context(0, tree_grid=args.tree_grid, ff_block=args.ff_block)
    meshes = [ctx.upload(m.verts, m.tris, m.sigma, n_gl=4) for m in w["meshes"]]
    batch = lsm.Batch(ctx, meshes)
    tol = 1e-10
    t0 = time.perf_counter()
    tune = batch.autotune(order=6, err_budget=4e-8) if not args.no_tune else None
    t_tune = time.perf_counter() - t0
    for _ in range(args.warmup):
        batch.solve_charts(order=6, tol=tol, precision=lsm.MIXED, use_graph=True, device_out=True)
    torch.cuda.synchronize()
    l0 = ctx.launch_count
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    clk = ClockSampler(0)
    clk.start()
    a.record()
    for _ in range(args.steps):
        x, h, st, stats = batch.solve_charts(order=6, tol=tol, precision=lsm.MIXED, use_graph=True, device_out=True)
    b.record()
    torch.cuda.synchronize()
    clocks = clk.stop()
    dt = a.elapsed_time(b) / 1e3 / args.steps
    launches = (ctx.launch_count - l0) // args.steps
    # the same work mesh by mesh, for comparison
    t1 = time.perf_counter()
    n_alone = 0
    for mesh in ([] if args.no_unbatched else meshes):
        _, _, _, s1 = mesh.solve_charts(order=6, tol=tol, precision=lsm.MIXED, device_out=True)
        n_alone += s1.n_converged
    torch.cuda.synchronize()
    dt_alone = max(time.perf_counter() - t1, 1e-9)
    print(json.dumps({
        "metric": "chart_nodes_per_s", "value": stats.n_converged / dt, "unit": "nodes/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+ff", "data": "synthetic",
        "config": {"workload": w["name"], "meshes": len(meshes), "triangles": sum(m.m for m in w["meshes"]),
                   "chart_nodes": stats.n_nodes, "order": 6, "tol": tol, "graph": True},
        "newton": {"sweeps": stats.iterations, "active_per_iter": stats.active_per_iter,
                   "n_failed": stats.n_failed, "max_residual": stats.max_residual},
        "gpu_launches_per_step": launches,
        "graph_replays_per_step": (stats.iterations + 1) // 2,
        "autotune": tune, "autotune_s": t_tune,
        "clocks": clocks,
        "unbatched": None if args.no_unbatched else {"seconds": dt_alone, "nodes_per_s": n_alone / dt_alone},
    }))


def bench_serve(args):
    """A Poisson stream of mesh requests (ellipsoid, graded torus, bumped
    icosphere; triangles log-uniform in [1e3, tmax]), order-8 charts to 1e-10,
    submitted at their arrival times to the continuous-batching server.

    Meshes come from a pool of templates (per generator, 24 sizes spread
    log-uniformly over the range), each request taking its generator's
    template nearest its size: building thousands of meshes of up to 5e5
    triangles on the host would otherwise pace the stream.  With
    --serve-seconds the stream is cut at that wall time: requests still
    queued then are cancelled and the running ones finish; latencies are those
    of the completed requests, and a queue that grows over the run is
    reported as unstable, with the completion rate as the capacity."""
    import paper_1909_13356_gb300 as lsm
    import synth
    from synth.workloads import make_request_mesh
    reqs = synth.serve_stream_c5(nreq=args.requests, rate=args.rate, tmax=args.tmax)
    sizes = np.exp(np.linspace(np.log(1e3), np.log(args.tmax), 24))
    templates = {}

    def mesh_of(r):
        k = int(np.argmin(np.abs(np.log(sizes) - np.log(r["T"]))))
        key = (r["kind"], k)
        if key not in templates:
            templates[key] = make_request_mesh(dict(kind=r["kind"], T=int(sizes[k]), seed=1000 * r["kind"] + k))
        return templates[key]

    ctx = lsm.Context(0, tree_grid=args.tree_grid, ff_block=args.ff_block)
    # warm the kernels once
    m0 = mesh_of(reqs[0])
    wm = ctx.upload(m0.verts, m0.tris, m0.sigma, n_gl=4)
    wm.solve_charts(order=8, tol=1e-10, precision=lsm.MIXED)
    wm.free()
    for r in reqs:            # build the templates before the clock starts
        mesh_of(r)
    srv = lsm.Server(ctx, slots=4)
    t_start = time.perf_counter()
    tickets = []
    queue_trace = []
    lag = []
    cut = args.serve_seconds if args.serve_seconds > 0 else float("inf")
    for r in reqs:
        delay = r["arrival"] - (time.perf_counter() - t_start)
        if delay > 0:
            time.sleep(delay)
        now = time.perf_counter() - t_start
        if now > cut:
            break
        m = mesh_of(r)
        tickets.append(srv.submit(m.verts, m.tris, m.sigma, n_gl=4, order=8, tol=1e-10))
        lag.append(now - r["arrival"])
        queue_trace.append((now, srv.info()["queued"]))
    # past the cut: stop admitting, cancel what still waits, let the rest finish
    while time.perf_counter() - t_start < min(cut, reqs[-1]["arrival"] + 1.0) and cut < float("inf"):
        time.sleep(0.05)
        queue_trace.append((time.perf_counter() - t_start, srv.info()["queued"]))
    n_cancel = sum(1 for t in tickets if srv.cancel(t)) if cut < float("inf") else 0
    res = [srv.result(t) for t in tickets]
    wall = time.perf_counter() - t_start
    info = srv.info()
    srv.close()
    done = [r for r in res if r["status"] == 0]
    lat = np.array([r["t_done_ms"] - r["t_submit_ms"] for r in done]) if done else np.array([np.nan])
    nodes = sum(r["stats"].n_converged for r in done)
    t_last_done = max((r["t_done_ms"] for r in done), default=0.0) / 1e3
    half = len(lat) // 2
    q = np.array([v for _, v in queue_trace]) if queue_trace else np.zeros(1)
    growing = bool(len(q) > 4 and q[-len(q) // 4:].mean() > 2.0 * max(1.0, q[:len(q) // 4].mean()))
    stable = (not growing and n_cancel == 0 and
              bool(np.median(lat[half:]) < 2.0 * np.median(lat[:half]) + 1000.0))
    print(json.dumps({
        "metric": "serve_latency_p50_ms", "value": float(np.percentile(lat, 50)), "unit": "ms", "n_gpus": 1,
        "steps": len(done), "warmup": 1, "ms_per_step": wall * 1e3 / max(1, len(done)), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+ff", "data": "synthetic",
        "config": {"workload": "serve_stream", "requests_in_stream": len(reqs), "requests_submitted": len(tickets),
                   "rate_per_s": args.rate, "triangles": [1000, args.tmax], "order": 8, "tol": 1e-10, "slots": 4,
                   "cut_s": args.serve_seconds or None, "mesh_templates": len(templates)},
        "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
        "completed": len(done), "cancelled": n_cancel,
        "failed": sum(r["status"] not in (0, -7) for r in res),
        "chart_nodes_per_s": nodes / max(t_last_done, 1e-9),
        "capacity_requests_per_s": len(done) / max(t_last_done, 1e-9),
        "submission_lag_s_max": float(max(lag)) if lag else None,
        "max_queued": int(q.max()), "queue_growing": growing, "max_running": info["max_running"],
        "peak_device_bytes": info["peak_in_use_bytes"], "stable": stable,
    }))


def bench_icosphere(args):
    """Bumped icosphere, level 8 (1,310,720 triangles, Duffy 4x4 sources =
    20,971,520 nodes), 2e7 targets within 3 sigma: one mixed-path Phi/grad-Phi
    evaluation per step (treecode far field).  Error: the mixed path against
    the float-float path (FP64-accurate; its parity with the FP64 oracle on
    this mesh is a test) on 1e5 targets."""
    import torch
    import paper_1909_13356_gb300 as lsm
    import synth
    n = args.targets if args.targets else 20_000_000
    w = synth.icosphere_c3(n_targets=n)
    m = w["mesh"]
    ctx = lsm.Context(0, tree_degree=args.tree_degree, tree_theta=args.tree_theta, tree_grid=args.tree_grid,
                      ff_block=args.ff_block, tree_cluster=args.tree_cluster)
    t0 = time.perf_counter()
    mesh = ctx.upload(m.verts, m.tris, m.sigma, n_gl=4)
    torch.cuda.synchronize()
    t_up = time.perf_counter() - t0
    x = torch.from_numpy(w["targets"]).cuda()
    phi = torch.empty(n, dtype=torch.float64, device="cuda")
    grad = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    # the autotuner picks the far field on windows of the targets (untimed);
    # then the first call builds the chosen tree (node boxes, proxy weights)
    t0 = time.perf_counter()
    tune = mesh.autotune(x, err_budget=4e-8) if not (args.tree_degree or args.tree_theta) else None
    t_tune = time.perf_counter() - t0
    t0 = time.perf_counter()
    mesh.eval_phi_grad(x[:4096], lsm.MIXED)
    torch.cuda.synchronize()
    t_tree = time.perf_counter() - t0
    for _ in range(args.warmup):
        mesh.eval_phi_grad(x, lsm.MIXED, phi=phi, grad=grad)
    torch.cuda.synchronize()
    ctx.read_stats(reset=True)
    ctx.set_profiling(True)
    l0 = ctx.launch_count
    clk = ClockSampler(0)
    clk.start()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(args.steps):
        mesh.eval_phi_grad(x, lsm.MIXED, phi=phi, grad=grad)
    b.record()
    torch.cuda.synchronize()
    clocks = clk.stop()
    ctx.set_profiling(False)
    stats = ctx.read_stats(reset=True)
    launches = ctx.launch_count - l0
    ms = a.elapsed_time(b) / args.steps
    nref = min(n, 100_000)
    pff, gff = mesh.eval_phi_grad(x[:nref], lsm.FF)
    err_ff = float((phi[:nref] - pff).abs().max())
    gerr_ff = float((grad[:nref] - gff).abs().max())
    peaks = ctx.measure_peaks()
    fp32_peak = _peak_fp32(peaks)
    # the mixed path against the FP64 direct sum (the reference path) on a
    # coherent sample of the targets (--fp64-check targets; untimed)
    err_fp64 = None
    if args.fp64_check:
        sel = torch.from_numpy(_coherent_sample(w["targets"], 4, max(256, args.fp64_check // 4))).cuda()
        p64, g64 = mesh.eval_phi_grad(x[sel], lsm.FP64)
        err_fp64 = {"targets": int(sel.shape[0]), "err_phi": float((phi[sel] - p64).abs().max()),
                    "err_grad": float((grad[sel] - g64).abs().max())}
    ms_k = stats["kind_ms"][0]
    fl = stats["kind_pairs_far"][0] * FLOPS_FAR_PAIR + stats["kind_pairs_near"][0] * FLOPS_NEAR_PAIR
    ach = fl / (ms_k / 1e3) / 1e12 if ms_k > 0 else None
    print(json.dumps({
        "metric": "phi_grad_evals_per_s", "value": n / (ms / 1e3), "unit": "evals/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+ff", "data": "synthetic",
        "config": {"workload": w["name"], "triangles": m.m, "sources": mesh.info()["n_sources"],
                   "targets": n, "precision": "mixed", "cutoff_sigma": {"mixed": 6.5},
                   "far_field": ("autotuned" if tune else
                                 f"treecode (degree {args.tree_degree or 'default'}, theta {args.tree_theta or 'default'})"),
                   "upload_s": t_up, "tree_build_s": t_tree, "autotune_s": t_tune, "autotune": tune,
                   "l2": "inputs (480 MB targets, 336 MB sources) larger than L2"},
        "pairs_evaluated_per_step": (stats["kind_pairs_far"][0] + stats["kind_pairs_near"][0]) / args.steps,
        "dense_equivalent_pairs_per_s": n * mesh.info()["n_sources"] / (ms / 1e3),
        "gpu_launches": launches,
        "roofline": {"bound": "alu", "achieved": ach, "peak": fp32_peak, "unit": "TFLOP/s",
                     "frac": ach / fp32_peak if ach else None, "traffic": None, "kernel": "k_eval_mixed",
                     "share_of_step": ms_k / (ms * args.steps),
                     "peak_source": "measured on this GPU by lsm_measure_peaks: max(FFMA, packed FFMA2)"},
        "peaks": peaks, "err_mixed_vs_fp64_direct": err_fp64,
        "clocks": clocks,
        "err_mixed_vs_ff_1e5": err_ff, "grad_err_mixed_vs_ff_1e5": gerr_ff,
    }))


FLOPS_HESS_FAR = 60    # Hessian of the double layer per far pair (FP32; rsqrt not counted)
FLOPS_HESS_NEAR = 90   # Hessian of the smoothed kernel per near pair (FP64; erf, exp not counted)


def bench_geometry(args):
    """Chart geometry on the graded torus: the charts are solved once (mixed,
    order 8, to 1e-12) and grad Phi taken on the float-float path, untimed;
    a step then evaluates the Hessian of Phi at every chart node, the frames,
    second derivatives and curvatures, the Gauss flux and the Gauss-Bonnet
    integral.  value = chart nodes per second."""
    import torch
    import paper_1909_13356_gb300 as lsm
    w = workload(args, 0)
    m = w["mesh"]
    ctx = lsm.Context(0, tree_grid=args.tree_grid, ff_block=args.ff_block)
    mesh = ctx.upload(m.verts, m.tris, m.sigma, n_gl=w["rule"]["n"], subdiv=w["rule"]["subdiv"])
    x, h, _, st = mesh.solve_charts(order=args.order, tol=args.tol, precision=lsm.MIXED, device_out=True)
    _, g = mesh.eval_phi_grad(x, lsm.FF)
    n = int(h.shape[0])
    wq = torch.from_numpy(np.tile(_duffy_weights(args.order // 2 + 2), m.m)).cuda()
    out = {}

    def step():
        H = mesh.eval_hessian(x)
        _, _, jac = mesh.chart_frames(args.order, h, g)
        _, _, _, km, kg = mesh.chart_curvature(args.order, h, g, H)
        out["eps0"] = mesh.gauss_flux(args.order, x, g, jac, (1.0, 0.0, 0.0))
        out["gb"] = float((wq * jac * kg).sum())
        out["km"] = (float(km.min()), float(km.max()))

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ctx.read_stats(reset=True)
    ctx.set_profiling(True)
    l0 = ctx.launch_count
    clk = ClockSampler(0)
    clk.start()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(args.steps):
        step()
    b.record()
    torch.cuda.synchronize()
    clocks = clk.stop()
    ctx.set_profiling(False)
    stats = ctx.read_stats(reset=True)
    ms = a.elapsed_time(b) / args.steps
    ms_k = stats["kind_ms"][3]
    far, near = stats["kind_pairs_far"][3], stats["kind_pairs_near"][3]
    peaks = ctx.measure_peaks()
    p32 = _peak_fp32(peaks)
    p64 = peaks["dfma_tflops"]
    f32 = far * FLOPS_HESS_FAR / (ms_k / 1e3) / 1e12
    f64 = near * FLOPS_HESS_NEAR / (ms_k / 1e3) / 1e12
    cpu = None
    if not args.no_cpu_baseline:
        cpu = cpu_baseline_hessian(w, args.cpu_seconds, w["rule"]["n"], x.cpu().numpy())
    print(json.dumps({
        "metric": "chart_geometry_nodes_per_s", "value": n / (ms / 1e3), "unit": "chart nodes/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64 near + f32 far", "data": "synthetic",
        "config": {"workload": w["name"] + "_chart_geometry", "chart_order": args.order, "chart_nodes": n,
                   "step": "Hessian at every node, frames, second derivatives, curvatures, Gauss flux, "
                           "Gauss-Bonnet integral",
                   "l2": "inputs larger than L2 (1.1e6 nodes x 13 doubles; 1.1e6 sources)"},
        "gpu_launches": (ctx.launch_count - l0) // max(1, args.steps),
        "roofline": {"bound": "alu", "kernel": "k_eval_hess", "achieved": f32 + f64, "unit": "TFLOP/s",
                     "peak": None, "frac": f32 / p32 + f64 / p64, "traffic": None,
                     "frac_fp32_far": f32 / p32, "frac_fp64_near": f64 / p64, "peaks": peaks,
                     "note": "far pairs on the FP32 pipe, near pairs on the FP64 pipe: frac is the sum of the two "
                             "pipes' fractions",
                     "pairs_far": far, "pairs_near": near, "share_of_step": ms_k / (ms * args.steps)},
        "eps0": out["eps0"], "gauss_bonnet_integral_K": out["gb"], "mean_curvature_range": out["km"],
        "clocks": clocks, "cpu_baseline": cpu,
    }))


def cpu_baseline_hessian(w, seconds, rule_n, nodes):
    """The FP64 oracle's Phi, grad Phi and Hessian (direct sums) on a sample of
    chart nodes, all host cores."""
    import oracle
    m = w["mesh"]
    y, nw, sg = oracle.sources(m.verts, m.tris, m.sigma, rule_n, 0)
    ncal = 4 * (os.cpu_count() or 1)
    t0 = time.perf_counter()
    oracle.phi_grad_hess(y, nw, sg, nodes[:ncal])
    dt = time.perf_counter() - t0
    k = int(max(ncal, min(len(nodes), ncal * seconds / max(dt, 1e-6))))
    t0 = time.perf_counter()
    oracle.phi_grad_hess(y, nw, sg, nodes[:k])
    dt = time.perf_counter() - t0
    return {"value": k / dt, "unit": "chart nodes/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{k} of {len(nodes)} chart nodes, FP64 Phi, grad, Hessian by direct sums ({dt:.1f} s)"}


def _peak_fp32(peaks):
    return max(peaks["ffma_tflops"], peaks["ffma2_tflops"])


# DRAM bytes per launch of a pair kernel on the bench step, from a one-pass ncu
# capture of that step (dram__bytes_read.sum + dram__bytes_write.sum over the
# timed step's launches, divided by the launches the library times), kept with
# the SHA-256 of the sources that decide it (the pair kernels and the
# interaction lists with their launch order): a change there reports null
# until the step is captured again.
DRAM_FILE = os.path.join(ROOT, "paper_1909_13356_gb300", "ncu_dram.json")
DRAM_SOURCES = ("eval.cu", "tree.cu", "ff.cuh")


def kernel_sources_sha256() -> str:
    import hashlib
    h = hashlib.sha256()
    for name in DRAM_SOURCES:
        with open(os.path.join(ROOT, "paper_1909_13356_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def _dram_traffic(kernel: str):
    try:
        with open(DRAM_FILE) as f:
            rec = json.load(f).get(kernel)
        sha = kernel_sources_sha256()
    except (OSError, ValueError):
        return None, None
    if not rec or rec.get("sources_sha256") != sha:
        return None, None
    return rec["dram_bytes_per_launch"], rec["summary"]


def _kernel_rooflines(stats, peaks, step_ms_total, kinds=(0, 1, 2)):
    """Rooflines of the pair kernels timed per launch by the library: counted
    algorithmic flops (FLOPS_FAR_PAIR per far pair, FLOPS_NEAR_PAIR per near
    pair) over the kernel's CUDA-event time, against the FP32 (mixed,
    float-float) or FP64 (FP64 path) FMA throughput measured on this GPU by
    lsm_measure_peaks; one special-function rsqrt per pair against the
    measured rsqrt rate."""
    names = ["k_eval_mixed", "k_eval_ff", "k_eval_fp64"]
    kern = {}
    for k in kinds:
        ms_k = stats["kind_ms"][k]
        if ms_k <= 0:
            continue
        far, near = stats["kind_pairs_far"][k], stats["kind_pairs_near"][k]
        fl = far * FLOPS_FAR_PAIR + near * FLOPS_NEAR_PAIR
        pk = _peak_fp32(peaks) if k < 2 else peaks["dfma_tflops"]
        ach = fl / (ms_k / 1e3) / 1e12
        traffic, tsrc = _dram_traffic(names[k])
        kern[names[k]] = {
            "bound": "alu", "achieved": ach, "peak": pk, "unit": "TFLOP/s", "frac": ach / pk,
            "traffic": traffic, "traffic_unit": "bytes per launch (DRAM read + write)",
            "traffic_source": tsrc, "launches": stats["kind_launches"][k],
            "avg_launch_ms": ms_k / max(1, stats["kind_launches"][k]),
            "pairs_far": far, "pairs_near": near,
            "share_of_step": ms_k / step_ms_total if step_ms_total else None,
            "mufu_rsqrt_util": (far + near) / (ms_k / 1e3) / (peaks["rsqrt_gops"] * 1e9),
            "peak_source": ("measured on this GPU by lsm_measure_peaks: max(FFMA, packed FFMA2) throughput"
                            if k < 2 else "measured on this GPU by lsm_measure_peaks: DFMA throughput"),
        }
    return kern


def _coherent_sample(points, n_chunks: int, chunk: int):
    """Indices of n_chunks contiguous runs of `chunk` points, equally spaced in
    the points' Morton order: spatially compact blocks, as the full set's."""
    from paper_1909_13356_gb300 import shard
    order = np.argsort(shard.morton_keys(points), kind="stable")
    n = len(order)
    starts = [int((n - chunk) * (k + 0.5) / n_chunks) // 256 * 256 for k in range(n_chunks)]
    return np.concatenate([order[s0:s0 + chunk] for s0 in starts])


def main():
    args = parse()
    if args.workload == "icosphere" and args.impl == "ours":
        bench_icosphere(args)
        return
    if args.workload == "ellipsoids" and args.impl == "ours":
        bench_ellipsoids(args)
        return
    if args.workload == "serve" and args.impl == "ours":
        bench_serve(args)
        return
    if args.workload == "geometry" and args.impl == "ours":
        bench_geometry(args)
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import paper_1909_13356_gb300 as lsm
    from paper_1909_13356_gb300 import shard
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    prec = {"mixed": lsm.MIXED, "fp64": lsm.FP64, "ff": lsm.FF}[args.precision]
    if prec == lsm.FF and not args.no_charts:
        raise SystemExit("--precision ff evaluates only (add --no-charts)")
    # one problem split into Morton ranges across ranks (mesh replicated), or
    # with --replicas an independent problem per rank
    sharded = world > 1 and not args.replicas

    w = workload(args, rank if args.replicas else 0)
    m = w["mesh"]
    ctx = lsm.Context(local, tree_degree=args.tree_degree, tree_theta=args.tree_theta, tree_grid=args.tree_grid,
                      ff_block=args.ff_block, mixed_block=args.mixed_block,
                      newton_tree_degree=args.newton_tree_degree, newton_tree_theta=args.newton_tree_theta,
                      newton_cutoff=args.newton_cutoff, tree_cluster=args.tree_cluster)
    # the pipes' measured throughput (roofline denominators), clocks sampled around the probe
    pclk = ClockSampler(local)
    pclk.start()
    peaks = ctx.measure_peaks()
    peaks["clocks"] = pclk.stop()
    if args.sigma_x:
        mesh = ctx.upload_sigma_x(m.verts, m.tris, n_gl=w["rule"]["n"], subdiv=w["rule"]["subdiv"])
    else:
        mesh = ctx.upload(m.verts, m.tris, m.sigma, n_gl=w["rule"]["n"], subdiv=w["rule"]["subdiv"])
    info = mesh.info()
    targets = w["targets"]
    tri_all, uvw_all = lsm.refined_nodes(args.order, np.zeros(m.m, dtype=np.int32))
    x0_all = shard.chart_node_positions(m.verts, m.tris, tri_all, uvw_all)
    if sharded:
        idx_t = shard.morton_ranges(targets, world)[rank]
        idx_c = shard.morton_ranges(x0_all, world)[rank]
        targets = targets[idx_t]
        tri_d = torch.from_numpy(tri_all[idx_c]).to(dev)
        uvw_d = torch.from_numpy(uvw_all[idx_c]).to(dev)
    x_dev = torch.from_numpy(targets).to(dev)
    nt = x_dev.shape[0]
    # far field of the mixed sweeps chosen by the autotuner (untimed)
    tune = None
    if prec == lsm.MIXED and not (args.tree_degree or args.tree_theta):
        tune = mesh.autotune(x_dev, err_budget=4e-8)
    phi = torch.empty(nt, dtype=torch.float64, device=dev)
    grad = torch.empty((nt, 3), dtype=torch.float64, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MB > L2

    last = {}
    eval_ms = []

    def solve():
        if sharded:
            return mesh.solve_charts_nodes(tri_d, uvw_d, tol=args.tol, precision=prec, device_out=True)
        return mesh.solve_charts(order=args.order, tol=args.tol, precision=prec, device_out=True)

    def step():
        ea = torch.cuda.Event(enable_timing=True)
        eb = torch.cuda.Event(enable_timing=True)
        ea.record()
        mesh.eval_phi_grad(x_dev, prec, phi=phi, grad=grad)
        eb.record()
        last["eval_events"] = (ea, eb)
        if args.no_charts:
            return nt, None
        xc, hc, _, st = solve()
        last["x"], last["h"] = xc, hc
        # full Phi + grad Phi evaluations: the near-only verification sweeps,
        # which reuse the far part recorded by the sweep before, are not counted
        return nt + st.evals_fp32 + st.evals_fp64 - st.evals_near_only, st

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    for _ in range(args.warmup):
        step()
    barrier()
    ctx.read_stats(reset=True)
    ctx.set_profiling(True)
    launches0 = ctx.launch_count
    clk = ClockSampler(local)
    clk.start()
    total_units = 0
    step_ms = []
    last_stats = None
    barrier()
    for _ in range(args.steps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        units, last_stats = step()
        b.record()
        torch.cuda.synchronize()
        step_ms.append(a.elapsed_time(b))
        eval_ms.append(last["eval_events"][0].elapsed_time(last["eval_events"][1]))
        total_units += units
    barrier()
    clocks = clk.stop()
    ctx.set_profiling(False)
    stats = ctx.read_stats(reset=True)
    launches = ctx.launch_count - launches0
    t_ms = sum(step_ms)
    t_ms, total_units = reduce_over_ranks(dist, t_ms, total_units, dev)
    value = total_units / (t_ms / 1e3)
    kern = _kernel_rooflines(stats, peaks, sum(step_ms))
    dom = max(kern, key=lambda n: kern[n]["avg_launch_ms"] * kern[n]["launches"]) if kern else None
    roofline = dict(kern[dom], kernel=dom) if dom else None

    # end to end through the C ABI with pinned host buffers: the same number
    # of steps as the device timing, after one warm-up step of the buffers
    e2e = None
    if not args.no_e2e:
        xh = torch.from_numpy(targets).pin_memory()
        ph = torch.empty(nt, dtype=torch.float64).pin_memory()
        gh = torch.empty((nt, 3), dtype=torch.float64).pin_memory()
        if sharded:
            tri_h, uvw_h = tri_all[idx_c], uvw_all[idx_c]

        def e2e_step():
            mesh.eval_phi_grad(xh, prec, phi=ph, grad=gh)
            if args.no_charts:
                return nt, 0
            if sharded:
                _, _, _, st = mesh.solve_charts_nodes(tri_h, uvw_h, tol=args.tol, precision=prec)
            else:
                _, _, _, st = mesh.solve_charts(order=args.order, tol=args.tol, precision=prec)
            return nt + st.evals_fp32 + st.evals_fp64 - st.evals_near_only, st.n_nodes

        e2e_step()
        barrier()
        units = 0
        ncn = 0
        t0 = time.perf_counter()
        for _ in range(args.steps):
            u, ncn = e2e_step()
            units += u
        torch.cuda.synchronize()
        dt_ms = (time.perf_counter() - t0) * 1e3
        dt_ms, units = reduce_over_ranks(dist, dt_ms, units, dev)
        e2e = {"value": units / (dt_ms / 1e3), "unit": "evals/s", "h2d_bytes_per_step": nt * 24 +
               (ncn * (4 + 24) if sharded else 0),
               "d2h_bytes_per_step": nt * 32 + ncn * (24 + 8 + 4), "steps": args.steps}

    # The same inputs on the three precision paths (untimed by the step, each
    # with CUDA events): the float-float evaluation at every target (Phi to
    # FP64 accuracy), the FP64 direct sum on a spatially coherent sample of
    # the targets (its cost is linear in the targets: extrapolated), and the
    # FP64 chart solve on a coherent sample of the chart nodes.
    paths = None
    fp64_kern = None
    if not args.no_charts and not args.sigma_x and prec == lsm.MIXED and not args.no_paths:
        def timed(fn):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record()
            r = fn()
            b.record()
            torch.cuda.synchronize()
            return r, a.elapsed_time(b)

        (pff, gff), ms_ff = timed(lambda: mesh.eval_phi_grad(x_dev, lsm.FF))
        sel = _coherent_sample(targets, 4, 4096)
        xs = x_dev[torch.from_numpy(sel).to(dev)]
        ctx.read_stats(reset=True)
        ctx.set_profiling(True)
        (p64, _), ms_64 = timed(lambda: mesh.eval_phi_grad(xs, lsm.FP64))
        ctx.set_profiling(False)
        fp64_kern = _kernel_rooflines(ctx.read_stats(reset=True), peaks, ms_64, kinds=(2,)).get("k_eval_fp64")
        if sharded:
            node_pts, tri_src, uvw_src = x0_all[idx_c], tri_all[idx_c], uvw_all[idx_c]
        else:
            node_pts, tri_src, uvw_src = x0_all, tri_all, uvw_all
        csel = _coherent_sample(node_pts, 4, 4096)
        (xc64, _, st64, s64), ms_s64 = timed(lambda: mesh.solve_charts_nodes(
            tri_src[csel], uvw_src[csel], tol=args.tol, precision=lsm.FP64, device_out=True))
        e_mx = nt / (statistics.median(eval_ms) / 1e3)
        e_ff = nt / (ms_ff / 1e3)
        e_64 = len(sel) / (ms_64 / 1e3)
        nodes_mx = last_stats.n_converged / (statistics.median(step_ms) / 1e3 - statistics.median(eval_ms) / 1e3)
        nodes_64 = s64.n_converged / (ms_s64 / 1e3)
        if not sharded:
            dx = float((xc64 - last["x"][torch.from_numpy(csel).to(dev)]).abs().max())
        else:
            dx = None
        paths = {
            "mixed": {"evals_per_s": e_mx, "targets": nt, "tol_phi": 1e-7,
                      "ms": statistics.median(eval_ms)},
            "float_float": {"evals_per_s": e_ff, "targets": nt, "tol_phi": 1e-12, "ms": ms_ff},
            "fp64": {"evals_per_s": e_64, "targets_timed": len(sel), "extrapolated": True, "ms": ms_64,
                     "sample": "4 runs of 4096 consecutive targets in Morton order, equally spaced; the "
                               "direct sum's cost per target does not depend on the other targets"},
            "speedup_float_float_vs_fp64": e_ff / e_64,
            "speedup_mixed_vs_fp64": e_mx / e_64,
            "chart_solve": {
                "mixed_then_float_float_nodes_per_s": nodes_mx,
                "fp64_nodes_per_s": nodes_64, "fp64_nodes_timed": len(csel), "fp64_extrapolated": True,
                "fp64_sweeps": s64.iterations, "fp64_max_residual": s64.max_residual,
                "mixed_max_residual": last_stats.max_residual,
                "max_node_position_difference": dx, "tol": args.tol,
                "speedup": nodes_mx / nodes_64,
            },
        }
        last["err_check"] = (sel[::32], pff, p64)

    # Gauss flux error of the last step's charts about the tube's centre line
    # (untimed): grad Phi at the nodes from the float-float path, then the
    # frames and the flux (Sec. 5)
    eps0 = None
    if "x" in last and not args.no_geometry and not sharded:
        _, gc = mesh.eval_phi_grad(last["x"], lsm.FF)
        _, _, jac = mesh.chart_frames(args.order, last["h"], gc)
        eps0 = {"x0": [1.0, 0.0, 0.0], "value": mesh.gauss_flux(args.order, last["x"], gc, jac, (1.0, 0.0, 0.0)),
                "grad": "float-float path"}
        # Gauss-Bonnet: the charts' Gaussian curvature integrates to 2 pi chi = 0
        # on the torus (Hessian at the nodes, untimed)
        gb = None
        if not args.sigma_x:
            hc = mesh.eval_hessian(last["x"])
            _, _, _, kmc, kgc = mesh.chart_curvature(args.order, last["h"], gc, hc)
            n_gl = args.order // 2 + 2
            wq = torch.from_numpy(np.tile(_duffy_weights(n_gl), m.m)).to(dev)
            gb = {"integral_K": float((wq * jac * kgc).sum()), "expected": 0.0,
                  "mean_curvature_range": [float(kmc.min()), float(kmc.max())]}
            del hc, kmc, kgc
        eps0["gauss_bonnet"] = gb
        del gc, jac

    cpu = None
    if not args.no_cpu_baseline and rank == 0 and world == 1:
        check = None
        if "err_check" in last:
            csel_t, pff, p64 = last["err_check"]
            check = targets[csel_t]
        cpu, phi_check = cpu_baseline(w, args.cpu_seconds, w["rule"]["n"], args.sigma_x, check)
        if paths is not None and phi_check is not None:
            # errors of the three paths against the oracle at the same targets
            csel_t, pff, p64 = last["err_check"]
            idx = torch.from_numpy(csel_t).to(dev)
            paths["mixed"]["err_phi_vs_oracle"] = float(np.abs(phi[idx].cpu().numpy() - phi_check).max())
            paths["float_float"]["err_phi_vs_oracle"] = float(np.abs(pff[idx].cpu().numpy() - phi_check).max())
            paths["fp64"]["err_phi_vs_oracle"] = float(np.abs(p64[::32].cpu().numpy() - phi_check).max())
            paths["err_sample"] = f"{len(csel_t)} targets (every 32nd of the FP64 sample), oracle FP64 direct sum"

    if rank == 0:
        st = last_stats
        out = {
            "metric": "phi_grad_evals_per_s",
            "value": value,
            "unit": "evals/s",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": t_ms / args.steps,
            "higher_is_better": True,
            "scaling": "strong" if sharded else "weak",
            "vs_baseline": None,
            "dtype": {lsm.MIXED: "f32+ff", lsm.FF: "ff", lsm.FP64: "f64"}[prec],
            "data": "synthetic",
            "config": {"workload": w["name"], "triangles": m.m, "sources": info["n_sources"],
                       "targets": len(w["targets"]), "chart_order": args.order,
                       "chart_nodes": len(tri_all) if not args.no_charts else 0,
                       "newton_tol": args.tol, "precision": args.precision, "autotune": tune,
                       # near-field cutoffs: the library's FP64 one; the mixed one as the autotuner
                       # chose it (candidates meeting erfc(c/sqrt2) + c sqrt(2/pi) e^(-c^2/2) <= 1e-8),
                       # else the default 6.5
                       "cutoff_sigma": {"fp64_and_float_float": 8.0,
                                        "mixed": (tune or {}).get("cutoff", 6.5) or 6.5},
                       "ff_targets_per_cta": args.ff_block or 64,
                       # the mixed Newton sweeps' own treecode (used where coarser than the mesh's)
                       "newton_mixed_tree": ("the mesh's mixed treecode" if args.newton_tree_degree < 0 else
                                             {"degree": args.newton_tree_degree or 5,
                                              "theta": args.newton_tree_theta or 0.5}),
                       "newton_mixed_cutoff_sigma": args.newton_cutoff or 5.0,
                       "sigma": ("sigma(x), eq. sigma2: lambda 2.5, sigma0 = max D / sqrt(2 ln 2) = "
                                 f"{mesh.sigma0:.5g}" if args.sigma_x else "per triangle, 0.5 sqrt(2 area)"),
                       "parallelism": (f"{world} ranks, targets and chart nodes in Morton ranges, mesh replicated"
                                       if sharded else
                                       (f"{world} ranks, one independent torus (own seed) each"
                                        if world > 1 else "single GPU")),
                       "l2": "flushed (256 MB write) before each timed step"},
            "units_per_step": ({"targets_mixed": nt, "newton_mixed": st.evals_fp32,
                                "newton_float_float_full": st.evals_fp64 - st.evals_near_only,
                                "newton_float_float_near_only_not_counted": st.evals_near_only}
                               if st else {"targets": nt}),
            # rank 0's units per second, by the error each is made to: the
            # mixed evaluation (1e-7), the mixed Newton sweeps (about 1e-6 on
            # their coarser treecode: they only steer the nodes, which the
            # float-float sweeps take to the tolerance) and the float-float
            # record sweeps (FP64 accuracy)
            "value_by_error_rank0": ({"mixed_1e-7": nt / (t_ms / args.steps / 1e3),
                                      "newton_mixed_steering_about_1e-6": st.evals_fp32 / (t_ms / args.steps / 1e3),
                                      "float_float_fp64_accuracy": (st.evals_fp64 - st.evals_near_only)
                                      / (t_ms / args.steps / 1e3)} if st else None),
            "chart_nodes_per_s": st.n_converged * world / (t_ms / args.steps / 1e3) if st else None,
            "newton": {"iterations": st.iterations, "active_per_iter": st.active_per_iter,
                       "n_failed": st.n_failed, "eps_newton": st.eps_newton,
                       "max_residual": st.max_residual, "evals_fp64": st.evals_fp64} if st else None,
            "precision_paths": paths,
            "gauss_flux_eps0": eps0,
            "gpu_launches": launches,
            "roofline": roofline,
            "roofline_kernels": dict(kern, **({"k_eval_fp64": fp64_kern} if fp64_kern else {})),
            "peaks": peaks,
            "clocks": clocks,
            "e2e": e2e,
            "cpu_baseline": cpu,
        }
        print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

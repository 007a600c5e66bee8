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
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FP32_LANES_PER_SM = 128          # FP32 FMA lanes per SM (4 SMSPs x 32)
NUM_SMS = 152
SM_MAX_MHZ = 2070.0
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
    ap.add_argument("--tree-degree", type=int, default=0, help="treecode degree (0: library default)")
    ap.add_argument("--tree-theta", type=float, default=0.0, help="treecode opening parameter (0: default)")
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
    return ap.parse_args()


def _duffy_weights(n: int) -> np.ndarray:
    """Weights of the n x n Duffy-collapsed Gauss-Legendre rule on the
    reference triangle, in the library's node order (xi-major)."""
    g, wg = np.polynomial.legendre.leggauss(n)
    g, wg = 0.5 * (g + 1), 0.5 * wg
    xi = np.repeat(g, n)
    return np.repeat(wg, n) * np.tile(wg, n) * xi


def rank_seed(rank: int) -> int:
    """Seed of the graded torus and its targets on one rank.  Every rank
    solves its own independent problem (weak scaling, no data-path
    collective); rank 0's is the single-GPU workload."""
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
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_rank{index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
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
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(w, seconds: float, rule_n: int, sigma_x: bool = False):
    """The FP64 oracle (direct sum, all pairs) on a target sample, all host
    cores; with sigma_x, sigma(x) and its gradient are part of each evaluation."""
    import oracle
    m = w["mesh"]
    if sigma_x:
        c, sj, dmax = oracle.sigma_sources(m.verts, m.tris)
        s0 = oracle.sigma0_default(dmax)
        y, nw, _ = oracle.sources(m.verts, m.tris, sj, rule_n, 0)

        def run(xx):
            sg, gs = oracle.sigma_x(c, sj, s0, xx)
            oracle.phi_grad_sigx(y, nw, xx, sg, gs)
    else:
        y, nw, sg = oracle.sources(m.verts, m.tris, m.sigma, rule_n, 0)

        def run(xx):
            oracle.phi_grad(y, nw, sg, xx)
    x = w["targets"]
    ncal = 8 * (os.cpu_count() or 1)
    t0 = time.perf_counter()
    run(x[:ncal])
    dt = time.perf_counter() - t0
    n = int(max(ncal, min(len(x), ncal * seconds / max(dt, 1e-6))))
    t0 = time.perf_counter()
    run(x[:n])
    dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": "evals/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{n} of {len(x)} targets, full FP64 direct sum over {len(y)} source nodes "
                      f"({dt:.1f} s)"}


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
    ctx = lsm.Context(0, tree_grid=args.tree_grid)
    meshes = [ctx.upload(m.verts, m.tris, m.sigma, n_gl=4) for m in w["meshes"]]
    batch = lsm.Batch(ctx, meshes)
    tol = 1e-10
    for _ in range(args.warmup):
        batch.solve_charts(order=6, tol=tol, precision=lsm.MIXED, use_graph=True, device_out=True)
    torch.cuda.synchronize()
    l0 = ctx.launch_count
    t0 = time.perf_counter()
    for _ in range(args.steps):
        x, h, st, stats = batch.solve_charts(order=6, tol=tol, precision=lsm.MIXED, use_graph=True, device_out=True)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / args.steps
    launches = (ctx.launch_count - l0) // args.steps
    # the same work mesh by mesh, for comparison
    t1 = time.perf_counter()
    n_alone = 0
    for mesh in meshes:
        _, _, _, s1 = mesh.solve_charts(order=6, tol=tol, precision=lsm.MIXED, device_out=True)
        n_alone += s1.n_converged
    torch.cuda.synchronize()
    dt_alone = time.perf_counter() - t1
    print(json.dumps({
        "metric": "chart_nodes_per_s", "value": stats.n_converged / dt, "unit": "nodes/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+ff", "data": "synthetic",
        "config": {"workload": w["name"], "meshes": len(meshes), "triangles": sum(m.m for m in w["meshes"]),
                   "chart_nodes": stats.n_nodes, "order": 6, "tol": tol, "graph": True},
        "newton": {"sweeps": stats.iterations, "active_per_iter": stats.active_per_iter,
                   "n_failed": stats.n_failed, "max_residual": stats.max_residual},
        "gpu_launches_per_step": launches,
        "unbatched": {"seconds": dt_alone, "nodes_per_s": n_alone / dt_alone},
    }))


def bench_serve(args):
    """A Poisson stream of mesh requests (ellipsoid, graded torus, bumped
    icosphere; triangles log-uniform in [1e3, tmax]), order-8 charts to 1e-10,
    submitted at their arrival times to the continuous-batching server."""
    import paper_1909_13356_gb300 as lsm
    import synth
    from synth.workloads import make_request_mesh
    reqs = synth.serve_stream_c5(nreq=args.requests, rate=args.rate, tmax=args.tmax)
    meshes = [make_request_mesh(r) for r in reqs]
    ctx = lsm.Context(0, tree_grid=args.tree_grid)
    # warm the kernels once
    m0 = meshes[0]
    wm = ctx.upload(m0.verts, m0.tris, m0.sigma, n_gl=4)
    wm.solve_charts(order=8, tol=1e-10, precision=lsm.MIXED)
    wm.free()
    srv = lsm.Server(ctx, slots=4)
    t_start = time.perf_counter()
    tickets = []
    max_queue = 0
    for r, m in zip(reqs, meshes):
        delay = r["arrival"] - (time.perf_counter() - t_start)
        if delay > 0:
            time.sleep(delay)
        tickets.append(srv.submit(m.verts, m.tris, m.sigma, n_gl=4, order=8, tol=1e-10))
        max_queue = max(max_queue, srv.info()["queued"])
    res = [srv.result(t) for t in tickets]
    wall = time.perf_counter() - t_start
    info = srv.info()
    srv.close()
    lat = np.array([r["t_done_ms"] - r["t_submit_ms"] for r in res])
    nodes = sum(r["stats"].n_converged for r in res if r["status"] == 0)
    half = len(lat) // 2
    print(json.dumps({
        "metric": "serve_latency_p50_ms", "value": float(np.percentile(lat, 50)), "unit": "ms", "n_gpus": 1,
        "steps": len(res), "warmup": 1, "ms_per_step": wall * 1e3 / len(res), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+ff", "data": "synthetic",
        "config": {"workload": "serve_stream", "requests": len(res), "rate_per_s": args.rate,
                   "triangles": [1000, args.tmax], "order": 8, "tol": 1e-10, "slots": 4},
        "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
        "chart_nodes_per_s": nodes / wall, "failed": sum(r["status"] != 0 for r in res),
        "max_queued": max_queue, "max_running": info["max_running"],
        "peak_device_bytes": info["peak_in_use_bytes"],
        "stable": bool(np.median(lat[half:]) < 2.0 * np.median(lat[:half]) + 1000.0),
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
    ctx = lsm.Context(0, tree_degree=args.tree_degree, tree_theta=args.tree_theta, tree_grid=args.tree_grid)
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
    fp32_peak = NUM_SMS * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
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
                     "share_of_step": ms_k / (ms * args.steps)},
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
    ctx = lsm.Context(0, tree_grid=args.tree_grid)
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
    p32 = NUM_SMS * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
    p64 = p32 / 64.0
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
                     "frac_fp32_far": f32 / p32, "frac_fp64_near": f64 / p64,
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

    w = workload(args, rank)
    m = w["mesh"]
    ctx = lsm.Context(local, tree_degree=args.tree_degree, tree_theta=args.tree_theta, tree_grid=args.tree_grid)
    if args.sigma_x:
        mesh = ctx.upload_sigma_x(m.verts, m.tris, n_gl=w["rule"]["n"], subdiv=w["rule"]["subdiv"])
    else:
        mesh = ctx.upload(m.verts, m.tris, m.sigma, n_gl=w["rule"]["n"], subdiv=w["rule"]["subdiv"])
    info = mesh.info()
    x_dev = torch.from_numpy(w["targets"]).to(dev)
    nt = x_dev.shape[0]
    # far field of the mixed sweeps chosen by the autotuner (untimed)
    tune = None
    if prec == lsm.MIXED and not (args.tree_degree or args.tree_theta):
        tune = mesh.autotune(x_dev, err_budget=4e-8)
    phi = torch.empty(nt, dtype=torch.float64, device=dev)
    grad = torch.empty((nt, 3), dtype=torch.float64, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MB > L2

    last = {}

    def step():
        mesh.eval_phi_grad(x_dev, prec, phi=phi, grad=grad)
        if args.no_charts:
            return nt, None
        xc, hc, _, st = mesh.solve_charts(order=args.order, tol=args.tol, precision=prec, device_out=True)
        last["x"], last["h"] = xc, hc
        return nt + sum(st.active_per_iter), st

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
        total_units += units
    barrier()
    clocks = clk.stop()
    ctx.set_profiling(False)
    stats = ctx.read_stats(reset=True)
    launches = ctx.launch_count - launches0
    t_ms = sum(step_ms)
    t_ms, total_units = reduce_over_ranks(dist, t_ms, total_units, dev)
    value = total_units / (t_ms / 1e3)

    # rooflines of the pair kernels, timed per launch by the library; the
    # dominant one (largest device time in the timed region) is "roofline"
    fp32_peak = NUM_SMS * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
    names = ["k_eval_mixed", "k_eval_ff", "k_eval_fp64"]
    kern = {}
    for k in range(3):
        ms_k = stats["kind_ms"][k]
        if ms_k <= 0:
            continue
        fl = stats["kind_pairs_far"][k] * FLOPS_FAR_PAIR + stats["kind_pairs_near"][k] * FLOPS_NEAR_PAIR
        pk = fp32_peak if k < 2 else fp32_peak / 64.0
        ach = fl / (ms_k / 1e3) / 1e12
        kern[names[k]] = {
            "bound": "alu", "achieved": ach, "peak": pk, "unit": "TFLOP/s", "frac": ach / pk,
            "traffic": None, "launches": stats["kind_launches"][k],
            "avg_launch_ms": ms_k / max(1, stats["kind_launches"][k]),
            "pairs_far": stats["kind_pairs_far"][k], "pairs_near": stats["kind_pairs_near"][k],
            "share_of_step": ms_k / sum(step_ms) if step_ms else None,
            "peak_source": ("FP32 FMA lanes: 152 SM x 128 x 2 flops x 2070 MHz" if k < 2 else
                            "FP32 FMA peak / 64 (GB300 FP64 rate)"),
        }
    dom = max(kern, key=lambda n: kern[n]["avg_launch_ms"] * kern[n]["launches"]) if kern else None
    roofline = dict(kern[dom], kernel=dom) if dom else None

    # end to end through the C ABI with pinned host buffers
    e2e = None
    if not args.no_e2e and rank == 0:
        xh = torch.from_numpy(w["targets"]).pin_memory()
        ph = torch.empty(nt, dtype=torch.float64).pin_memory()
        gh = torch.empty((nt, 3), dtype=torch.float64).pin_memory()
        units = 0
        e2e_steps = 1
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ncn = 0
        for _ in range(e2e_steps):
            mesh.eval_phi_grad(xh, prec, phi=ph, grad=gh)
            units += nt
            if not args.no_charts:
                _, _, _, st = mesh.solve_charts(order=args.order, tol=args.tol, precision=prec)
                units += sum(st.active_per_iter)
                ncn = st.n_nodes
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        e2e = {"value": units / dt, "unit": "evals/s", "h2d_bytes_per_step": nt * 24,
               "d2h_bytes_per_step": nt * 32 + ncn * (24 + 8 + 4), "steps": e2e_steps}

    # Gauss flux error of the last step's charts about the tube's centre line
    # (untimed): grad Phi at the nodes from the float-float path, then the
    # frames and the flux (Sec. 5)
    eps0 = None
    if "x" in last and not args.no_geometry:
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
        cpu = cpu_baseline(w, args.cpu_seconds, w["rule"]["n"], args.sigma_x)

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
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": {lsm.MIXED: "f32+ff", lsm.FF: "ff", lsm.FP64: "f64"}[prec],
            "data": "synthetic",
            "config": {"workload": w["name"], "triangles": m.m, "sources": info["n_sources"],
                       "targets": nt, "chart_order": args.order, "chart_nodes": st.n_nodes if st else 0,
                       "newton_tol": args.tol, "precision": args.precision, "autotune": tune,
                       # the library's default near-field cutoffs (lsm_options), unchanged here: the
                       # mixed one meets erfc(c/sqrt2) + c sqrt(2/pi) e^(-c^2/2) <= 1e-8 (3.6e-9 at 6.5)
                       "cutoff_sigma": {"fp64_and_float_float": 8.0, "mixed": 6.5},
                       "sigma": ("sigma(x), eq. sigma2: lambda 2.5, sigma0 = max D / sqrt(2 ln 2) = "
                                 f"{mesh.sigma0:.5g}" if args.sigma_x else "per triangle, 0.5 sqrt(2 area)"),
                       "parallelism": (f"{world} ranks, one independent torus (own seed) each"
                                       if world > 1 else "single GPU"),
                       "l2": "flushed (256 MB write) before each timed step"},
            "chart_nodes_per_s": st.n_converged / (t_ms / args.steps / 1e3) if st else None,
            "newton": {"iterations": st.iterations, "active_per_iter": st.active_per_iter,
                       "n_failed": st.n_failed, "eps_newton": st.eps_newton,
                       "max_residual": st.max_residual, "evals_fp64": st.evals_fp64} if st else None,
            "gauss_flux_eps0": eps0,
            "gpu_launches": launches,
            "roofline": roofline,
            "roofline_kernels": kern,
            "clocks": clocks,
            "e2e": e2e,
            "cpu_baseline": cpu,
        }
        print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

#!/usr/bin/env python
"""Time-to-solution benchmark of the GB300 double-layer Stokes solver.

One step = one pass of the whole hot path on one synthetic porous-pipe
geometry: build the handle from device-resident boundary arrays, assemble
and factorise the block-diagonal preconditioner, solve A sigma = f (pipe-flow
data) by GMRES to a relative residual of 1e-8, and evaluate the velocity at
4096 interior points.

Default workload (the large configuration): outer wall |x/20|^8 + |y/2|^8 = 1
with 8192 nodes, 1000 pores (lognormal radii, median 0.15, sigma 0.3, placed
with gap >= 0.05; radii scaled by 0.95 to make the packing feasible), 128
nodes per pore: N = 136,192 nodes, 272,384 unknowns.

Output: one JSON line (rank 0). `--impl reference` times the CPU oracle on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

FLOPS_PER_PAIR = 18          # 2 sub, rho^2 3, r.a 3, r.sigma 3, products 3, accumulate 4 (FMA = 2)
SM_COUNT = 152
SM_MAX_MHZ = 2070.0
FP32_LANES_PER_SM = 128
FP64_NOMINAL_TFLOPS = 1.25   # nominal dense FP64 of the part
# FP32-pipe operations per pair of the double-float formulation, counted from
# its algorithm (error-free transformations): r 24, rho^2 19, 1/rho^2 3,
# r.a 19, r.sigma 19, coefficient 21, accumulation 24 (an FMA is one op)
DF64_OPS_PER_PAIR = 129
# FP32-pipe operations per pair of the single-precision kernel: r with hi/lo
# parts 6, rho^2 2, r.a 2, r.sigma 2, coefficient 3, accumulation 2
F32_OPS_PER_PAIR = 17
METRIC = "time-to-solution @1e-8 rel. residual; Stokes matvec Gpairs/s vs FLOP peak"
# DRAM bytes (read + write) per launch of the pair kernels on the 136,192-node
# workload, from one ncu capture of each shape (profiles/k_dlp_pairs_*_pipe1000.md);
# keyed by (kernel, threads, targets per thread, tile). A shape that is not
# listed, or a kernel changed since its capture, reports traffic null.
MEASURED_TRAFFIC = {("k_dlp_pairs_df64", 256, 1, 256): 9820672.0,
                    ("k_dlp_pairs_f32", 256, 4, 256): 7642624.0}


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=1)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="pipe1000", choices=["pipe1000", "pipe10"])
    p.add_argument("--precision", default=None, choices=["mixed", "df64", "fp64"])
    p.add_argument("--pc", default=None, choices=["bd", "twogrid"])
    p.add_argument("--coarsen", type=int, default=4)
    p.add_argument("--restart", type=int, default=None)
    p.add_argument("--tol", type=float, default=1e-8)
    p.add_argument("--max-iter", type=int, default=5000)
    p.add_argument("--targets", type=int, default=4096)
    p.add_argument("--e2e-steps", type=int, default=1)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-tune", action="store_true", help="skip the pair kernels' launch-shape autotuner")
    p.add_argument("--kernel-bench", action="store_true",
                   help="time only operator applications (A sigma) of each precision on the workload")
    p.add_argument("--batch-bench", action="store_true",
                   help="time the batched operator and lockstep solve on a multi-geometry batch")
    p.add_argument("--batch-geoms", type=int, default=16)
    p.add_argument("--reps", type=int, default=5)
    p.add_argument("--precisions", default="fp32,df64,fp64")
    p.add_argument("--shape", default="",
                   help="kernel-bench launch shapes, e.g. df64:2:4,fp32:4:8 (precision:variant:ctas_per_sm)")
    return p.parse_args()


def workload_config(name):
    if name == "pipe1000":
        return {"workload": "porous pipe, 1000 pores x 128 nodes + 8192-node wall (N=136192, 272384 unknowns)",
                "outer": "|x/20|^8+|y/2|^8=1", "pores": 1000, "nodes_per_pore": 128, "wall_nodes": 8192,
                "bc": "pipe flow", "tol": 1e-8}
    return {"workload": "porous pipe, 10 pores x 64 nodes + 512-node wall (N=1152, 2304 unknowns)",
            "outer": "|x/4|^8+|y|^8=1", "pores": 10, "nodes_per_pore": 64, "wall_nodes": 512,
            "bc": "pipe flow", "tol": 1e-10}


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    def __init__(self, index=0):
        self.index = index
        self.samples = []
        self.proc = None

    def start(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 7:
                self.samples.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in self.samples for k in range(4) if s[3 + k] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        dist.init_process_group(backend=backend)
        pg = dist
    return world, rank, local, pg


def solver_params(args):
    """Defaults: the 1152-node case is the plain method of its configuration
    (block diagonal, GMRES(50), FP64); the 136,192-node case needs the
    two-grid preconditioner and a long Krylov basis to converge in minutes,
    with double-float operators and FP64 true residuals."""
    big = args.workload == "pipe1000"
    prec = args.precision or ("df64" if big else "fp64")
    pc = args.pc or ("twogrid" if big else "bd")
    restart = args.restart or (600 if big else 50)
    return prec, restart, pc


# ---------------------------------------------------------------------------
# CPU oracle leg: bounded sample of the same workload
# ---------------------------------------------------------------------------

def oracle_sample(geom, iters, budget_s=15.0):
    """Times the oracle's matrix-free operator rows (FP64 numpy) on a sample
    of rows and extrapolates to the pair work of a solve of `iters`
    iterations (one operator application per iteration + one per restart is
    ignored: a lower bound on the oracle's time)."""
    import oracle
    import stokes_inputs as si
    sig = si.random_density(geom, 2).reshape(-1)
    rng = np.random.default_rng(0)
    rows_done = 0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < budget_s:
        rows = rng.choice(geom.n_nodes, 256, replace=False)
        oracle.apply_rows(geom, sig, rows)
        rows_done += rows.size
    el = time.perf_counter() - t0
    pairs = rows_done * geom.n_nodes
    pairs_per_s = pairs / el
    full_matvec_s = geom.n_nodes ** 2 / pairs_per_s
    return {"pairs_per_s": pairs_per_s, "sample_rows": rows_done, "sample_s": el,
            "est_time_to_solution_s": iters * full_matvec_s, "cores": 1}


def run_reference(args):
    world, rank, local, pg = dist_setup(args)
    if rank != 0:
        return
    import stokes_inputs as si
    geom = si.cached_geometry(args.workload, 0)
    # iteration count of the plain block-diagonal solve at this size is
    # taken from the GPU run when known; the reference leg assumes the same
    # number of operator applications (its time is a lower bound)
    iters = int(os.environ.get("STOKES_REF_ITERS", "23" if args.workload == "pipe1000" else "67"))
    times = []
    info = None
    for s in range(args.warmup + args.steps):
        info = oracle_sample(geom, iters, budget_s=8.0)
        if s >= args.warmup:
            times.append(info["est_time_to_solution_s"])
    v = float(np.mean(times))
    cfg = workload_config(args.workload)
    line = {"metric": METRIC, "value": v, "unit": "s", "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": v, "unit": "s", "cores": info["cores"], "kind": "oracle",
                             "sample": f"{info['sample_rows']} random rows of A sigma per step (numpy FP64, "
                                       f"{info['pairs_per_s']/1e6:.1f} Mpairs/s), extrapolated to {iters} "
                                       f"full operator applications"},
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU leg
# ---------------------------------------------------------------------------

def kernel_bench(args):
    """A sigma on the workload for each precision; prints one JSON line per
    precision with the pair kernel's device time from the library's event
    timing (also the entry point used for ncu captures)."""
    import torch
    import paper_1609_04484_gb300 as S
    import stokes_inputs as si
    dev = torch.device("cuda", 0)
    geom = si.cached_geometry(args.workload, 0)
    stream = torch.cuda.current_stream(dev)
    G = S.Geometry(geom, stream=stream.cuda_stream)
    sig = torch.tensor(si.random_density(geom, 1).reshape(-1), device=dev)
    y = torch.empty_like(sig)
    kinds = {"fp32": (S.STOKES_FP32, S.STOKES_PROF_PAIRS_FP32, "k_dlp_pairs_f32"),
             "df64": (S.STOKES_DF64, S.STOKES_PROF_PAIRS_DF64, "k_dlp_pairs_df64"),
             "fp64": (S.STOKES_FP64, S.STOKES_PROF_PAIRS_FP64, "k_dlp_pairs_f64")}
    shapes = {}
    for item in filter(None, args.shape.split(",")):
        name, v, c = item.split(":")
        S.stokes_set_pair_shape(G.handle, kinds[name][0], int(v), int(c))
        shapes[name] = (int(v), int(c))
    for name in args.precisions.split(","):
        prec, kind, kname = kinds[name]
        for _ in range(args.warmup):
            S.stokes_matvec(G.handle, sig, y, prec)
        torch.cuda.synchronize()
        S.stokes_profile_enable(G.handle, True)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.reps):
            S.stokes_matvec(G.handle, sig, y, prec)
        ev1.record(stream)
        torch.cuda.synchronize()
        n, ms, pairs = S.stokes_profile_read(G.handle, kind)
        ne, mse, _ = S.stokes_profile_read(G.handle, S.STOKES_PROF_EPILOGUE)
        S.stokes_profile_enable(G.handle, False)
        avg = ms / n
        gp = pairs / n / (avg * 1e-3)
        v, c = S.stokes_get_pair_shape(G.handle, prec, geom.n_nodes)
        print(json.dumps({"kernel": kname, "precision": name, "workload": workload_config(args.workload)["workload"],
                          "shape": {"variant": v, "threads_tpt_tile": S.stokes_pair_shape_info(prec, v),
                                    "ctas_per_sm": c},
                          "matvec_ms": round(ev0.elapsed_time(ev1) / args.reps, 3),
                          "pair_kernel_ms": round(avg, 3), "epilogue_ms": round(mse / max(ne, 1), 3),
                          "gpairs_per_s": round(gp / 1e9, 1),
                          "tflops_18_per_pair": round(FLOPS_PER_PAIR * gp / 1e12, 3)}), flush=True)
    G.close()


def batch_workload(n):
    """Uneven batch of porous pipes: pore counts uniform in [20, 120], 64 or
    128 nodes per pore, 1024 or 2048 wall nodes (the batch configuration's
    shape, scaled down so that every geometry's block-diagonal setup and
    dense oracle checks stay small)."""
    import stokes_inputs as si
    return [si.cached_geometry(f"batchsmall{i}", 0) for i in range(n)]


def batch_bench(args):
    """Batched operator (all geometries x 4 right-hand sides in one
    persistent launch) against the single-geometry kernels, and the lockstep
    mixed-precision solve against one solve per system."""
    import torch
    import paper_1609_04484_gb300 as S
    import stokes_inputs as si
    world, rank, local, pg = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    geoms = batch_workload(args.batch_geoms)
    if world > 1:  # independent geometries: each rank solves its share, no collective on the data path
        from paper_1609_04484_gb300.replicas import shard_by_cost
        geoms = [geoms[i] for i in shard_by_cost([g.n_nodes ** 2 for g in geoms], world, rank)]
    R = 4
    Gs = [S.Geometry(g, stream=stream.cuda_stream) for g in geoms]
    hs = [G.handle for G in Gs]
    for G in Gs:
        S.stokes_precond_setup_twogrid(G.handle, args.coarsen)
    sig = [torch.tensor(si.random_density(g, r).reshape(-1), device=dev) for g in geoms for r in range(R)]
    ys = [torch.empty_like(x) for x in sig]
    pairs = float(sum(g.n_nodes ** 2 for g in geoms)) * R
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    cfg = {"workload": f"{len(geoms)} porous pipes x {R} right-hand sides (pores 20-120, 64/128 nodes per pore, "
                       f"1024/2048 wall nodes)", "nodes": [g.n_nodes for g in geoms]}
    for name, prec in (("fp32", S.STOKES_FP32), ("df64", S.STOKES_DF64)):
        for _ in range(max(1, args.warmup)):
            S.stokes_batch_matvec(hs, R, sig, ys, prec)
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.reps):
            S.stokes_batch_matvec(hs, R, sig, ys, prec)
        ev1.record(stream)
        torch.cuda.synchronize()
        t_batch = ev0.elapsed_time(ev1) / args.reps
        ev0.record(stream)
        for _ in range(args.reps):
            for k, G in enumerate(Gs):
                for r in range(R):
                    S.stokes_matvec(G.handle, sig[k * R + r], ys[k * R + r], prec)
        ev1.record(stream)
        torch.cuda.synchronize()
        t_single = ev0.elapsed_time(ev1) / args.reps
        print(json.dumps({"batch_operator": name, "config": cfg["workload"], "pair_rhs_per_launch": pairs,
                          "batch_ms": round(t_batch, 3), "one_call_per_system_ms": round(t_single, 3),
                          "gpairs_rhs_per_s": round(pairs / (t_batch * 1e-3) / 1e9, 1),
                          "speedup": round(t_single / t_batch, 2)}), flush=True)
    fs = []
    for g in geoms:
        fs += [torch.tensor(b.reshape(-1), device=dev) for b in
               (si.pipe_bc(g), si.reversed_pipe_bc(g), si.outer_shear_bc(g), si.stokeslet_rotlet_bc(g, 0))]
    for attempt in range(2):  # the first call also captures the cycle graph
        xs = [torch.zeros_like(f) for f in fs]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        iters, relres, status = S.stokes_batch_solve(hs, R, fs, xs, tol=args.tol, restart=100, max_iter=3000,
                                                     precision=S.STOKES_MIXED_IR)
        torch.cuda.synchronize()
        t_batch = time.perf_counter() - t0
    t0 = time.perf_counter()
    it_single = []
    for k, G in enumerate(Gs):
        for r in range(R):
            x1 = torch.zeros_like(fs[k * R + r])
            code, it, rr, _ = S.stokes_gmres_solve(G.handle, fs[k * R + r], x1, tol=args.tol, restart=100,
                                                   max_iter=3000, precision=S.STOKES_MIXED_IR)
            it_single.append(it)
    torch.cuda.synchronize()
    t_single = time.perf_counter() - t0
    print(json.dumps({"batch_solve": f"mixed (FP32 inner, FP64 outer), two-grid (q = {args.coarsen}), FGMRES(100)",
                      "config": cfg["workload"], "systems": len(fs), "tol": args.tol,
                      "batch_s": round(t_batch, 3), "one_solve_per_system_s": round(t_single, 3),
                      "speedup": round(t_single / t_batch, 2), "iters_max": max(iters),
                      "iters_mean": round(float(np.mean(iters)), 1), "single_iters_mean":
                      round(float(np.mean(it_single)), 1), "relres_max": max(relres),
                      "all_converged": all(s == S.STOKES_OK for s in status)}), flush=True)
    for G in Gs:
        G.close()


def main():
    args = parse_args()
    if args.batch_bench:
        batch_bench(args)
        return
    if args.kernel_bench:
        kernel_bench(args)
        return
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    world, rank, local, pg = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import paper_1609_04484_gb300 as S
    import stokes_inputs as si

    geom = si.cached_geometry(args.workload, 0)
    f_h = si.pipe_bc(geom).reshape(-1)
    T_h = si.interior_targets(geom, args.targets, min_dist=0.05, seed=3).reshape(-1)
    prec_name, restart, pc_name = solver_params(args)
    prec = {"mixed": S.STOKES_MIXED_IR, "df64": S.STOKES_DF64, "fp64": S.STOKES_FP64}[prec_name]
    vel_prec = S.STOKES_FP64 if prec_name == "fp64" else S.STOKES_DF64
    max_iter = args.max_iter
    tol = args.tol if args.workload == "pipe1000" else min(args.tol, 1e-10)

    d = lambda a: torch.tensor(np.ascontiguousarray(a).reshape(-1), dtype=torch.float64, device=dev)
    nodes, normals = d(geom.nodes), d(geom.normals)
    weights, curv = d(geom.weights), d(geom.curvature)
    centres = np.ascontiguousarray(geom.centres).reshape(-1)
    f = d(f_h)
    targets = d(T_h)
    sig = torch.zeros_like(f)
    u = torch.empty(T_h.size, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    sptr = stream.cuda_stream
    prof_acc = {}
    result = {}

    def run_step(profile=False, host=None):
        if host is None:
            arrs = (nodes, normals, weights, curv, f, sig, targets, u)
        else:
            arrs = host
        h = S.stokes_geometry_create(arrs[0], arrs[1], arrs[2], arrs[3], geom.offsets, geom.n_comp,
                                     geom.outer_comp, centres, sptr)
        try:
            if profile:
                S.stokes_profile_enable(h, True)
            if pc_name == "twogrid":
                S.stokes_precond_setup_twogrid(h, args.coarsen)
            else:
                S.stokes_precond_setup(h, S.STOKES_PC_BLOCKDIAG)
            arrs[5].zero_() if hasattr(arrs[5], "zero_") else arrs[5].fill(0.0)
            code, iters, rr, pr = S.stokes_gmres_solve(h, arrs[4], arrs[5], tol=tol, restart=restart,
                                                       max_iter=args.max_iter, precision=prec)
            S.stokes_eval_velocity(h, arrs[5], arrs[6], arrs[7], vel_prec)
            if profile:
                for kind in range(7):
                    n, ms, units = S.stokes_profile_read(h, kind)
                    a = prof_acc.setdefault(kind, [0, 0.0, 0.0])
                    a[0] += n
                    a[1] += ms
                    a[2] += units
            result.update(code=code, iters=iters, relres=rr)
        finally:
            S.stokes_geometry_destroy(h)

    # launch shapes of the pair kernels this solve uses, tuned once for the
    # workload's size class (kept in the library's process-wide cache)
    tuned = {}
    if not args.no_tune:
        h = S.stokes_geometry_create(nodes, normals, weights, curv, geom.offsets, geom.n_comp, geom.outer_comp,
                                     centres, sptr)
        try:
            for name, p in (("fp32", S.STOKES_FP32), ("df64", S.STOKES_DF64)):
                if prec_name in ("mixed",) and name == "df64":
                    continue
                if prec_name == "fp64":
                    continue
                v, c, ms = S.stokes_autotune(h, p, 2)
                tuned[name] = {"variant": v, "shape": S.stokes_pair_shape_info(p, v), "ctas_per_sm": c,
                               "ms": round(ms, 3)}
        finally:
            S.stokes_geometry_destroy(h)
    # warm-up
    for _ in range(args.warmup):
        run_step()
    torch.cuda.synchronize()
    if pg is not None:
        pg.barrier()
    launches0 = S.stokes_kernel_launches()
    clocks = ClockSampler(local)
    clocks.start()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        run_step(profile=True)
    ev1.record(stream)
    torch.cuda.synchronize()
    if pg is not None:
        pg.barrier()
    clk = clocks.stop()
    launches = S.stokes_kernel_launches() - launches0
    ms_step = ev0.elapsed_time(ev1) / args.steps
    if pg is not None:
        from paper_1609_04484_gb300.replicas import reduce_max
        ms_step = reduce_max(ms_step, device=dev)

    # end to end through the public API with host (pinned) buffers
    pin = lambda a: torch.tensor(np.ascontiguousarray(a).reshape(-1), dtype=torch.float64).pin_memory()
    host = (pin(geom.nodes), pin(geom.normals), pin(geom.weights), pin(geom.curvature), pin(f_h),
            torch.zeros(f_h.size, dtype=torch.float64).pin_memory(), pin(T_h),
            torch.empty(T_h.size, dtype=torch.float64).pin_memory())
    e2e_s = None
    if args.e2e_steps > 0:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            run_step(host=host)
            _ = host[7].numpy().sum()  # the result is read on the host
        e2e_s = (time.perf_counter() - t0) / args.e2e_steps
    h2d = 8 * (2 * geom.n_nodes * 2 + 2 * geom.n_nodes + f_h.size + f_h.size + T_h.size)
    d2h = 8 * (f_h.size + T_h.size)

    if rank != 0:
        return
    # roofline of the dominant pair kernel
    pair_kinds = {S.STOKES_PROF_PAIRS_FP64: ("k_dlp_pairs_f64", "fp64"),
                  S.STOKES_PROF_PAIRS_FP32: ("k_dlp_pairs_f32", "fp32"),
                  S.STOKES_PROF_PAIRS_DF64: ("k_dlp_pairs_df64", "df64")}
    dom = max(pair_kinds, key=lambda k: prof_acc.get(k, [0, 0.0, 0.0])[1])
    n_l, ms_l, pairs_l = prof_acc[dom]
    avg_ms = ms_l / max(n_l, 1)
    pairs_per_launch = pairs_l / max(n_l, 1)
    achieved = FLOPS_PER_PAIR * pairs_per_launch / (avg_ms * 1e-3) / 1e12
    kname, kp = pair_kinds[dom]
    gps = pairs_per_launch / (avg_ms * 1e-3)
    issue_peak = SM_COUNT * FP32_LANES_PER_SM * SM_MAX_MHZ * 1e6 / 1e12   # T FP32-pipe ops/s
    if kp == "fp64":
        roofline = {"bound": "alu", "kernel": kname, "achieved": round(achieved, 3),
                    "peak": FP64_NOMINAL_TFLOPS, "unit": "TFLOP/s", "frac": round(achieved / FP64_NOMINAL_TFLOPS, 4),
                    "peak_source": "nominal dense FP64 of the part (1.25 TFLOP/s)"}
    else:
        ops = DF64_OPS_PER_PAIR if kp == "df64" else F32_OPS_PER_PAIR
        ach = ops * gps / 1e12
        roofline = {"bound": "alu", "kernel": kname, "achieved": round(ach, 3), "peak": round(issue_peak, 2),
                    "unit": "T FP32-pipe ops/s", "frac": round(ach / issue_peak, 4),
                    "ops_per_pair": ops,
                    "peak_source": "FP32 pipes: 152 SMs x 128 lanes x 2070 MHz, one op per lane per clock",
                    "fp64_class_tflops_at_18_flops_per_pair": round(achieved, 3)}
    traffic = None
    if args.workload == "pipe1000" and kp in tuned:
        traffic = MEASURED_TRAFFIC.get((kname, *tuned[kp]["shape"]))
    roofline.update({"traffic": traffic, "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum, "
                     "one capture of this kernel shape on this workload" if traffic else None,
                     "gpairs_per_s": round(gps / 1e9, 2), "avg_launch_ms": round(avg_ms, 4),
                     "launches": n_l, "flops_per_pair": FLOPS_PER_PAIR})
    phases = {}
    names = {0: "pairs_fp64", 1: "pairs_fp32", 2: "pairs_df64", 3: "epilogue", 4: "bd_apply", 5: "arnoldi",
             6: "bd_setup"}
    for k, (n, ms, units) in prof_acc.items():
        if n:
            phases[names[k]] = {"launches": n, "ms": round(ms / args.steps, 2)}
    cfg = workload_config(args.workload)
    cfg.update({"precision": prec_name, "restart": restart, "targets": args.targets,
                "pc": {"bd": "block-diagonal (right)",
                       "twogrid": f"two-grid, coarse = every {args.coarsen}th node (flexible GMRES, right)"}[pc_name],
                "l2": "working set (block inverses and factors > 2.6 GB, Krylov basis) exceeds L2; no flush",
                "pair_shapes": tuned or "defaults",
                "parallelism": f"replicas x{world}"})
    value = ms_step / 1e3
    line = {"metric": METRIC, "value": round(value, 4), "unit": "s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_step, 2), "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None,
            "dtype": {"mixed": "f32 inner / f64 outer", "df64": "df64 (float pairs), f64 residuals",
                      "fp64": "f64"}[prec_name],
            "data": "synthetic", "config": cfg,
            "solve": {"iters": result.get("iters"), "true_relres": result.get("relres"),
                      "status": result.get("code"), "solves_per_s_all_gpus": round(world / value, 4)},
            "phases_ms_per_step": phases, "roofline": roofline, "clocks": clk, "gpu_launches": launches,
            "e2e": ({"value": round(e2e_s, 4), "unit": "s", "h2d_bytes_per_step": h2d,
                     "d2h_bytes_per_step": d2h} if e2e_s is not None else None)}
    if not args.no_cpu_baseline and world == 1:
        iters = result.get("iters") or 1
        ob = oracle_sample(geom, iters, budget_s=15.0)
        line["cpu_baseline"] = {"value": round(ob["est_time_to_solution_s"], 1), "unit": "s",
                                "cores": ob["cores"], "kind": "oracle",
                                "sample": f"{ob['sample_rows']} random rows of A sigma (numpy FP64, "
                                          f"{ob['pairs_per_s']/1e6:.1f} Mpairs/s) in {ob['sample_s']:.1f} s, "
                                          f"extrapolated to {iters} full operator applications"}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()

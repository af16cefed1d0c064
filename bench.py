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
LU_PANEL_TC = 128  # panel width of the coarse LU with tensor-core trailing updates (8192 rows and up)
# DRAM bytes (read + write) per launch of a kernel on the 136,192-node
# workload, from one ncu capture of that kernel shape (the summaries are kept
# with the profiles); keyed by (kernel, threads, targets per thread, tile). A
# kernel or shape not listed, or changed since its capture, reports null.
MEASURED_TRAFFIC = {("k_dlp_pairs_df64", 256, 1, 256): 9828608.0,
                    ("k_dlp_pairs_f32", 256, 4, 256): 7642624.0}
# DRAM bytes per algorithmic byte of a kernel whose launches differ in size,
# from ncu captures of launches of this workload (k_tc_trailing: the first
# trailing updates of the 136,192-node step); the traffic of an average
# launch is this ratio times its algorithmic bytes. Empty: not captured as the
# kernel now stands
MEASURED_TRAFFIC_RATIO = {"k_tc_trailing": 1.02}


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
    p.add_argument("--no-batch-record", dest="batch_record", action="store_false",
                   help="skip the 64-geometry batched sub-record (about 2 minutes)")
    p.add_argument("--no-sub-records", dest="sub_records", action="store_false",
                   help="skip the other configurations' records (measured once after the timed region)")
    p.add_argument("--coarse-train", type=int, default=2000,
                   help="training geometries of the learned coarse correction's record (0: skip)")
    p.add_argument("--baseline-budget", type=float, default=150.0,
                   help="seconds for the plain FP64 block-diagonal GMRES baseline (0: skip)")
    p.add_argument("--no-tune", action="store_true", help="skip the pair kernels' launch-shape autotuner")
    p.add_argument("--kernel-bench", action="store_true",
                   help="time only operator applications (A sigma) of each precision on the workload")
    p.add_argument("--batch-bench", action="store_true",
                   help="time the batched operator and lockstep solve on a multi-geometry batch")
    p.add_argument("--coarse-bench", action="store_true",
                   help="time the two-grid coarse LU kernels alone on a small case (used for ncu captures)")
    p.add_argument("--batch-geoms", type=int, default=16)
    p.add_argument("--batch-set", default="small", choices=["small", "config4"],
                   help="batch bench geometries: the 16-geometry small batch or the 64-geometry subset of the "
                        "batched configuration")
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
# CPU oracle legs (the only code here that runs the oracle)
# ---------------------------------------------------------------------------

def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _rows_worker(args):
    """One worker of the all-core oracle sample: random rows of A sigma for
    `budget_s` seconds; returns (rows, seconds)."""
    name, seed, budget_s = args
    import oracle
    import stokes_inputs as si
    geom = si.cached_geometry(name, 0)
    sig = si.random_density(geom, 2).reshape(-1)
    rng = np.random.default_rng(seed)
    rows = 0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < budget_s:
        rr = rng.choice(geom.n_nodes, 64, replace=False)
        oracle.apply_rows(geom, sig, rr)
        rows += rr.size
    return rows, time.perf_counter() - t0


def cpu_baseline_operator_rate(name, budget_s):
    """The oracle's matrix-free operator rows (numpy FP64) on every host
    core (a process pool started with spawn, one single-threaded numpy per
    worker) for `budget_s` seconds: returns the oracle's pair rate and the
    time of one full operator application A sigma it implies."""
    import multiprocessing as mp
    import stokes_inputs as si
    n_nodes = si.cached_geometry(name, 0).n_nodes  # generated once, before the workers read the cache
    cores = host_cores()
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    try:
        with mp.get_context("spawn").Pool(cores) as pool:
            t0 = time.perf_counter()
            res = pool.map(_rows_worker, [(name, 1000 + c, budget_s) for c in range(cores)])
            wall = time.perf_counter() - t0
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    rows = sum(r for r, _ in res)
    busy = max(t for _, t in res)
    pairs_per_s = rows * n_nodes / busy
    return {"pairs_per_s": pairs_per_s, "rows": rows, "cores": cores, "busy_s": busy, "wall_s": wall,
            "matvec_s": n_nodes ** 2 / pairs_per_s}


def cpu_baseline_small_solve(geom, f, tol, restart):
    """The oracle's own plain method solved for real on a small geometry:
    dense assembly, block-diagonal LU, right-preconditioned GMRES(restart)
    to `tol`; also its dense LU solution (the FP64 reference the GPU results
    are compared with)."""
    import oracle
    t0 = time.perf_counter()
    r = oracle.solve_gmres(geom, f, tol=tol, restart=restart, max_iter=5000, precond="bd")
    t_solve = time.perf_counter() - t0
    t0 = time.perf_counter()
    x_dense = oracle.solve_dense(geom, f)
    t_dense = time.perf_counter() - t0
    return {"gmres_s": t_solve, "iters": r["iters"], "relres": r["relres"], "x": r["x"],
            "dense_lu_s": t_dense, "x_dense": x_dense}


def cpu_baseline_dense_solution(geom, f):
    import oracle
    return oracle.solve_dense(geom, f)


def cpu_baseline_velocity(geom, sigma, targets):
    import oracle
    return oracle.velocity(geom, sigma, targets)


def run_reference(args):
    """The oracle timed on the host cores (rank 0 only). The 1152-node
    workload is solved for real each step; for the 136,192-node workload a
    step is a bounded all-core sample of the oracle's operator rows, scaled
    to the operator applications of the two-grid flexible GMRES solve (the
    same method as the GPU arm; the oracle's coarse setup is not counted, so
    the value is an estimate and a lower bound)."""
    world, rank, local, pg = dist_setup(args)
    if rank != 0:
        return
    import stokes_inputs as si
    geom = si.cached_geometry(args.workload, 0)
    f = si.pipe_bc(geom).reshape(-1)
    cfg = workload_config(args.workload)
    times = []
    info = None
    per_step = max(2.0, min(15.0, 150.0 / max(1, args.warmup + args.steps)))
    applications = int(os.environ.get("STOKES_REF_APPLICATIONS", "25"))
    for s in range(args.warmup + args.steps):
        if args.workload == "pipe10":
            r = cpu_baseline_small_solve(geom, f, tol=1e-10, restart=50)
            t = r["gmres_s"]
            info = {"cores": 1, "sample": f"full oracle solve: dense assembly, block-diagonal LU, GMRES(50) to "
                                          f"1e-10 ({r['iters']} iterations, numpy FP64, one core)",
                    "estimate": False}
        else:
            o = cpu_baseline_operator_rate(args.workload, per_step)
            t = applications * o["matvec_s"]
            info = {"cores": o["cores"],
                    "sample": f"{o['rows']} random rows of A sigma on {o['cores']} cores in {o['busy_s']:.1f} s "
                              f"(numpy FP64, {o['pairs_per_s'] / 1e6:.1f} Mpairs/s): one operator application "
                              f"{o['matvec_s']:.1f} s, times the {applications} applications of the two-grid "
                              f"flexible GMRES solve",
                    "estimate": True}
        if s >= args.warmup:
            times.append(t)
    v = float(np.mean(times))
    line = {"metric": METRIC, "value": v, "unit": "s", "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": v, "unit": "s", "cores": info["cores"], "kind": "oracle",
                             "sample": info["sample"], "estimate": info["estimate"]},
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    if info["estimate"]:
        line["estimate_note"] = ("value is the oracle's time scaled from a bounded sample, not a timed solve: "
                                 "each step ran for about %.0f s" % per_step)
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


def coarse_bench(args):
    """The two-grid preconditioner's coarse LU kernels alone on a small case
    (the entry point of the ncu captures of the tensor-core trailing update,
    the panel factorisation and the coarse triangular solve): a porous pipe
    of 120 pores x 64 nodes and a 4096-node wall (11,776 nodes; coarse
    operator of every 2nd node, 11,776 rows, 0.55 GB of float factors, more
    than the L2 cache), `--reps` setups and `--reps` x 10 applies, with
    the library's CUDA-event timing per kernel class."""
    import torch
    import paper_1609_04484_gb300 as S
    import stokes_inputs as si
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    g = si.batch_geometry(3, n_pores=120, n_per_pore=64, n_outer=4096)
    v = torch.tensor(si.random_density(g, 1).reshape(-1), device=dev)
    z = torch.empty_like(v)
    G = S.Geometry(g, stream=stream.cuda_stream)
    try:
        S.stokes_precond_setup_twogrid_ex(G.handle, 2, S.STOKES_TG_COARSE_LU)  # warm-up
        S.stokes_precond_apply(G.handle, v, z)
        torch.cuda.synchronize()
        S.stokes_profile_enable(G.handle, True)
        for _ in range(args.reps):
            S.stokes_precond_setup_twogrid_ex(G.handle, 2, S.STOKES_TG_COARSE_LU)
            for _ in range(10):
                S.stokes_precond_apply(G.handle, v, z)
        torch.cuda.synchronize()
        m = g.n_nodes
        rec = {"case": "coarse LU of a 11,776-node pipe (every 2nd node: 11,776 rows)", "reps": args.reps}
        for kind, name in ((S.STOKES_PROF_LU_GEMM, "lu_gemm"), (S.STOKES_PROF_LU_PANEL, "lu_panel"),
                           (S.STOKES_PROF_COARSE_SOLVE, "coarse_solve")):
            n, ms, units = S.stokes_profile_read(G.handle, kind)
            rec[name] = {"launches": n, "ms_total": round(ms, 3), "ms_per_launch": round(ms / max(n, 1), 4)}
            if name == "lu_gemm":
                rec[name]["tflops"] = round(units / (ms * 1e-3) / 1e12, 2)
            if name == "coarse_solve":
                rec[name]["gbs"] = round(units / (ms * 1e-3) / 1e9, 1)
                rec[name]["bytes_per_apply"] = 4.0 * m * m
        print(json.dumps(rec), flush=True)
    finally:
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


def batch_config4_record(args, S, torch, dev, stream):
    """The batched configuration on a subset: 64 geometries (pores uniform in
    [50, 200] instead of [50, 800]; 64/128/256 nodes per pore; 2048/4096/8192
    wall nodes) x 4 right-hand sides (pipe, reversed pipe, wall shear,
    Stokeslet/rotlet data), two-grid preconditioners (every 4th node, float
    explicit coarse inverses), all 256 systems solved by the lockstep
    mixed-precision flexible GMRES(100) to 1e-8 (FP32 batched operator in one
    persistent launch per step, FP64 residuals; the cycle is a captured CUDA
    graph). Timed on the host around synchronised calls, once per run."""
    import stokes_inputs as si
    t0 = time.perf_counter()
    geoms = generate_geometries("batch_config4_geometry", range(64))
    gen_s = time.perf_counter() - t0
    R = 4
    free0 = torch.cuda.mem_get_info(dev)[0]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Gs = [S.Geometry(g, stream=stream.cuda_stream) for g in geoms]
    hs = [G.handle for G in Gs]
    try:
        for G in Gs:
            S.stokes_precond_setup_twogrid_ex(G.handle, 4, S.STOKES_TG_COARSE_INVERSE)
        torch.cuda.synchronize()
        setup_s = time.perf_counter() - t0
        mem_gb = (free0 - torch.cuda.mem_get_info(dev)[0]) / 1e9
        fs = []
        for g in geoms:
            fs += [torch.tensor(b.reshape(-1), device=dev) for b in
                   (si.pipe_bc(g), si.reversed_pipe_bc(g), si.outer_shear_bc(g), si.stokeslet_rotlet_bc(g, 0))]
        pairs = float(sum(g.n_nodes ** 2 for g in geoms)) * R
        ys = [torch.empty_like(f) for f in fs]
        S.stokes_batch_matvec(hs, R, fs, ys, S.STOKES_FP32)
        a, b = _events(torch, stream)
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(3):
            S.stokes_batch_matvec(hs, R, fs, ys, S.STOKES_FP32)
        b.record(stream)
        torch.cuda.synchronize()
        op_ms = a.elapsed_time(b) / 3
        out = None
        for attempt in range(2):  # the first call also captures the cycle graph
            xs = [torch.zeros_like(f) for f in fs]
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            iters, relres, status = S.stokes_batch_solve(hs, R, fs, xs, tol=1e-8, restart=100, max_iter=3000,
                                                         precision=S.STOKES_MIXED_IR)
            torch.cuda.synchronize()
            out = (time.perf_counter() - t0, iters, relres, status)
        solve_s, iters, relres, status = out
    finally:
        for G in Gs:
            G.close()
    return {"workload": "64 porous pipes x 4 right-hand sides: pores 50-200 (stated: 50-800), 64/128/256 nodes "
                        "per pore, 2048/4096/8192 wall nodes",
            "nodes_min_max": [int(min(g.n_nodes for g in geoms)), int(max(g.n_nodes for g in geoms))],
            "systems": len(fs), "pc": "two-grid, every 4th node, float explicit coarse inverses",
            "solver": "lockstep flexible GMRES(100), FP32 inner / FP64 outer, tol 1e-8",
            "generate_s": round(gen_s, 1), "setup_s": round(setup_s, 2), "preconditioner_gb": round(mem_gb, 1),
            "batched_operator_ms": round(op_ms, 2),
            "batched_operator_gpairs_rhs_per_s": round(pairs / (op_ms * 1e-3) / 1e9, 1),
            "solve_s": round(solve_s, 2), "iters_mean": round(float(np.mean(iters)), 1), "iters_max": int(max(iters)),
            "true_relres_max": float(max(relres)), "converged": int(sum(st == S.STOKES_OK for st in status))}


def main():
    args = parse_args()
    if args.batch_bench:
        if args.batch_set == "config4":
            import torch
            import paper_1609_04484_gb300 as S
            dev = torch.device("cuda", 0)
            print(json.dumps(batch_config4_record(args, S, torch, dev, torch.cuda.current_stream(dev))), flush=True)
        else:
            batch_bench(args)
        return
    if args.kernel_bench:
        kernel_bench(args)
        return
    if args.coarse_bench:
        coarse_bench(args)
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
                for kind in range(10):
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
    prof_acc["_steps"] = args.steps
    # full operator applications per step, from the pair work the library
    # recorded (the velocity's 4096 targets add a small fraction)
    pair_units = sum(prof_acc.get(k, [0, 0.0, 0.0])[2] for k in (0, 1, 2))
    result["applications"] = int(round(pair_units / args.steps / float(geom.n_nodes) ** 2))
    peaks = measured_peaks()
    rooflines = kernel_rooflines(S, prof_acc, peaks)
    dom = max(rooflines, key=lambda r: r["ms_per_step"] if r["candidate"] else -1.0)
    roofline = dict(dom)
    roofline.pop("candidate", None)
    traffic, source = dom.get("traffic"), dom.get("traffic_source")
    if traffic is None and args.workload == "pipe1000":
        key = (dom["kernel"],) + tuple(tuned.get(dom.get("precision"), {}).get("shape", ()))
        traffic = MEASURED_TRAFFIC.get(key)
        source = ("ncu dram__bytes_read.sum + dram__bytes_write.sum, one capture of this kernel shape on this "
                  "workload" if traffic else "no ncu capture of this kernel as it now stands")
    roofline["traffic"] = traffic
    roofline["traffic_source"] = source
    phases = {}
    for k, (n, ms, units) in ((k, v) for k, v in prof_acc.items() if isinstance(k, int)):
        if n:
            phases[PROF_NAMES[k]] = {"launches": n, "ms": round(ms / args.steps, 2)}
    cfg = workload_config(args.workload)
    cfg.update({"precision": prec_name, "restart": restart, "targets": args.targets,
                "pc": {"bd": "block-diagonal (right)",
                       "twogrid": f"two-grid, coarse = every {args.coarsen}th node (flexible GMRES, right)"}[pc_name],
                "l2": "working set (coarse factors, block inverses, Krylov basis) exceeds L2; no flush",
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
            "phases_ms_per_step": phases, "roofline": roofline,
            "kernels": [{k: v for k, v in r.items() if k != "candidate"} for r in rooflines],
            "clocks": clk, "gpu_launches": launches,
            "e2e": ({"value": round(e2e_s, 4), "unit": "s", "h2d_bytes_per_step": h2d,
                     "d2h_bytes_per_step": d2h} if e2e_s is not None else None)}
    if not args.no_cpu_baseline and world == 1:
        o = cpu_baseline_operator_rate(args.workload, 15.0)
        apps = result.get("applications") or (result.get("iters") or 0) + 2
        line["cpu_baseline"] = {
            "value": round(apps * o["matvec_s"], 1), "unit": "s", "cores": o["cores"], "kind": "oracle",
            "estimate": True,
            "sample": f"{o['rows']} random rows of A sigma on {o['cores']} host cores in {o['busy_s']:.1f} s "
                      f"(numpy FP64, {o['pairs_per_s'] / 1e6:.1f} Mpairs/s): one operator application "
                      f"{o['matvec_s']:.1f} s, times the {apps} operator applications of this two-grid flexible "
                      f"GMRES solve (same method; the oracle's coarse setup not counted: a lower bound)"}
    if args.sub_records and world == 1 and args.workload == "pipe1000":
        line["sub_records"] = sub_records(args, S, torch, dev, stream)
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# Roofline of each kernel class timed inside the step
# ---------------------------------------------------------------------------

PROF_NAMES = {0: "pairs_fp64", 1: "pairs_fp32", 2: "pairs_df64", 3: "epilogue", 4: "precond_apply",
              5: "arnoldi", 6: "precond_setup", 7: "lu_gemm", 8: "lu_panel", 9: "coarse_solve"}
FP32_FLOP_PEAK = SM_COUNT * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12   # TFLOP/s, FMA = 2
FP32_ISSUE_PEAK = SM_COUNT * FP32_LANES_PER_SM * SM_MAX_MHZ * 1e6 / 1e12     # T FP32-pipe ops/s
TF32_PER_BF16 = 1.1 / 2.25   # nominal dense TF32 / BF16 tensor rates of the part


def measured_peaks():
    """MEASURED_PEAKS.json (driver-written on this pool), else the profiling
    recipe's fallback figures."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return {"hbm_gbs": float(d["hbm_gbs"]), "bf16_tflops": float(d["bf16_tflops"]),
                "bf16_tflops_sustained": float(d.get("bf16_tflops_sustained", d["bf16_tflops"])),
                "source": "of measured (MEASURED_PEAKS.json)"}
    except (OSError, KeyError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "source": "of fallback (profiling recipe)"}


def kernel_rooflines(S, prof_acc, peaks):
    """One entry per kernel class with recorded launches: its share of the
    step and its algorithmic work per launch against the bound that limits
    it. Pair kernels: 18 flop per pair (FMA = 2) against the FP32 CUDA-core
    FLOP peak (152 SMs x 128 lanes x 2 x 2070 MHz = 80.5 TFLOP/s) and, for
    the FP64-class kernels, the multiple of the part's nominal FP64 rate;
    the double-float kernel's FP32-pipe issue use is kept separately. The
    coarse LU's trailing updates (tensor cores): the bytes of C read and
    written per launch (8 rest^2) against the HBM copy bandwidth, with the
    tensor pipe's issued TF32 rate beside (on the CUDA-core GEMM: 2 M N K
    flop against the FP32 peak). The coarse solve: bytes of the factors read
    per apply against the HBM copy bandwidth."""
    out = []
    steps = max(1, prof_acc.get("_steps", 1))
    for kind, (n, ms, units) in sorted((k, v) for k, v in prof_acc.items() if isinstance(k, int)):
        if n == 0 or ms <= 0:
            continue
        name = PROF_NAMES[kind]
        sec = ms * 1e-3
        r = {"class": name, "launches": n, "ms_per_step": round(ms / steps, 2), "avg_launch_ms": round(ms / n, 4),
             "candidate": kind not in (S.STOKES_PROF_BD_APPLY, S.STOKES_PROF_BD_SETUP)}
        if kind in (S.STOKES_PROF_PAIRS_FP64, S.STOKES_PROF_PAIRS_FP32, S.STOKES_PROF_PAIRS_DF64):
            gps = units / sec
            ach = FLOPS_PER_PAIR * gps / 1e12
            kname = {0: "k_dlp_pairs_f64", 1: "k_dlp_pairs_f32", 2: "k_dlp_pairs_df64"}[kind]
            r.update({"kernel": kname, "precision": {0: "fp64", 1: "fp32", 2: "df64"}[kind], "bound": "alu",
                      "achieved": round(ach, 3), "peak": round(FP32_FLOP_PEAK, 2), "unit": "TFLOP/s",
                      "frac": round(ach / FP32_FLOP_PEAK, 4), "gpairs_per_s": round(gps / 1e9, 2),
                      "flops_per_pair": FLOPS_PER_PAIR,
                      "peak_source": "FP32 CUDA cores: 152 SMs x 128 lanes x 2 flop x 2070 MHz (derived)"})
            if kind != S.STOKES_PROF_PAIRS_FP32:
                r["fp64_nominal_multiple"] = round(ach / FP64_NOMINAL_TFLOPS, 3)
            if kind == S.STOKES_PROF_PAIRS_DF64:
                issue = DF64_OPS_PER_PAIR * gps / 1e12
                r["fp32_issue"] = {"achieved": round(issue, 2), "peak": round(FP32_ISSUE_PEAK, 2),
                                   "unit": "T FP32-pipe ops/s", "frac": round(issue / FP32_ISSUE_PEAK, 4),
                                   "ops_per_pair": DF64_OPS_PER_PAIR}
        elif kind == S.STOKES_PROF_LU_GEMM:
            flops = units / sec
            if os.environ.get("STOKES_TG_GEMM", "") == "simt":
                r.update({"kernel": "k_sgemm128", "bound": "alu", "achieved": round(flops / 1e12, 2),
                          "peak": round(FP32_FLOP_PEAK, 2), "unit": "TFLOP/s",
                          "frac": round(flops / 1e12 / FP32_FLOP_PEAK, 4),
                          "peak_source": "FP32 CUDA cores (derived)"})
            else:
                # rank-kb updates (kb = 128: 128-column panels from 8192 coarse
                # rows on): each launch reads and writes its rest x rest block
                # of C once (8 bytes per entry per 2 kb flops)
                gbs = units / (2.0 * LU_PANEL_TC) * 8.0 / sec / 1e9
                tf32_peak = peaks["bf16_tflops"] * TF32_PER_BF16
                r.update({"kernel": "k_tc_trailing", "bound": "hbm", "achieved": round(gbs, 1),
                          "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": round(gbs / peaks["hbm_gbs"], 4),
                          "peak_source": peaks["source"],
                          "algorithmic_bytes": "8 rest^2 per launch (C read and written; the rest x 128 operands "
                                               "come from L2)",
                          "traffic": (round(MEASURED_TRAFFIC_RATIO["k_tc_trailing"] * units / (2.0 * LU_PANEL_TC)
                                            * 8.0 / max(n, 1)) if "k_tc_trailing" in MEASURED_TRAFFIC_RATIO
                                      else None),
                          "traffic_source": ("ncu DRAM bytes / algorithmic bytes of the first launches of this "
                                             "workload's step, times the average launch's algorithmic bytes"
                                             if "k_tc_trailing" in MEASURED_TRAFFIC_RATIO else
                                             "no ncu capture of this kernel as it now stands"),
                          "tensor": {"useful_tflops": round(flops / 1e12, 2),
                                     "issued_tflops": round(3 * flops / 1e12, 2),
                                     "tf32_peak": round(tf32_peak, 1),
                                     "frac_issued": round(3 * flops / 1e12 / tf32_peak, 4),
                                     "peak_source": "measured bf16 peak x 1.1 / 2.25 (nominal TF32 / BF16)"}})
        elif kind in (S.STOKES_PROF_COARSE_SOLVE, S.STOKES_PROF_BD_APPLY, S.STOKES_PROF_ARNOLDI):
            gbs = units / sec / 1e9
            kname = {S.STOKES_PROF_COARSE_SOLVE: "k_lu_solve_flags", S.STOKES_PROF_BD_APPLY: "(preconditioner apply)",
                     S.STOKES_PROF_ARNOLDI: "k_dot_partial + k_orth_update"}[kind]
            r.update({"kernel": kname, "bound": "hbm", "achieved": round(gbs, 1), "peak": peaks["hbm_gbs"],
                      "unit": "GB/s", "frac": round(gbs / peaks["hbm_gbs"], 4), "peak_source": peaks["source"]})
        elif kind == S.STOKES_PROF_LU_PANEL:
            r.update({"kernel": "k_panel_lu32", "bound": "latency", "achieved": round(units / sec, 1),
                      "unit": "columns/s", "note": "one grid barrier per column"})
        else:
            r.update({"kernel": name})
        out.append(r)
    return out


# ---------------------------------------------------------------------------
# Sub-records: the other configurations, measured once per run after the
# timed region (each with its own timing and its error against the oracle)
# ---------------------------------------------------------------------------

def _events(torch, stream):
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def _handle(S, geom, dev, torch, sptr):
    d = lambda a: torch.tensor(np.ascontiguousarray(a).reshape(-1), dtype=torch.float64, device=dev)
    return S.stokes_geometry_create(d(geom.nodes), d(geom.normals), d(geom.weights), d(geom.curvature),
                                    geom.offsets, geom.n_comp, geom.outer_comp,
                                    np.ascontiguousarray(geom.centres).reshape(-1), sptr)


def _rel(a, b):
    a = np.asarray(a).reshape(-1)
    b = np.asarray(b).reshape(-1)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def small_config_records(args, S, torch, dev, stream):
    """The 1152-node pipe (10 pores x 64 nodes + 512-node wall): the plain
    FP64 block-diagonal GMRES(50) solve to 1e-10, and the mixed-precision
    solve (FP32 inner GMRES(30), FP64 refinement to 1e-8). Each is timed on
    the device (handle, setup, solve, velocity at 4096 targets; mean of 5
    after 2 warm-ups) and compared with the oracle's dense FP64 solution and
    its velocity at the same targets."""
    import stokes_inputs as si
    geom = si.cached_geometry("pipe10", 0)
    f_h = si.pipe_bc(geom).reshape(-1)
    T_h = si.interior_targets(geom, 4096, min_dist=0.05, seed=3)
    sptr = stream.cuda_stream
    f = torch.tensor(f_h, device=dev)
    tg = torch.tensor(T_h.reshape(-1), device=dev)
    u = torch.empty(T_h.size, dtype=torch.float64, device=dev)
    ref = cpu_baseline_small_solve(geom, f_h, tol=1e-10, restart=50)
    u_ref = cpu_baseline_velocity(geom, ref["x_dense"], T_h)
    out = {}
    for name, prec, tol, restart in (("config1_fp64_block_diagonal", S.STOKES_FP64, 1e-10, 50),
                                     ("config3_mixed_fp32_inner_fp64_refinement", S.STOKES_MIXED_IR, 1e-8, 30)):
        times, res = [], None
        for rep in range(7):
            sig = torch.zeros_like(f)
            a, b = _events(torch, stream)
            torch.cuda.synchronize()
            a.record(stream)
            h = _handle(S, geom, dev, torch, sptr)
            try:
                S.stokes_precond_setup(h, S.STOKES_PC_BLOCKDIAG)
                res = S.stokes_gmres_solve(h, f, sig, tol=tol, restart=restart, max_iter=5000, precision=prec)
                S.stokes_eval_velocity(h, sig, tg, u, S.STOKES_FP64)
            finally:
                S.stokes_geometry_destroy(h)
            b.record(stream)
            torch.cuda.synchronize()
            if rep >= 2:
                times.append(a.elapsed_time(b))
        code, iters, relres, _ = res
        x = sig.cpu().numpy()
        out[name] = {"workload": "porous pipe, 10 pores x 64 nodes + 512-node wall (N=1152, 2304 unknowns)",
                     "method": ("block-diagonal GMRES(50), FP64" if prec == S.STOKES_FP64 else
                                "block-diagonal, FP32 inner GMRES(30) in FP64 iterative refinement"),
                     "tol": tol, "time_to_solution_s": round(float(np.mean(times)) / 1e3, 5),
                     "iters": iters, "true_relres": relres, "status": code,
                     "density_rel_err_vs_oracle": _rel(x, ref["x_dense"]),
                     "velocity_rel_err_vs_oracle_4096_targets": _rel(u.cpu().numpy(), u_ref),
                     "timing": "CUDA events around handle creation, setup, solve and velocity; mean of 5 after 2"}
    out["config1_cpu_oracle"] = {"gmres_s": round(ref["gmres_s"], 3), "iters": ref["iters"],
                                 "relres": ref["relres"], "dense_lu_s": round(ref["dense_lu_s"], 3), "cores": 1,
                                 "kind": "oracle",
                                 "sample": "full oracle solve (dense assembly, block-diagonal LU, GMRES(50) to 1e-10)"}
    return out


def plain_bd_baseline(args, S, torch, dev, stream):
    """Plain FP64 block-diagonal GMRES on the 136,192-node pipe (the paper's
    baseline preconditioner, Sec. 4.1; unrestarted, right-preconditioned,
    native FP64 operator). A 10-iteration pilot gives the time per
    iteration; the measured solve then runs to 1e-8 or until its iteration
    cap, chosen so that it takes about --baseline-budget seconds (at most
    2000 iterations, the paper's cap at 826 pores)."""
    import stokes_inputs as si
    geom = si.cached_geometry("pipe1000", 0)
    f = torch.tensor(si.pipe_bc(geom).reshape(-1), device=dev)
    sptr = stream.cuda_stream
    h = _handle(S, geom, dev, torch, sptr)
    try:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        S.stokes_precond_setup(h, S.STOKES_PC_BLOCKDIAG)
        torch.cuda.synchronize()
        setup_s = time.perf_counter() - t0
        sig = torch.zeros_like(f)
        t0 = time.perf_counter()
        S.stokes_gmres_solve(h, f, sig, tol=1e-8, restart=10, max_iter=10, precision=S.STOKES_FP64)
        torch.cuda.synchronize()
        per_iter = (time.perf_counter() - t0) / 10.0
        cap = int(max(10, min(2000, args.baseline_budget / per_iter)))
        sig.zero_()
        t0 = time.perf_counter()
        code, iters, relres, _ = S.stokes_gmres_solve(h, f, sig, tol=1e-8, restart=cap, max_iter=cap,
                                                      precision=S.STOKES_FP64)
        torch.cuda.synchronize()
        solve_s = time.perf_counter() - t0
    finally:
        S.stokes_geometry_destroy(h)
    return {"workload": workload_config("pipe1000")["workload"],
            "method": "block-diagonal (Sec. 4.1) right-preconditioned GMRES, unrestarted, FP64 operator",
            "setup_s": round(setup_s, 3), "solve_s": round(solve_s, 2), "iters": iters, "iteration_cap": cap,
            "true_relres": relres, "status": code, "converged": code == S.STOKES_OK,
            "s_per_iter": round(solve_s / max(1, iters), 4),
            "timing": "host clock around synchronised calls, measured once per run after the timed region"}


def _geometry_worker(args):
    import stokes_inputs as si
    fn, idx = args
    return getattr(si, fn)(idx)


def generate_geometries(fn_name, indices):
    """Input geometries drawn on every host core (a spawn pool: the GPU is
    already in use in this process)."""
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(host_cores()) as pool:
        return pool.map(_geometry_worker, [(fn_name, i) for i in indices], chunksize=8)


def learned_coarse_record(args, S, torch, dev, stream):
    """The learned coarse correction (the configuration's network: per-pore
    features, 35 -> 256 -> 256 -> 153, bf16 tensor-core kernels, Adam),
    trained on the GPU from the exact coarse inverses the solver computes
    for `--coarse-train` seeded training geometries, then evaluated on 100
    held-out 1152-node pipes against plain block-diagonal GMRES and the
    exact coarse level: iterations and time to 1e-8 (right-preconditioned
    GMRES, restart 300), each solve timed with CUDA events around handle
    creation, preconditioner setup and the solve."""
    import stokes_inputs as si
    sptr = stream.cuda_stream
    t0 = time.perf_counter()
    train = generate_geometries("coarse_train_geometry", range(args.coarse_train))
    held = generate_geometries("coarse_eval_geometry", range(100))
    gen_s = time.perf_counter() - t0
    model = S.stokes_coarse_model_create(si.mlp_initial_params(0), sptr)
    try:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for g in train:
            h = _handle(S, g, dev, torch, sptr)
            try:
                S.stokes_coarse_model_add_geometry(model, h)
            finally:
                S.stokes_geometry_destroy(h)
        torch.cuda.synchronize()
        data_s = time.perf_counter() - t0
        t0 = time.perf_counter()
        losses = [S.stokes_coarse_model_train(model, 1, 1e-3)]
        for steps, lr in ((1500, 1e-3), (1000, 3e-4), (500, 1e-4)):
            losses.append(S.stokes_coarse_model_train(model, steps, lr))
        train_s = time.perf_counter() - t0
        kinds = (("block_diagonal", S.STOKES_PC_BLOCKDIAG), ("exact_coarse", S.STOKES_PC_BD_COARSE),
                 ("learned_coarse", S.STOKES_PC_BD_LEARNED))
        res = {k: {"iters": [], "ms": [], "relres": [], "ok": 0} for k, _ in kinds}
        errs = {k: [] for k, _ in kinds}
        for gi, g in enumerate(held):
            f = torch.tensor(si.pipe_bc(g).reshape(-1), device=dev)
            x_ref = cpu_baseline_dense_solution(g, f.cpu().numpy()) if gi < 10 else None
            for name, kind in kinds:
                for rep in range(2):  # the first solve of each kind warms up
                    sig = torch.zeros_like(f)
                    a, b = _events(torch, stream)
                    torch.cuda.synchronize()
                    a.record(stream)
                    h = _handle(S, g, dev, torch, sptr)
                    try:
                        S.stokes_precond_setup(h, kind, model if kind == S.STOKES_PC_BD_LEARNED else None)
                        code, it, rr, _ = S.stokes_gmres_solve(h, f, sig, tol=1e-8, restart=300, max_iter=3000,
                                                               precision=S.STOKES_FP64)
                    finally:
                        S.stokes_geometry_destroy(h)
                    b.record(stream)
                    torch.cuda.synchronize()
                    if gi > 0 or rep == 1:
                        break
                r = res[name]
                r["iters"].append(it)
                r["ms"].append(a.elapsed_time(b))
                r["relres"].append(rr)
                r["ok"] += int(code == S.STOKES_OK)
                if x_ref is not None:
                    errs[name].append(_rel(sig.cpu().numpy(), x_ref))
    finally:
        S.stokes_coarse_model_destroy(model)
    summary = {}
    for name, r in res.items():
        summary[name] = {"iters_mean": round(float(np.mean(r["iters"])), 2), "iters_max": int(np.max(r["iters"])),
                         "time_to_solution_ms_mean": round(float(np.mean(r["ms"])), 3),
                         "true_relres_max": float(np.max(r["relres"])), "converged": r["ok"],
                         "density_rel_err_vs_oracle_max_first10": float(np.max(errs[name]))}
    bd = summary["block_diagonal"]
    for name in ("exact_coarse", "learned_coarse"):
        summary[name]["iteration_gain_vs_block_diagonal"] = round(1.0 - summary[name]["iters_mean"] / bd["iters_mean"], 4)
        summary[name]["time_gain_vs_block_diagonal"] = round(
            1.0 - summary[name]["time_to_solution_ms_mean"] / bd["time_to_solution_ms_mean"], 4)
    return {"training": {"geometries": len(train), "samples": int(sum(g.n_pores for g in train)),
                         "pores_per_geometry": [int(min(g.n_pores for g in train)), int(max(g.n_pores for g in train))],
                         "adam_steps": 3000, "loss_first_last": [losses[0], losses[-1]],
                         "generate_s": round(gen_s, 1), "coarse_inverses_s": round(data_s, 2),
                         "train_s": round(train_s, 2)},
            "evaluation": {"geometries": "100 held-out pipes, 10 pores x 64 nodes + 512-node wall (seeds 10000-10099)",
                           "solver": "right-preconditioned GMRES(300) to 1e-8, FP64 operator", **summary}}


def sub_records(args, S, torch, dev, stream):
    out = {}
    out.update(small_config_records(args, S, torch, dev, stream))
    if args.coarse_train > 0:
        out["config5_learned_coarse_correction"] = learned_coarse_record(args, S, torch, dev, stream)
    if args.baseline_budget > 0:
        out["baseline_plain_fp64_block_diagonal"] = plain_bd_baseline(args, S, torch, dev, stream)
    if args.batch_record:
        out["config4_batched_subset"] = batch_config4_record(args, S, torch, dev, stream)
    return out


if __name__ == "__main__":
    main()

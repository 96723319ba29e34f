#!/usr/bin/env python3
"""Benchmark: HISQ even-odd CG time to a 1e-10 true residual on one GB300, mixed precision vs
plain FP64, with the sloppy Dslash's HBM roofline fraction.

Workload (default): 32^3 x 8 lattice, seeded SU(3) links U = exp(i 0.5 H), fat = U,
long = -1/24 U U U, m = 0.01, one Gaussian source on even sites, tol 1e-10 on the
recomputed FP64 residual.  One step = one complete solve with inputs resident in HBM.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  N > 1 runs N independent replicas (one per GPU, launched
by torch.distributed.run); value is the max-over-ranks time per solve.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Dslash GB/s vs HBM peak; CG time to 1e-10 true residual vs plain FP64 CG"
WORKLOAD = "mixed-precision even-odd CG, 32^3x8, eps=0.5, m=0.01, 1 RHS, tol 1e-10"
DIMS, EPS, LINK_SEED, SRC_SEED, MASS, TOL = (32, 32, 32, 8), 0.5, 1001, 2100, 0.01, 1e-10
HBM_FALLBACK = 6800.0


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu, self.rows, self.proc = gpu, [], None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if len(r) > 5 + i and r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ------------------------------------------------------------------------------------- oracle
def oracle_sample(seconds_budget: float, fp64_iters: int):
    """Time the FP64 oracle's CG iterations on the host cores; scale to a full solve."""
    import numpy as np

    import oracle
    from hisq_inputs import fields
    threads = os.cpu_count() or 1
    oracle.set_threads(threads)
    fat, lng = fields.recipe_links(DIMS, EPS, LINK_SEED)
    b = fields.gaussian_source(DIMS, SRC_SEED)[0].numpy()
    fat, lng = fat.numpy(), lng.numpy()
    oracle.cg_fixed(DIMS, fat, lng, MASS, b, 1)            # warm
    done, t0 = 0, time.perf_counter()
    while True:
        oracle.cg_fixed(DIMS, fat, lng, MASS, b, 10)
        done += 10
        el = time.perf_counter() - t0
        if el >= seconds_budget or done >= 2000:
            break
    per_iter_ms = 1e3 * el / done
    return {"value": per_iter_ms * fp64_iters, "unit": "ms", "cores": threads, "kind": "oracle",
            "sample": f"{done} FP64 oracle CG iterations on 32^3x8 ({el:.1f} s, {threads} threads), "
                      f"scaled to the {fp64_iters} iterations of the GPU's plain FP64 solve",
            "per_iteration_ms": per_iter_ms}


def oracle_table():
    """--oracle-table: the FP64 oracle (OpenMP C) on the host cores with one thread and with all
    cores, one JSON line per row: full CG solves on 8^4 (eps 0.3, m 0.1) and on the 32^3 x 8
    solver workload (all cores; one thread: a 10-iteration sample scaled to the solve's
    iteration count), and the time per CG iteration on 64^3 x 16 (eps 0.3, m 0.01).  The thread
    count is set with omp_set_num_threads between the oracle's parallel regions."""
    import oracle
    from hisq_inputs import fields
    cores = os.cpu_count() or 1

    def emit(row):
        row.update({"kind": "oracle", "host_cores": cores})
        print(json.dumps(row), flush=True)

    for name, dims, eps, lseed, sseed, m, full in (
            ("8^4", (8, 8, 8, 8), 0.3, 1000, 2000, 0.1, "both"),
            ("32^3x8", DIMS, EPS, LINK_SEED, SRC_SEED, MASS, "all"),
            ("64^3x16", (64, 64, 64, 16), 0.3, 1002, 2200, 0.01, "none")):
        fat, lng = fields.recipe_links(dims, eps, lseed)
        fat, lng = fat.numpy(), lng.numpy()
        b = fields.gaussian_source(dims, sseed)[0].numpy()
        iters = None
        for threads in (cores, 1):
            oracle.set_threads(threads)
            if full == "both" or (full == "all" and threads == cores):
                t0 = time.perf_counter()
                _, iters, _, res = oracle.cg(dims, fat, lng, m, b, tol=TOL)
                el = time.perf_counter() - t0
                emit({"lattice": name, "threads": threads, "cg_ms": 1e3 * el, "iterations": iters,
                      "true_residual": res, "per_iteration_ms": 1e3 * el / iters})
            else:
                n = 10 if full == "all" else (3 if threads > 1 else 1)
                oracle.cg_fixed(dims, fat, lng, m, b, 1)  # warm
                t0 = time.perf_counter()
                oracle.cg_fixed(dims, fat, lng, m, b, n)
                per = 1e3 * (time.perf_counter() - t0) / n
                row = {"lattice": name, "threads": threads, "per_iteration_ms": per, "sample_iterations": n}
                if iters:
                    row.update({"cg_ms_extrapolated": per * iters, "iterations": iters})
                emit(row)
        del fat, lng, b
    oracle.set_threads(cores)


def run_reference(args, world, rank):
    """--impl reference: the FP64 oracle as it stands, on the host cores (rank 0 only)."""
    if rank != 0:
        return
    # iteration count of the FP64 solve: from one full oracle solve (untimed)
    import oracle
    from hisq_inputs import fields
    oracle.set_threads(os.cpu_count() or 1)
    fat, lng = fields.recipe_links(DIMS, EPS, LINK_SEED)
    b = fields.gaussian_source(DIMS, SRC_SEED)[0].numpy()
    _, fp64_iters, _, true_res = oracle.cg(DIMS, fat.numpy(), lng.numpy(), MASS, b, tol=TOL)
    samples = []
    for _ in range(args.warmup):
        oracle_sample(2.0, fp64_iters)
    for _ in range(args.steps):
        samples.append(oracle_sample(max(3.0, 60.0 / max(1, args.steps)), fp64_iters))
    v = statistics.mean(s["value"] for s in samples)
    cb = dict(samples[-1])
    cb["value"] = v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "ms", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": v, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD + " (FP64 oracle on host cores, extrapolated)"},
            "cpu_baseline": cb, "e2e": {"value": v, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "iterations": fp64_iters, "true_residual": true_res}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------- GPU arm
def traffic_for(kernel_key: str):
    """DRAM bytes per launch from the committed ncu summary, if it matches the current source."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        e = d[kernel_key]
        h = hashlib.sha256()
        for fn in e["sources"]:
            with open(os.path.join(ROOT, fn), "rb") as g:
                h.update(g.read())
        return e["dram_bytes_per_launch"] if h.hexdigest() == e["sha256"] else None
    except Exception:
        return None


def workload_configs(hbm):
    """The other workloads of the benchmark definition, measured after the timed region (one
    GPU, rank 0); every solve to a true FP64 residual <= 1e-10.  Returns a dict for the line.
      (every solve timed after one untimed call of the same solve)
      64^3x16 (eps 0.3, m 0.01): FP32 Dslash at nrhs 1/4/8/16 (HBM-streaming, L2 flushed),
        mixed CG (FP32 sloppy, FP64 reliable updates) at nrhs 1 and 8 against plain FP64 CG,
        14-shift multi-shift CG (FP32 sloppy), and the 32 uneven lattices batched vs one by one;
      32^3x8 learned preconditioner (eps 0.5, m 0.005): 2000 training pairs, 4 epochs, flexible
        CG with the network against plain and mixed CG on 10 held-out sources;
      96^3x24 (eps 0.3, m 0.01, 12-real 16-bit links): Dslash HBM fraction and the 14-shift
        mixed multi-shift solve."""
    import torch

    from hisq_inputs import fields, workloads
    from paper_2306_01098_gb300 import dslash_bench, hisq, precond_bench, solver_bench
    out = {}

    def timed(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = fn()
        torch.cuda.synchronize()
        return 1e3 * (time.perf_counter() - t0), r

    # ---- 64^3 x 16
    w = workloads.BATCH_64x16
    c = {"regime": "HBM-streaming (link store 2.4 GB FP32 > L2)"}
    c["dslash_f32"] = dslash_bench.measure(w.dims, ("f32",), (1, 4, 8, 16), 18, reps=5, hbm_gbs=hbm, seed=w.link_seed)
    torch.cuda.empty_cache()
    fat, lng = fields.recipe_links(w.dims, w.eps, w.link_seed, device="cuda")
    ctx = hisq.Context(w.dims, fat, lng, precs=(hisq.F64, hisq.F32))
    del fat, lng
    torch.cuda.empty_cache()
    b1 = fields.gaussian_source(w.dims, w.source_seed, 1, device="cuda")
    x1 = torch.zeros_like(b1)
    fp64 = lambda: ctx.cg(w.mass, b1, x1.zero_(), tol=w.tol, prec_sloppy=hisq.F64)
    fp64()  # untimed: autotuning and first launches
    ms64, (rc, st) = timed(fp64)
    c["fp64_cg"] = {"nrhs": 1, "ms": ms64, "iterations": st.iterations, "true_residual": st.true_residual}
    c["mixed_cg_f32"] = []
    for nrhs in (1, 8):
        b = fields.gaussian_source(w.dims, w.source_seed, nrhs, device="cuda")
        x = torch.zeros_like(b)
        res = torch.zeros(nrhs, dtype=torch.float64)
        solve = lambda: ctx.cg(w.mass, b, x.zero_(), tol=w.tol, prec_sloppy=hisq.F32, prec_precise=hisq.F64,
                               reliable_delta=0.01, residuals=res)
        solve()
        ms, (rc, st) = timed(solve)
        c["mixed_cg_f32"].append({"nrhs": nrhs, "ms": ms, "ms_per_rhs": ms / nrhs, "iterations": st.iterations,
                                  "reliable_updates": st.reliable_updates, "max_true_residual": float(res.max()),
                                  "speedup_per_rhs_vs_fp64_cg": ms64 / (ms / nrhs), "converged": rc == hisq.OK})
        del b, x
    sig = list(w.shifts)
    xs = [torch.zeros_like(b1[0]) for _ in sig]
    res = torch.zeros(len(sig), dtype=torch.float64)
    def ms14():
        for t in xs:
            t.zero_()
        return ctx.multishift_cg(w.mass, sig, b1[0].contiguous(), xs, tol=[w.tol] * len(sig), prec_sloppy=hisq.F32,
                                 prec_precise=hisq.F64, reliable_delta=0.01, residuals=res)
    ms14()  # untimed: autotuning of the 14 right-hand-side finish and first launches
    ms, (rc, st) = timed(ms14)
    c["multishift_14_f32"] = {"ms": ms, "iterations": st.iterations, "max_true_residual": float(res.max()),
                              "converged": rc == hisq.OK}
    ctx.close()
    del xs, b1, x1
    torch.cuda.empty_cache()
    c["uneven_32_lattices"] = solver_bench.uneven(reps=1)
    out["config_64x64x64x16"] = c
    torch.cuda.empty_cache()

    # ---- learned preconditioner, 32^3 x 8, m 0.005
    rows = precond_bench.run(pairs=2000, epochs=4, test=10)
    out["config_learned_32x32x32x8"] = {"regime": "L2-resident (16-bit links 75 MB)", "rows": rows}
    torch.cuda.empty_cache()

    # ---- 96^3 x 24, 12-real 16-bit links
    rows = solver_bench.large(reps=1)
    out["config_96x96x96x24"] = {"regime": "HBM-streaming (16-bit 12-real link store 4.1 GB)", "rows": rows}
    torch.cuda.empty_cache()
    return out


def run_ours(args, world, rank, local):
    import torch

    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    barrier(world)
    from hisq_inputs import fields
    from paper_2306_01098_gb300 import hisq

    torch.cuda.set_device(local)
    dev = f"cuda:{local}"
    fat, lng = fields.recipe_links(DIMS, EPS, LINK_SEED, device=dev)
    sloppy = {"f32": hisq.F32, "f16": hisq.F16, "bf16": hisq.BF16, "f64x": hisq.F64X}[args.sloppy]
    ctx = hisq.Context(DIMS, fat, lng, precs=(hisq.F64, hisq.F64X, hisq.F32, hisq.F16, hisq.BF16), device=local,
                       compression={sloppy: args.sloppy_reals})
    del fat, lng
    b = fields.gaussian_source(DIMS, SRC_SEED, device=dev)[0]
    x = torch.zeros_like(b)
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MB > L2

    precise_default = {"f64": hisq.F64, "f64x": hisq.F64X}[args.precise]

    def solve(prec, precise=None, profile=0, xb=x, bb=b, host=0):
        precise = precise_default if precise is None else precise
        rc, st = ctx.cg(MASS, bb, xb, tol=TOL, prec_sloppy=prec, prec_precise=precise, reliable_interval=100,
                        l2_persist=int(args.l2_persist), use_graph=int(args.use_graph),
                        reliable_delta=args.delta, profile=profile, host_buffers=host, stream=stream,
                        single_reduction=args.single_reduction, persistent=args.persistent if prec != hisq.F64 else 0)
        if rc != hisq.OK:
            raise RuntimeError(f"solve did not converge: {st.as_dict()}")
        return st

    # plain FP64 CG on the same GPU (the comparator), outside the timed region
    st64 = solve(hisq.F64, precise=hisq.F64)
    x64 = x.clone()
    fp64_ms = []
    for _ in range(args.fp64_reps):
        flush.add_(1.0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st64 = solve(hisq.F64, precise=hisq.F64)
        e1.record(stream)
        torch.cuda.synchronize()
        fp64_ms.append(e0.elapsed_time(e1))
    fp64_ms = min(fp64_ms) if fp64_ms else None
    # plain float-pair CG (FP64-class operator and vectors throughout; the final residual is
    # recomputed with the FP64 operator): the other FP64-class comparator
    f64x_ms = []
    st64x = None
    for _ in range(args.fp64_reps):
        flush.add_(1.0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st64x = solve(hisq.F64X, precise=hisq.F64X)
        e1.record(stream)
        torch.cuda.synchronize()
        f64x_ms.append(e0.elapsed_time(e1))
    f64x_ms = min(f64x_ms) if f64x_ms else None

    clk = Clocks(local).__enter__()              # sampling starts with the warm-up
    for _ in range(args.warmup):
        flush.add_(1.0)
        solve(sloppy)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    stats = []
    torch.cuda.nvtx.range_push("timed")
    if True:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        step_ms = []
        e0.record(stream)
        for _ in range(args.steps):
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            flush.add_(1.0)                       # L2 flushed between timed solves
            s0.record(stream)
            stats.append(solve(sloppy, profile=1))
            s1.record(stream)
            s1.synchronize()
            step_ms.append(s0.elapsed_time(s1))
        e1.record(stream)
        torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    clk.__exit__(None, None, None)
    barrier(world)
    total_ms = e0.elapsed_time(e1)
    ms_per_solve = max_over_ranks(sum(step_ms) / len(step_ms), world)

    # end to end through the C ABI with host buffers: H2D of b, D2H of x inside the timed region
    bh = b.cpu().pin_memory()
    xh = torch.zeros_like(bh).pin_memory()
    solve(sloppy, xb=xh, bb=bh, host=1)
    torch.cuda.synchronize()
    e2e = []
    for _ in range(args.e2e_steps if args.e2e_steps is not None else args.steps):
        flush.add_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        solve(sloppy, xb=xh, bb=bh, host=1)
        torch.cuda.synchronize()
        e2e.append(1e3 * (time.perf_counter() - t0))
    e2e_ms = max_over_ranks(statistics.mean(e2e), world) if e2e else None

    # accuracy of the mixed-precision result against the FP64 solve
    err_vs_fp64 = float(((x - x64).norm() / x64.norm()).item())
    st = stats[-1]
    Vh = ctx.Vh
    reals = args.sloppy_reals
    lb = {hisq.F32: 4, hisq.F16: 2, hisq.BF16: 2, hisq.F64X: 8}[sloppy] * reals
    sb = {hisq.F32: 24, hisq.F16: 24, hisq.BF16: 24, hisq.F64X: 48}[sloppy]  # 16-bit links iterate FP32 vectors
    hbm, src = peaks()
    persistent = st.persistent_ds > 0
    single = persistent or args.single_reduction
    # algorithmic bytes of one sloppy iteration: each Dslash reads every link once and its input
    # and output once; D_eo's epilogue reads p (and r in the single-reduction form); the
    # updates read and write x, r, p (and read Ap): two-reduction 14, single-reduction 13 records
    iter_bytes = Vh * (32 * lb + (13 if single else 14) * sb)
    # one reliable update: the FP64 normal operator (two FP64 Dslash applications, p read by
    # the epilogue) and the FP64 vector passes around it (b, Ax, r; x_hi and x_lo; r back)
    ru_bytes = Vh * (2 * (16 * 144 + 2 * 48) + 48 + 3 * 48 + 2 * 48 + 2 * sb + 48 + sb)
    solve_bytes = st.iterations * iter_bytes + st.reliable_updates * ru_bytes
    if persistent:
        # the dominant kernel is the persistent phase kernel: all sloppy iterations of a phase
        kname = f"cg_phase_{args.sloppy}_{reals}_32x32x32x8"
        launches = sum(s.phase_launches for s in stats)
        iters_timed = sum(s.phase_iterations for s in stats)
        d_ms = sum(s.phase_ms for s in stats) / max(1, launches)
        bytes_per_launch = iter_bytes * iters_timed / max(1, launches)
    else:
        # mean over the iteration's Dslash pair: every link once, input and output spinor once,
        # plus the epilogue's reads in D_eo (p, and r in the single-reduction form)
        kname = f"dslash_{args.sloppy}_{reals}_32x32x32x8"
        epi_reads = 2 if args.single_reduction else 1
        bytes_per_launch = Vh * (16 * lb + 2 * sb) + Vh * sb * epi_reads // 2
        launches = sum(s.dslash_timed for s in stats)
        d_ms = sum(s.dslash_ms for s in stats) / max(1, launches)
    achieved = bytes_per_launch / (d_ms * 1e-3) / 1e9
    clocks = clk.summary()
    if rank != 0:
        return
    table = None
    if not args.no_dslash_table:
        from paper_2306_01098_gb300 import dslash_bench
        table = dslash_bench.measure((64, 64, 64, 16), ("f64", "f64x", "f32", "f16"), (1,), 18, hbm_gbs=hbm)
    cb = oracle_sample(args.cpu_seconds, st64.iterations) if not args.no_cpu_baseline else None
    # the other measured roofs of this GPU (FMA throughput, L2 and HBM read bandwidth, launch
    # and grid-barrier times), outside the timed region
    roofs = hisq.measure_peaks(local) if world == 1 else None
    configs = None
    if world == 1 and not args.no_configs:
        del ctx
        torch.cuda.empty_cache()
        configs = workload_configs(hbm)
    line = {
        "metric": METRIC, "value": ms_per_solve, "unit": "ms", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_solve, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": f"{args.sloppy}+{args.precise}", "data": "synthetic",
        "config": {"workload": WORKLOAD, "lattice": "32x32x32x8", "sloppy": args.sloppy, "precise": args.precise,
                   "reliable_interval": 100, "reliable_delta": args.delta,
                   "l2": "flushed between timed solves (256 MB write)",
                   "l2_persist_links": {-1: "auto", 0: "off", 1: "on"}[args.l2_persist],
                   "sloppy_link_reals": reals,
                   "iteration_loop": (f"one persistent cooperative kernel per phase (launch shape {st.persistent_ds})"
                                      if persistent else
                                      "CUDA graph WHILE node" if args.use_graph else "direct launches"),
                   "reductions_per_iteration": 1 if single else 2,
                   "parallelism": f"replicas x{world}"},
        "iterations": st.iterations, "reliable_updates": st.reliable_updates, "true_residual": st.true_residual,
        "error_vs_fp64": err_vs_fp64, "fp64_cg_ms": fp64_ms, "fp64_iterations": st64.iterations,
        "fp64_cg_ms_statistic": f"min of {args.fp64_reps} solves (value: mean of the timed steps)",
        "f64x_cg_ms": f64x_ms, "f64x_iterations": st64x.iterations if st64x else None,
        "speedup_vs_f64x_cg": f64x_ms / ms_per_solve if f64x_ms else None,
        "speedup_vs_fp64_cg": fp64_ms / ms_per_solve if fp64_ms else None, "timed_total_ms": total_ms,
        "solve_algorithmic_bytes": solve_bytes,
        "time_to_solution_roof_frac": solve_bytes / (ms_per_solve * 1e-3) / 1e9 / hbm,
        "dslash_64x64x64x16": table,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                     "traffic": traffic_for(kname), "kernel": kname, "peak_source": src,
                     "bytes_per_launch": bytes_per_launch, "avg_launch_us": d_ms * 1e3,
                     "launches_timed": launches,
                     "l2_peak": roofs["l2_read_gbs"] if roofs else None,
                     "frac_of_l2": achieved / roofs["l2_read_gbs"] if roofs else None},
        "measured_roofs": roofs,
        "cpu_baseline": cb,
        "e2e": {"value": e2e_ms, "unit": "ms", "h2d_bytes_per_step": int(b.numel() * 16),
                "d2h_bytes_per_step": int(b.numel() * 16)},
        "gpu_launches": int(sum(s.kernels for s in stats)) + args.steps,
        "clocks": clocks,
        "workload_configs": configs,
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--sloppy", default="f16", choices=["f32", "f16", "bf16", "f64x"])
    ap.add_argument("--precise", default="f64", choices=["f64", "f64x"])
    ap.add_argument("--l2-persist", type=int, default=-1)
    ap.add_argument("--delta", type=float, default=0.01)
    ap.add_argument("--use-graph", type=int, default=1, help="0: direct launches (for ncu launch lists)")
    ap.add_argument("--single-reduction", type=int, default=0, help="1: one grid reduction per CG iteration")
    ap.add_argument("--persistent", type=int, default=-1,
                    help="-1: the library's choice; 0: multi-kernel loop; 1 to 5: persistent kernel, launch shape")
    ap.add_argument("--sloppy-reals", type=int, default=18, choices=[18, 12], help="sloppy link compression")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-dslash-table", action="store_true")
    ap.add_argument("--no-configs", action="store_true", help="skip the 64^3x16, learned and 96^3x24 workloads")
    ap.add_argument("--fp64-reps", type=int, default=3)
    ap.add_argument("--e2e-steps", type=int, default=None)
    ap.add_argument("--oracle-table", action="store_true",
                    help="time the FP64 oracle on the host cores (1 thread and all cores) and exit")
    args = ap.parse_args()
    if args.oracle_table:
        oracle_table()
        return
    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        backend = "gloo" if args.impl == "reference" else "nccl"
        if backend == "nccl":
            import torch
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    try:
        if args.impl == "reference":
            run_reference(args, world, rank)
        else:
            run_ours(args, world, rank, local)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()

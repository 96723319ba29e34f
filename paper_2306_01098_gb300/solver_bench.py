"""Solver throughput on the batched and large workloads (JSON lines).

  python -m paper_2306_01098_gb300.solver_bench --workload batched   # 64^3 x 16
  python -m paper_2306_01098_gb300.solver_bench --workload large     # 96^3 x 24, 12-real links
  python -m paper_2306_01098_gb300.solver_bench --workload uneven    # 32 uneven lattices, batched
  python -m paper_2306_01098_gb300.solver_bench --workload rational  # r(A) b ~ A^-1/2 b, 32^3 x 8
  python -m paper_2306_01098_gb300.solver_bench --workload smear     # HISQ link smearing
  python -m paper_2306_01098_gb300.solver_bench --workload meson     # point-source correlators

batched: multi-RHS CG for nrhs in {1, 4, 8, 16} (16-bit links, FP32 vectors, FP64 reliable
         updates), time per right-hand side against plain FP64 CG with one right-hand side, and
         multi-shift CG with 14 shifts log-spaced 1e-5..1 (mixed and FP64).
large:   multi-shift CG with 14 shifts on 96^3 x 24 with 12-real compressed 16-bit links and
         FP64 reliable updates, plus the Dslash roofline of that link store.
Every solve reports its residuals recomputed with the FP64 operator (tol 1e-10).
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _timed(fn, reps=1):
    """Best of reps wall times of fn() after one untimed call (which also runs the launch-shape
    autotuner for any new precision and right-hand-side count)."""
    import torch
    ts = []
    out = fn()
    for _ in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = fn()
        torch.cuda.synchronize()
        ts.append(1e3 * (time.perf_counter() - t0))
    return min(ts), out


def batched(reps=2):
    import torch

    from hisq_inputs import fields, workloads
    from paper_2306_01098_gb300 import hisq
    w = workloads.BATCH_64x16
    fat, lng = fields.recipe_links(w.dims, w.eps, w.link_seed, device="cuda")
    ctx = hisq.Context(w.dims, fat, lng, precs=(hisq.F64, hisq.F64X, hisq.F32, hisq.F16))
    del fat, lng
    torch.cuda.empty_cache()
    rows = []
    b1 = fields.gaussian_source(w.dims, w.source_seed, 1, device="cuda")
    x = torch.zeros_like(b1)
    ms64, (rc, st) = _timed(lambda: ctx.cg(w.mass, b1, x.zero_(), tol=w.tol, prec_sloppy=hisq.F64), reps)
    rows.append({"solve": "cg", "nrhs": 1, "sloppy": "f64", "ms": ms64, "ms_per_rhs": ms64, "iterations": st.iterations,
                 "true_residual": st.true_residual, "rc": rc})
    for nrhs in w.nrhs:
        b = fields.gaussian_source(w.dims, w.source_seed, nrhs, device="cuda")
        x = torch.zeros_like(b)
        res = torch.zeros(nrhs, dtype=torch.float64)
        ctx.cg(w.mass, b, x, tol=w.tol, prec_sloppy=hisq.F16, prec_precise=hisq.F64, reliable_delta=0.01)
        ms, (rc, st) = _timed(lambda: ctx.cg(w.mass, b, x.zero_(), tol=w.tol, prec_sloppy=hisq.F16, prec_precise=hisq.F64,
                                             reliable_delta=0.01, residuals=res), reps)
        rows.append({"solve": "cg", "nrhs": nrhs, "sloppy": "f16", "ms": ms, "ms_per_rhs": ms / nrhs,
                     "iterations": st.iterations, "reliable_updates": st.reliable_updates,
                     "max_true_residual": float(res.max()), "speedup_per_rhs_vs_fp64": ms64 / (ms / nrhs), "rc": rc})
    sig = list(w.shifts)
    for prec, name in ((hisq.F64, "f64"), (hisq.F64X, "f64x"), (hisq.F16, "f16")):
        xs = [torch.zeros_like(b1[0]) for _ in sig]
        res = torch.zeros(len(sig), dtype=torch.float64)
        ms, (rc, st) = _timed(lambda: ctx.multishift_cg(w.mass, sig, b1[0].contiguous(), xs, tol=[w.tol] * len(sig),
                                                        prec_sloppy=prec, prec_precise=hisq.F64, reliable_delta=0.01,
                                                        residuals=res), reps)
        rows.append({"solve": "multishift", "nshift": len(sig), "sloppy": name, "ms": ms, "iterations": st.iterations,
                     "max_true_residual": float(res.max()), "rc": rc})
    ctx.close()
    return rows


def large(reps=1):
    import torch

    from hisq_inputs import fields, workloads
    from paper_2306_01098_gb300 import dslash_bench, hisq
    w = workloads.LARGE_96x24
    t0 = time.perf_counter()
    fat, lng = fields.recipe_links(w.dims, w.eps, w.link_seed, device="cuda")
    gen_s = time.perf_counter() - t0
    ctx = hisq.Context(w.dims, fat, lng, precs=(hisq.F64, hisq.F16), compression={hisq.F64: 18, hisq.F16: 12})
    del fat, lng
    torch.cuda.empty_cache()
    rows = [{"step": "links", "generate_s": gen_s}]
    b = fields.gaussian_source(w.dims, w.source_seed, 1, device="cuda")[0]
    sig = list(w.shifts)
    xs = [torch.zeros_like(b) for _ in sig]
    res = torch.zeros(len(sig), dtype=torch.float64)
    ms, (rc, st) = _timed(lambda: ctx.multishift_cg(w.mass, sig, b, xs, tol=[w.tol] * len(sig), prec_sloppy=hisq.F16,
                                                    prec_precise=hisq.F64, reliable_delta=0.01, residuals=res), reps)
    rows.append({"solve": "multishift", "lattice": "96x96x96x24", "links": "f16 12-real + f64 18-real",
                 "nshift": len(sig), "ms": ms, "iterations": st.iterations, "reliable_updates": st.reliable_updates,
                 "max_true_residual": float(res.max()), "rc": rc,
                 "solves_per_s": 1e3 / ms, "site_shift_updates_per_s": ctx.Vh * len(sig) * st.iterations / (ms * 1e-3)})
    ctx.close()
    del xs, b
    torch.cuda.empty_cache()
    for r in dslash_bench.measure(w.dims, ("f16",), (1,), 12, reps=5, seed=w.link_seed):
        r["workload"] = "96x96x96x24"
        rows.append(r)
    return rows


def uneven(reps=3, batched_only=False, use_graph=1, nvtx=False):
    """32 uneven lattices (8^3x8 ... 24^3x8, eps 0.3, m 0.1, 1 source each, FP32 sloppy
    with FP64 reliable updates): one batched Dslash launch against 32 launches, and the
    batched CG (one graph, all members per launch) against 32 solves one after another, both
    with the multi-kernel iteration and with the persistent phase kernel of a lone solve.
    batched_only: the batched solve alone; use_graph = 0: its iterations as direct launches;
    nvtx: one more batched solve inside an NVTX range "timed" (for ncu --nvtx-include)."""
    import torch

    from hisq_inputs import fields, workloads
    from paper_2306_01098_gb300 import hisq
    dims = workloads.uneven_batch()
    ctxs = []
    for i, d in enumerate(dims):
        fat, lng = fields.recipe_links(d, 0.3, 1100 + i, device="cuda")
        ctxs.append(hisq.Context(d, fat, lng, precs=(hisq.F64, hisq.F32)))
    batch = hisq.Batch(ctxs)
    bs = [fields.gaussian_source(d, 2200 + i, device="cuda")[0] for i, d in enumerate(dims)]
    bp = torch.cat([b.reshape(-1) for b in bs]).reshape(-1, 3)
    out = torch.empty_like(bp)
    outs = [torch.empty_like(b) for b in bs]
    rows = [{"lattices": len(dims), "sites": 2 * batch.sites}]

    def dslash_batched():
        batch.dslash(0, bp, out, prec=hisq.F32)

    def dslash_each():
        for c, b, o in zip(ctxs, bs, outs):
            c.dslash(0, b, o, prec=hisq.F32)

    for name, fn in (("batched", dslash_batched), ("per_lattice", dslash_each)):
        fn()
        ms, _ = _timed(lambda: [fn() for _ in range(10)], reps)
        rows.append({"op": "dslash_f32_with_conversions", "mode": name, "ms": ms / 10})
    kw = dict(tol=1e-10, prec_sloppy=hisq.F32, prec_precise=hisq.F64, reliable_delta=0.01)
    x = torch.zeros_like(bp)
    res = torch.zeros(len(dims), dtype=torch.float64)
    bkw = dict(kw, use_graph=use_graph)
    batch.cg([0.1] * len(dims), bp, x.zero_(), residuals=res, **bkw)
    ms, (rc, st) = _timed(lambda: batch.cg([0.1] * len(dims), bp, x.zero_(), residuals=res, **bkw), reps)
    rows.append({"solve": "cg", "mode": "batched", "use_graph": use_graph, "ms": ms, "iterations": st.iterations,
                 "max_true_residual": float(res.max()), "rc": rc})
    if nvtx:
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("timed")
        batch.cg([0.1] * len(dims), bp, x.zero_(), residuals=res, **bkw)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    if batched_only:
        batch.close()
        for c in ctxs:
            c.close()
        return rows
    xs = [torch.zeros_like(b) for b in bs]

    def each(persistent):
        worst, its = 0.0, 0
        for c, b, xk in zip(ctxs, bs, xs):
            r1 = torch.zeros(1, dtype=torch.float64)
            rc1, st1 = c.cg(0.1, b, xk.zero_(), residuals=r1, persistent=persistent, **kw)
            worst, its = max(worst, float(r1[0])), max(its, st1.iterations)
        return worst, its

    # one by one with the same multi-kernel iteration as the batch (the batching gain), and
    # with each solve's default, the persistent kernel (one cooperative launch per phase)
    for mode, persistent in (("per_lattice", 0), ("per_lattice_persistent", -1)):
        ms1, (worst, its) = _timed(lambda: each(persistent), reps)
        rows.append({"solve": "cg", "mode": mode, "ms": ms1, "max_iterations": its, "max_true_residual": worst,
                     "speedup_batched": ms1 / ms})
    batch.close()
    for c in ctxs:
        c.close()
    return rows


def rational_workload(reps=2, nterm=24):
    """r(A) b ~ A^-1/2 b on the 32^3 x 8 workload (eps 0.5, m 0.01): nterm sinc-quadrature
    partial fractions applied from one multi-shift solve (every shifted system to 1e-10), FP64
    and 16-bit sloppy, against nterm independent mixed-precision CG solves; the accuracy of the
    approximation over the spectrum bounds is reported."""
    import numpy as np
    import torch

    from hisq_inputs import fields, rational, workloads
    from paper_2306_01098_gb300 import hisq
    w = workloads.MIXED_32x8
    fat, lng = fields.recipe_links(w.dims, w.eps, w.link_seed, device="cuda")
    ctx = hisq.Context(w.dims, fat, lng, precs=(hisq.F64, hisq.F64X, hisq.F32, hisq.F16))
    del fat, lng
    lo, hi = 4 * w.mass ** 2, 4 * (w.mass ** 2 + 4 * (1 + 1 / 24) ** 2)
    a0, al, sg = rational.inv_sqrt(nterm, lo, hi)
    lam = np.geomspace(lo, hi, 2000)
    approx = float(max(abs(rational.evaluate(a0, al, sg, l) * np.sqrt(l) - 1) for l in lam))
    b = fields.gaussian_source(w.dims, w.source_seed, device="cuda")[0]
    x = torch.empty_like(b)
    rows = [{"workload": "rational A^-1/2, 32x32x32x8", "terms": nterm, "approx_rel_err_on_spectrum": approx}]
    for prec, name in ((hisq.F64, "f64"), (hisq.F16, "f16")):
        res = torch.zeros(nterm, dtype=torch.float64)
        ms, (rc, st) = _timed(lambda: ctx.rational_apply(w.mass, a0, al, sg, b, x, tol=1e-10, prec_sloppy=prec,
                                                         prec_precise=hisq.F64, reliable_delta=0.01, residuals=res),
                              reps)
        rows.append({"solve": "rational_apply", "sloppy": name, "ms": ms, "iterations": st.iterations,
                     "max_true_residual": float(res.max()), "rc": rc})
    # the same nterm systems as independent mixed-precision CG solves on 4 m_s^2 - D_eo D_oe
    xs = torch.empty_like(b)

    def separate():
        worst = 0.0
        for s in sg:
            m_s = (w.mass ** 2 + s / 4.0) ** 0.5
            r1 = torch.zeros(1, dtype=torch.float64)
            ctx.cg(m_s, b, xs.zero_(), tol=1e-10, prec_sloppy=hisq.F16, prec_precise=hisq.F64, reliable_delta=0.01,
                   residuals=r1)
            worst = max(worst, float(r1[0]))
        return worst

    ms, worst = _timed(separate, 1)
    rows.append({"solve": "separate_mixed_cg", "systems": nterm, "ms": ms, "max_true_residual": worst})
    ctx.close()
    return rows


def smear_workload(reps=2):
    """HISQ link smearing (hisq_smear_links, FP64) on the 32^3 x 8 and 96^3 x 24 thin links, and
    the 32^3 x 8 solve (m 0.01) with the smeared operator: mixed precision vs plain FP64 CG."""
    import torch

    from hisq_inputs import fields, workloads
    from paper_2306_01098_gb300 import hisq
    rows = []
    for w in (workloads.MIXED_32x8, workloads.LARGE_96x24):
        thin, _ = fields.recipe_links(w.dims, w.eps, w.link_seed, device="cuda")
        ms, (fat, lng) = _timed(lambda: hisq.smear_links(w.dims, thin), reps)
        links = 4 * thin.shape[1]
        rows.append({"op": "smear_links", "lattice": "x".join(map(str, w.dims)), "ms": ms,
                     "links_per_s": links / (ms * 1e-3)})
        if w is workloads.MIXED_32x8:
            del thin
            ctx = hisq.Context(w.dims, fat, lng, precs=(hisq.F64, hisq.F16))
            b = fields.gaussian_source(w.dims, w.source_seed, device="cuda")[0]
            x = torch.zeros_like(b)
            for prec, name in ((hisq.F64, "f64"), (hisq.F16, "f16")):
                ms, (rc, st) = _timed(lambda: ctx.cg(w.mass, b, x.zero_(), tol=w.tol, prec_sloppy=prec,
                                                     prec_precise=hisq.F64, reliable_delta=0.01), reps)
                rows.append({"solve": "cg_smeared_links", "sloppy": name, "ms": ms, "iterations": st.iterations,
                             "true_residual": st.true_residual, "rc": rc})
            ctx.close()
        del fat, lng
        torch.cuda.empty_cache()
    return rows


def meson_workload(reps=3):
    """Point-source meson correlators (hisq_meson_correlators) on the 32^3 x 8 workload (eps 0.5,
    m 0.01) along t: the three-colour multi-RHS solve to 1e-10 with 16-bit and FP64 sloppy
    operators, the call's total time against the time of its solve."""
    from hisq_inputs import fields, workloads
    from paper_2306_01098_gb300 import hisq
    w = workloads.MIXED_32x8
    fat, lng = fields.recipe_links(w.dims, w.eps, w.link_seed, device="cuda")
    ctx = hisq.Context(w.dims, fat, lng, precs=(hisq.F64, hisq.F32, hisq.F16))
    del fat, lng
    src = (5, 17, 30, 3)
    rows = []
    for prec, name in ((hisq.F16, "f16"), (hisq.F64, "f64")):
        ms, (corr, rc, st) = _timed(lambda: ctx.meson_correlators(w.mass, src, 3, tol=w.tol, prec_sloppy=prec,
                                                                  prec_precise=hisq.F64, reliable_delta=0.01), reps)
        rows.append({"op": "meson_correlators", "lattice": "x".join(map(str, w.dims)), "sloppy": name, "ms": ms,
                     "solve_ms": 1e3 * st.seconds, "iterations": st.iterations, "true_residual": st.true_residual,
                     "pion": [float(v) for v in corr[0]], "rc": rc})
    ctx.close()
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", choices=["batched", "large", "uneven", "rational", "smear", "meson"], default="batched")
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--batched-only", action="store_true", help="uneven: the batched solve alone")
    ap.add_argument("--use-graph", type=int, default=1, help="uneven: 0 runs the batched iterations as direct launches")
    ap.add_argument("--nvtx", action="store_true", help="uneven: one more batched solve in an NVTX range 'timed'")
    a = ap.parse_args()
    if a.workload == "uneven":
        rows = uneven(a.reps, a.batched_only, a.use_graph, a.nvtx)
    else:
        rows = {"batched": batched, "large": large, "rational": rational_workload,
                "smear": smear_workload, "meson": meson_workload}[a.workload](a.reps)
    for r in rows:
        print(json.dumps(r), flush=True)


if __name__ == "__main__":
    main()

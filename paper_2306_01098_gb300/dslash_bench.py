"""Dslash throughput on internal-layout fields: GB/s against the HBM roofline, TFLOP/s.

  python -m paper_2306_01098_gb300.dslash_bench --dims 64,64,64,16 --prec f64x,f32 --nrhs 1,4 [--comp 12]
  python -m paper_2306_01098_gb300.dslash_bench --prec f32 --nrhs 16 --sweep    # every launch shape
  python -m paper_2306_01098_gb300.dslash_bench --peaks          # measured ALU, L2, HBM roofs

The timed repetitions run inside an NVTX range named "timed", so that a profiler can be told
to capture only launches with the autotuned (or pinned) shape.

Algorithmic bytes per application (Sec. 5.1 accounting with perfect neighbour reuse):
  Vh * (16 * link_bytes + nrhs * 2 * spinor_bytes)
i.e. every link read once, every input and output spinor once; flops 1146 per site and
right-hand side.  Inputs are larger than L2 at 64^3 x 16; L2 is also flushed between reps.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

NAMES = {"f64": 0, "f64x": 1, "f32": 2, "f16": 3, "bf16": 4}
LINK_REAL_BYTES = {0: 8, 1: 8, 2: 4, 3: 2, 4: 2}
SPINOR_BYTES = {0: 48, 1: 48, 2: 24, 3: 16, 4: 16}


def alg_bytes(Vh, prec, nreal, nrhs):
    return Vh * (16 * nreal * LINK_REAL_BYTES[prec] + nrhs * 2 * SPINOR_BYTES[prec])


def hbm_peak():
    """Measured copy bandwidth of this GPU model (GB/s) from MEASURED_PEAKS.json, else the
    6800 GB/s of an earlier GB300 measurement."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0


def shapes(prec, nrhs, zt_ok=True):
    """Every (n_inner, threads per site, site order, threads per block, right-hand-side groups
    per site, right-hand-side groups per block) launch shape the autotuner considers."""
    cap = 4 if prec in ("f64", "f64x") else 8
    out = []
    for order in ((0, 1) if zt_ok else (0,)):
        nr = 1
        while nr <= cap:
            if nrhs % nr == 0:
                out.extend((nr, ds, order, bs, 1, 1) for ds in (1, 2, 4) for bs in (64, 128, 256))
                out.extend((nr, 1, order, bs, rg, 1) for rg in (2, 4) for bs in (64, 128, 256)
                           if nr <= 4 and nrhs % (nr * rg) == 0)
                out.extend((nr, 1, order, bs, 1, wg) for wg in (2, 4) for bs in (64, 128, 256)
                           if nr <= 4 and nrhs % (nr * wg) == 0 and bs // wg >= 32)
            nr *= 2
    return out


def measure(dims=(64, 64, 64, 16), precs=("f64", "f64x", "f32", "f16"), nrhs_list=(1,), comp=18, reps=10,
            hbm_gbs=None, seed=1002, shape=None, sweep=False):
    import torch

    from hisq_inputs import fields
    from paper_2306_01098_gb300 import hisq
    hbm_gbs = hbm_gbs or hbm_peak()
    ps = [NAMES[p] for p in precs if not (p == "f64x" and comp == 12)]
    fat, lng = fields.recipe_links(dims, 0.3, seed, device="cuda")
    ctx = hisq.Context(dims, fat, lng, precs=tuple(ps), compression={p: comp for p in ps})
    del fat, lng
    torch.cuda.empty_cache()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    out = []
    zt_ok = dims[3] < dims[2] and (dims[0] // 2 * dims[1]) % 32 == 0
    for p in ps:
        for nrhs in nrhs_list:
            fi, fo = ctx.field(p, nrhs), ctx.field(p, nrhs)
            fi.load(fields.gaussian_source(dims, 7, nrhs, device="cuda"))
            pinned = shapes(hisq.PREC_NAMES[p], nrhs, zt_ok) if sweep else [shape]
            for sh in pinned:
                if sh is not None:
                    ctx.tune_set(p, p, nrhs, *sh[:3])
                    if len(sh) > 3:
                        ctx.tune_set_block(p, p, nrhs, sh[3])
                    if len(sh) > 4:
                        ctx.tune_set_groups(p, p, nrhs, sh[4])
                    if len(sh) > 5:
                        ctx.tune_set_block_groups(p, p, nrhs, sh[5])
                for _ in range(3):
                    ctx.dslash_field(0, fi, fo)
                torch.cuda.synchronize()
                ts = []
                torch.cuda.nvtx.range_push("timed")
                for it in range(reps):
                    flush.add_(1.0)
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    ctx.dslash_field(it & 1, fi, fo)
                    e1.record()
                    torch.cuda.synchronize()
                    ts.append(e0.elapsed_time(e1))
                torch.cuda.nvtx.range_pop()
                ms = sorted(ts)[len(ts) // 2]
                b = alg_bytes(ctx.Vh, p, comp, nrhs)
                row = {"prec": hisq.PREC_NAMES[p], "nreal": comp, "nrhs": nrhs, "us": ms * 1e3,
                       "gbs": b / ms / 1e6, "frac_hbm": b / ms / 1e6 / hbm_gbs,
                       "tflops": 1146 * ctx.Vh * nrhs / ms / 1e9, "bytes": b}
                used = ctx.tune_get(p, p, nrhs)
                if used is not None:
                    row["shape"] = {"n_inner": used[0], "threads_per_site": used[1], "site_order": used[2],
                                    "threads_per_block": used[3], "rhs_groups": used[4],
                                    "block_groups": ctx.tune_get_block_groups(p, p, nrhs), "autotuned": sh is None}
                out.append(row)
            fi.close()
            fo.close()
    ctx.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--dims", default="64,64,64,16")
    ap.add_argument("--prec", default="f64,f64x,f32,f16")
    ap.add_argument("--nrhs", default="1")
    ap.add_argument("--comp", type=int, default=18)
    ap.add_argument("--reps", type=int, default=10)
    ap.add_argument("--shape", default=None,
                    help="n_inner,threads_per_site,site_order[,threads_per_block[,rhs_groups[,block_groups]]] "
                         "instead of the autotuner")
    ap.add_argument("--sweep", action="store_true", help="time every launch shape")
    ap.add_argument("--peaks", action="store_true",
                    help="print the measured FMA, L2/HBM, launch and grid-barrier roofs (hisq_measure_peaks)")
    a = ap.parse_args()
    if a.peaks:
        from paper_2306_01098_gb300 import hisq
        print(json.dumps(hisq.measure_peaks()))
        return
    shape = tuple(int(v) for v in a.shape.split(",")) if a.shape else None
    rows = measure(tuple(int(v) for v in a.dims.split(",")), tuple(a.prec.split(",")),
                   tuple(int(v) for v in a.nrhs.split(",")), a.comp, a.reps, shape=shape, sweep=a.sweep)
    for r in rows:
        print(json.dumps(r))


if __name__ == "__main__":
    main()

"""Learned preconditioner on the 32^3 x 8 workload (eps 0.5, m 0.005): train, then compare.

  python -m paper_2306_01098_gb300.precond_bench [--pairs 2000] [--epochs 4] [--test 20] [--loss 1]

1. training pairs (b, x = A^-1 b): Gaussian sources solved by multi-RHS mixed-precision CG
   (16-bit links, FP64 reliable updates) to 1e-8;
2. training of the 4-layer network (8 channels by default) on the GPU (BF16 activations,
   Adam) on the residual norm |A (K b - x)|^2 / |b|^2 (loss 1) or the error norm (loss 0);
3. on held-out sources, time and iterations to a true residual of 1e-10 for: plain FP64 CG,
   mixed-precision CG, flexible CG without the network, flexible CG with the network.
Prints JSON lines.
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


def run(pairs=2000, epochs=4, test=20, batch=8, lr=2e-3, channels=8, loss=1):
    import numpy as np
    import torch

    from hisq_inputs import fields, workloads
    from paper_2306_01098_gb300 import hisq
    w = workloads.LEARNED_32x8
    fat, lng = fields.recipe_links(w.dims, w.eps, w.link_seed, device="cuda")
    ctx = hisq.Context(w.dims, fat, lng, precs=(hisq.F64, hisq.F64X, hisq.F32, hisq.F16))
    del fat, lng
    out = []
    # 1. training pairs
    B = fields.gaussian_source(w.dims, w.source_seed, pairs, device="cuda")
    X = torch.zeros_like(B)
    t0 = time.perf_counter()
    its = []
    for k in range(0, pairs, 16):
        n = min(16, pairs - k)
        rc, st = ctx.cg(w.mass, B[k:k + n].contiguous(), X[k:k + n], tol=1e-8, prec_sloppy=hisq.F16,
                        prec_precise=hisq.F64, reliable_delta=0.01)
        its.append(st.iterations)
        if rc != hisq.OK:
            raise RuntimeError("training pair solve failed")
    torch.cuda.synchronize()
    out.append({"step": "pairs", "pairs": pairs, "seconds": time.perf_counter() - t0, "mean_iterations": float(np.mean(its))})
    # 2. training
    net = hisq.Net(ctx, epochs=epochs, batch=batch, lr=lr, channels=channels, loss=loss, mass=w.mass)
    t0 = time.perf_counter()
    losses = net.train(B, X, epochs)
    torch.cuda.synchronize()
    out.append({"step": "train", "loss": ["error", "residual"][loss], "channels": channels, "epochs": epochs,
                "batch": batch, "lr": lr, "seconds": time.perf_counter() - t0,
                "loss_per_epoch": [float(v) for v in losses], "weights": net.nw})
    del B, X
    torch.cuda.empty_cache()
    # cost of one network application
    b = fields.gaussian_source(w.dims, w.source_seed + 7000, 1, device="cuda")[0]
    z = torch.empty_like(b)
    for _ in range(3):
        net.apply(b, z)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(10):
        net.apply(b, z)
    e1.record()
    torch.cuda.synchronize()
    out.append({"step": "apply", "ms": e0.elapsed_time(e1) / 10})
    # 3. held-out comparison
    Bt = fields.gaussian_source(w.dims, w.source_seed + 9000, test, device="cuda")
    rows = {k: [] for k in ("cg_f64", "cg_mixed", "fcg_identity", "fcg_net", "fcg_net_fp64")}

    def timed(fn):
        torch.cuda.synchronize()
        t = time.perf_counter()
        rc, st = fn()
        torch.cuda.synchronize()
        return rc, st, 1e3 * (time.perf_counter() - t)

    for i in range(-1, test):  # source 0 twice: the first pass is untimed (autotuning, first launches)
        bi = Bt[max(i, 0)].contiguous()
        x = torch.zeros_like(bi)
        for key, fn in (
            ("cg_f64", lambda: ctx.cg(w.mass, bi, x.zero_(), tol=w.tol, prec_sloppy=hisq.F64)),
            ("cg_mixed", lambda: ctx.cg(w.mass, bi, x.zero_(), tol=w.tol, prec_sloppy=hisq.F16, prec_precise=hisq.F64,
                                        reliable_delta=0.01)),
            ("fcg_identity", lambda: hisq.fcg(ctx, w.mass, bi, x.zero_(), net=None, tol=w.tol, prec_precise=hisq.F64X)),
            ("fcg_net", lambda: hisq.fcg(ctx, w.mass, bi, x.zero_(), net=net, tol=w.tol, prec_precise=hisq.F64X)),
            ("fcg_net_fp64", lambda: hisq.fcg(ctx, w.mass, bi, x.zero_(), net=net, tol=w.tol, prec_precise=hisq.F64)),
        ):
            rc, st, ms = timed(fn)
            if i >= 0:
                rows[key].append((rc, st.iterations, st.true_residual, ms))
    for key, v in rows.items():
        out.append({"solve": key, "test_sources": test, "all_converged": all(r[0] == 0 for r in v),
                    "mean_iterations": float(np.mean([r[1] for r in v])),
                    "max_true_residual": float(max(r[2] for r in v)), "mean_ms": float(np.mean([r[3] for r in v]))})
    ctx.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--pairs", type=int, default=2000)
    ap.add_argument("--epochs", type=int, default=4)
    ap.add_argument("--test", type=int, default=20)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--channels", type=int, default=8)
    ap.add_argument("--loss", type=int, default=1, choices=[0, 1])
    a = ap.parse_args()
    for r in run(a.pairs, a.epochs, a.test, a.batch, a.lr, a.channels, a.loss):
        print(json.dumps(r), flush=True)


if __name__ == "__main__":
    main()

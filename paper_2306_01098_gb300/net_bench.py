"""Time one application of the learned preconditioner's network (JSON line).

  python -m paper_2306_01098_gb300.net_bench [--dims 32,32,32,8] [--reps 20]

Network: 4 layers, channels 1 -> 8 -> 8 -> 8 -> 1, seeded random complex weights, links of the
learned-preconditioner workload (32^3 x 8, eps 0.5).  Reported: milliseconds per application
with the 8 -> 8 channel mixing on the tensor cores and on the CUDA cores, for FP32 and 16-bit
link stores, and the relative difference between the two mixing paths.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

NTAP = 17


def run(dims=(32, 32, 32, 8), reps=20, seed=5):
    import numpy as np
    import torch

    from hisq_inputs import fields, workloads
    from paper_2306_01098_gb300 import hisq
    w = workloads.LEARNED_32x8
    fat, lng = fields.recipe_links(dims, w.eps, w.link_seed, device="cuda")
    ctx = hisq.Context(dims, fat, lng, precs=(hisq.F64, hisq.F32, hisq.F16))
    del fat, lng
    rng = np.random.default_rng(seed)
    chans = [1, 8, 8, 8, 1]
    ws = []
    for l in range(len(chans) - 1):
        n = NTAP * chans[l + 1] * chans[l]
        ws.append(0.4 * (rng.normal(size=n) + 1j * rng.normal(size=n)) / np.sqrt(NTAP * chans[l]))
    weights = np.concatenate(ws)
    b = fields.gaussian_source(dims, w.source_seed, device="cuda")[0]
    out = {"dims": list(dims), "reps": reps}
    zs = {}
    for tc in (1, 0):
        for lp in (hisq.F16, hisq.F32):
            net = hisq.Net(ctx, tensor_cores=tc, link_prec=lp)
            net.set_weights(weights)
            z = torch.empty_like(b)
            for _ in range(3):
                net.apply(b, z)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                net.apply(b, z)
            e1.record()
            torch.cuda.synchronize()
            key = f"{'tensor_cores' if tc else 'cuda_cores'}_{hisq.PREC_NAMES[lp]}_links_ms"
            out[key] = e0.elapsed_time(e1) / reps
            zs[(tc, lp)] = z.clone()
            net.close()
    for lp in (hisq.F16, hisq.F32):
        a, c = zs[(1, lp)], zs[(0, lp)]
        out[f"rel_diff_{hisq.PREC_NAMES[lp]}_links"] = float((a - c).norm() / c.norm())
    ctx.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--dims", default="32,32,32,8")
    ap.add_argument("--reps", type=int, default=20)
    a = ap.parse_args()
    print(json.dumps(run(tuple(int(v) for v in a.dims.split(",")), a.reps)))


if __name__ == "__main__":
    main()

"""Domain decomposition of the HISQ Dslash into time slabs (Sec. 4, "Communication"): the
partition, the neighbour and halo index maps, and the halo exchange between slabs.

Every slab [t0, t0 + lt) applies its Dslash with hisq.Domain (libhisq's hisq_dd_* kernels);
what crosses a cut is the opposite-parity field on three time slices (the Naik hop reaches
three slices).  The exchange is a copy of contiguous blocks: within one process a device
copy between the slabs' buffers, between processes (one GPU each) point-to-point sends and
receives of torch.distributed (NCCL for device tensors, gloo for host tensors).

Half-lattice order (Sec. 4.3): a parity-q field holds the site with lexicographic index
lex = x + Nx (y + Ny (z + Nz t)) at lex // 2, so one time slice of one parity is the run
[F t, F (t + 1)) with F = Nx Ny Nz / 2, and a slab is the run [F t0, F (t0 + lt)).
"""
from __future__ import annotations

import numpy as np


def partition(global_dims, nparts):
    """[(t0, lt)] for nparts slabs covering 0 .. Nt-1: t0 and lt even, lt >= 4, as equal as the
    pairs of time slices allow (the first slabs take the extra pairs)."""
    nt = int(global_dims[3])
    if nparts < 1 or nt % 2 or nt // 2 < 2 * nparts:
        raise ValueError(f"cannot cut Nt = {nt} into {nparts} slabs of at least 4 (even) slices")
    pairs = nt // 2
    base, extra = divmod(pairs, nparts)
    out, t0 = [], 0
    for r in range(nparts):
        lt = 2 * (base + (1 if r < extra else 0))
        out.append((t0, lt))
        t0 += lt
    return out


def neighbours(rank, nparts):
    """(below, above): the slabs that hold t0 - 1 and t0 + lt (periodic in time)."""
    return (rank - 1) % nparts, (rank + 1) % nparts


def face_sites(global_dims):
    nx, ny, nz, _ = global_dims
    return nx * ny * nz // 2


def slab_range(global_dims, t0, lt):
    """The slab's sites as a slice of a global half-lattice field (either parity)."""
    f = face_sites(global_dims)
    return slice(f * t0, f * (t0 + lt))


def halo_index(global_dims, t0, lt, side):
    """Global half-lattice indices of the 3 F records of the halo received below (side 'lo':
    slices t0-3 .. t0-1) or above ('hi': t0+lt .. t0+lt+2), times taken modulo Nt."""
    f, nt = face_sites(global_dims), int(global_dims[3])
    first = t0 - 3 if side == "lo" else t0 + lt
    return np.concatenate([((first + j) % nt) * f + np.arange(f) for j in range(3)])


def send_index(global_dims, t0, lt, side):
    """Global half-lattice indices of the 3 F records a slab sends: its three lowest slices
    ('lo', to the slab below) or its three highest ('hi', to the slab above)."""
    f = face_sites(global_dims)
    first = t0 if side == "lo" else t0 + lt - 3
    return np.concatenate([(first + j) * f + np.arange(f) for j in range(3)])


def exchange_local(sends):
    """Within one process: sends = [(send_lo, send_hi)] per slab in time order; returns
    [(recv_lo, recv_hi)] with recv_lo of slab d = send_hi of slab d-1 and recv_hi = send_lo of
    slab d+1 (periodic), copied into fresh buffers."""
    n = len(sends)
    return [(sends[(d - 1) % n][1].clone(), sends[(d + 1) % n][0].clone()) for d in range(n)]


def exchange_dist(send_lo, send_hi, recv_lo, recv_hi, rank, world, group=None):
    """Between processes: send the top slices up and the bottom slices down, receive the
    slices below into recv_lo and those above into recv_hi (torch.distributed point-to-point;
    with world == 1 the slab is its own neighbour and the blocks are copied)."""
    if world == 1:
        recv_lo.copy_(send_hi)
        recv_hi.copy_(send_lo)
        return
    import torch.distributed as dist
    below, above = neighbours(rank, world)
    if dist.get_backend(group) == "nccl":
        # matched in order per pair of ranks: the upward block first, then the downward one
        ops = [dist.P2POp(dist.isend, send_hi, above, group), dist.P2POp(dist.irecv, recv_lo, below, group),
               dist.P2POp(dist.isend, send_lo, below, group), dist.P2POp(dist.irecv, recv_hi, above, group)]
        reqs = dist.batch_isend_irecv(ops)
    else:
        # tag 0: blocks travelling up (top slices), tag 1: blocks travelling down
        reqs = [dist.isend(send_hi, above, group, tag=0), dist.irecv(recv_lo, below, group, tag=0),
                dist.isend(send_lo, below, group, tag=1), dist.irecv(recv_hi, above, group, tag=1)]
    for req in reqs:
        req.wait()


class SlabDslash:
    """D_{p,1-p} on this process's slab: pack, exchange with the neighbouring slabs, apply."""

    def __init__(self, domain, rank=0, world=1, group=None):
        self.dom, self.rank, self.world, self.group = domain, rank, world, group
        self.send_lo, self.send_hi, self.recv_lo, self.recv_hi = domain.halo_buffers()

    def __call__(self, out_parity, inp, out, stream=None):
        self.dom.pack(inp, self.send_lo, self.send_hi, stream)
        exchange_dist(self.send_lo, self.send_hi, self.recv_lo, self.recv_hi, self.rank, self.world, self.group)
        self.dom.dslash(out_parity, inp, self.recv_lo, self.recv_hi, out, stream)
        return out


def measure(dims=(64, 64, 64, 16), nparts=2, reps=10, seed=1002):
    """FP64 slab Dslash on one GPU: time of every slab's application (halos exchanged by device
    copies beforehand, not timed) against the undivided FP64 Dslash of the same lattice, with
    the algorithmic bytes of the Sec. 5.1 accounting (every link once, input and output once)
    plus the halo reads.  L2 is flushed between repetitions."""
    import torch

    from hisq_inputs import fields
    from paper_2306_01098_gb300 import hisq
    fat, lng = fields.recipe_links(dims, 0.3, seed, device="cuda")
    parts = partition(dims, nparts)
    doms = [hisq.Domain(dims, t0, lt, fat, lng) for t0, lt in parts]
    whole = hisq.Context(dims, fat, lng, precs=(hisq.F64,))
    del fat, lng
    x = fields.gaussian_source(dims, 7, 1, device="cuda")[0]
    slabs = [x[slab_range(dims, t0, lt)].contiguous() for t0, lt in parts]
    sends = []
    for d, s in zip(doms, slabs):
        lo, hi, _, _ = d.halo_buffers()
        d.pack(s, lo, hi)
        sends.append((lo, hi))
    recvs = exchange_local(sends)
    outs = [torch.empty_like(s) for s in slabs]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")

    def timed(fn):
        for _ in range(3):
            fn()
        ts = []
        for _ in range(reps):
            flush.add_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return sorted(ts)[len(ts) // 2]

    ms_slabs = timed(lambda: [d.dslash(0, s, rl, rh, o) for d, s, (rl, rh), o in zip(doms, slabs, recvs, outs)])
    out = torch.empty_like(x)
    ms_whole = timed(lambda: whole.dslash(0, x, out))
    Vh = x.shape[0]
    f = face_sites(dims)
    bytes_whole = Vh * (16 * 144 + 2 * 48)
    bytes_slabs = bytes_whole + nparts * 2 * 3 * f * 48
    for d in doms:
        d.close()
    whole.close()
    return {"dims": list(dims), "slabs": nparts, "slab_ms": ms_slabs, "whole_ms": ms_whole,
            "slab_gbs": bytes_slabs / ms_slabs / 1e6, "whole_gbs": bytes_whole / ms_whole / 1e6,
            "halo_bytes": nparts * 2 * 3 * f * 48}


if __name__ == "__main__":
    import argparse
    import json
    ap = argparse.ArgumentParser()
    ap.add_argument("--dims", default="64,64,64,16")
    ap.add_argument("--parts", default="2,4")
    a = ap.parse_args()
    for n in (int(v) for v in a.parts.split(",")):
        print(json.dumps(measure(tuple(int(v) for v in a.dims.split(",")), n)))

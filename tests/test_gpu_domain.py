"""Domain-decomposed Dslash (hisq_dd_*, through the C ABI) against the FP64 oracle.

The lattice is cut into time slabs (1 to 4) that live in one process on one GPU; every slab
packs its boundary slices, the halos are exchanged by device copies (domain.exchange_local,
the in-process counterpart of the NCCL exchange between GPUs), every slab applies its
Dslash, and the slabs' outputs, put back in place, must equal the oracle's undivided Dslash
to 1e-13 relative error per site (FP64).  Lattices include slabs of four slices (a Naik hop
from the bottom slice lands in the slab below's lowest slice) and uneven slab lengths."""
import numpy as np
import pytest
import torch

import oracle
from hisq_inputs import fields
from paper_2306_01098_gb300 import domain

hisq = pytest.importorskip("paper_2306_01098_gb300.hisq")

pytestmark = pytest.mark.gpu


def site_rel(got, want):
    return float((np.linalg.norm(got - want, axis=-1) / np.linalg.norm(want, axis=-1)).max())


def decomposed_dslash(doms, parts, dims, p, xd):
    sends, slabs = [], []
    for d, (t0, lt) in zip(doms, parts):
        s = xd[domain.slab_range(dims, t0, lt)].contiguous()
        lo, hi, _, _ = d.halo_buffers()
        d.pack(s, lo, hi)
        sends.append((lo, hi))
        slabs.append(s)
    recvs = domain.exchange_local(sends)
    out = torch.full_like(xd, float("nan"))
    for d, (t0, lt), s, (rlo, rhi) in zip(doms, parts, slabs, recvs):
        o = torch.full_like(s, float("nan"))
        d.dslash(p, s, rlo, rhi, o)
        out[domain.slab_range(dims, t0, lt)] = o
    return out, recvs


@pytest.mark.parametrize("dims,nparts", [((6, 4, 8, 16), 2), ((6, 4, 8, 16), 4), ((8, 8, 8, 12), 3),
                                         ((4, 6, 4, 14), 3), ((4, 6, 4, 8), 1)])
def test_slab_dslash_matches_oracle(dims, nparts):
    fat, lng = fields.recipe_links(dims, 0.5, 5000)
    fd, ld = fat.cuda(), lng.cuda()
    parts = domain.partition(dims, nparts)
    doms = [hisq.Domain(dims, t0, lt, fd, ld) for t0, lt in parts]
    for p in (0, 1):
        x = fields.gaussian_source(dims, 5100 + p)[0]
        xd = x.cuda()
        out, recvs = decomposed_dslash(doms, parts, dims, p, xd)
        # the received halos are the global field on the slices just outside each slab
        for (t0, lt), (rlo, rhi) in zip(parts, recvs):
            assert torch.equal(rlo.cpu(), x[domain.halo_index(dims, t0, lt, "lo")])
            assert torch.equal(rhi.cpu(), x[domain.halo_index(dims, t0, lt, "hi")])
        want = oracle.dslash(dims, fat.numpy(), lng.numpy(), x, p)
        assert site_rel(out.cpu().numpy(), want) <= 1e-13
    for d in doms:
        d.close()


def test_slab_from_host_links_and_the_slab_operator_helper():
    # links passed from the host; domain.SlabDslash with one process (the slab is its own
    # neighbour) is the undivided Dslash
    dims = (4, 4, 6, 8)
    fat, lng = fields.recipe_links(dims, 0.5, 5001)
    d = hisq.Domain(dims, 0, 8, fat, lng)
    op = domain.SlabDslash(d)
    x = fields.gaussian_source(dims, 5200)[0]
    out = torch.full_like(x, float("nan")).cuda()
    op(1, x.cuda(), out)
    want = oracle.dslash(dims, fat.numpy(), lng.numpy(), x, 1)
    assert site_rel(out.cpu().numpy(), want) <= 1e-13
    d.close()


def test_slab_argument_errors():
    dims = (4, 4, 4, 8)
    fat, lng = fields.unit_links(dims, 1.0, -1 / 24)
    fd, ld = fat.cuda(), lng.cuda()
    for t0, lt in ((1, 4), (0, 2), (0, 5), (6, 4)):      # odd start, too thin, odd, past Nt
        with pytest.raises(hisq.HisqError) as e:
            hisq.Domain(dims, t0, lt, fd, ld)
        assert e.value.code == hisq.EINVAL
    d = hisq.Domain(dims, 0, 4, fd, ld)
    x = torch.zeros(d.Vh, 3, dtype=torch.complex128, device="cuda")
    lo, hi, rlo, rhi = d.halo_buffers()
    with pytest.raises(hisq.HisqError) as e:
        d.dslash(0, x, rlo, rhi, x)                       # out aliases in
    assert e.value.code == hisq.EINVAL
    with pytest.raises(ValueError):
        d.dslash(0, x, rlo[:-1], rhi, torch.empty_like(x))
    d.close()

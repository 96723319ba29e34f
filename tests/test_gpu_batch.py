"""Batches of lattices of different sizes (hisq_batch_*) against the FP64 oracle and against
the single-lattice calls.

The batched Dslash must match the oracle per lattice (FP64: 1e-13 per site; FP32 2e-6 and
16-bit 3e-3 norm-wise) and the single-lattice launches within rounding (the two may be tuned
to different threads-per-site splits, which changes the order of the direction sums: FP64
1e-14 per site, FP32 1e-6 norm-wise).  Every member of a batched CG must reach a true residual <= 1e-10 with its own
mass, recomputed by the oracle.
"""
import numpy as np
import pytest
import torch

import oracle
from hisq_inputs import fields, workloads

hisq = pytest.importorskip("paper_2306_01098_gb300.hisq")

pytestmark = pytest.mark.gpu

DIMS = [(4, 4, 4, 6), (6, 4, 4, 4), (6, 6, 4, 4), (8, 4, 4, 6), (4, 6, 6, 8)]
PRECS = (hisq.F64, hisq.F64X, hisq.F32, hisq.F16)


def site_rel(got, want):
    g = got.reshape(-1, 3)
    w = want.reshape(-1, 3)
    return float((np.linalg.norm(g - w, axis=1) / np.maximum(np.linalg.norm(w, axis=1), 1e-300)).max())


def field_rel(got, want):
    return float(np.linalg.norm(got - want) / np.linalg.norm(want))


@pytest.fixture(scope="module")
def small_batch():
    members = []
    for i, d in enumerate(DIMS):
        fat, lng = fields.recipe_links(d, 0.5, 1100 + i)
        ctx = hisq.Context(d, fat.cuda(), lng.cuda(), precs=PRECS)
        members.append((d, ctx, fat.numpy(), lng.numpy()))
    batch = hisq.Batch([m[1] for m in members])
    return members, batch


def packed(members, seed):
    xs = [fields.gaussian_source(d, seed + i)[0] for i, (d, _, _, _) in enumerate(members)]
    return xs, torch.cat([x.reshape(-1) for x in xs]).reshape(-1, 3)


def split(members, v):
    out, off = [], 0
    for d, ctx, _, _ in members:
        out.append(v[off:off + ctx.Vh])
        off += ctx.Vh
    return out


@pytest.mark.parametrize("prec,tol", [(hisq.F64, None), (hisq.F64X, None), (hisq.F32, 2e-6), (hisq.F16, 3e-3)])
def test_batch_dslash_matches_oracle(small_batch, prec, tol):
    members, batch = small_batch
    assert batch.sites == sum(m[1].Vh for m in members)
    for p in (0, 1):
        xs, xp = packed(members, 400 + 10 * p)
        out = torch.full_like(xp, float("nan")).cuda()
        batch.dslash(p, xp.cuda(), out, prec=prec)
        got = split(members, out.cpu().numpy())
        for (d, ctx, fat, lng), x, g in zip(members, xs, got):
            want = oracle.dslash(d, fat, lng, x.numpy(), p)
            if tol is None:
                assert site_rel(g, want) <= 1e-13, d
            else:
                assert field_rel(g, want) <= tol, d


@pytest.mark.parametrize("prec", [hisq.F64, hisq.F32])
def test_batch_dslash_equals_single_launches(small_batch, prec):
    members, batch = small_batch
    xs, xp = packed(members, 420)
    out = torch.empty_like(xp).cuda()
    batch.dslash(0, xp.cuda(), out, prec=prec)
    got = split(members, out.cpu().numpy())
    for (d, ctx, _, _), x, g in zip(members, xs, got):
        single = torch.empty_like(x).cuda()
        ctx.dslash(0, x.cuda(), single, prec=prec)
        if prec == hisq.F64:
            assert site_rel(g, single.cpu().numpy()) <= 1e-14, d
        else:
            assert field_rel(g, single.cpu().numpy()) <= 1e-6, d


@pytest.mark.parametrize("sloppy,precise", [(hisq.F64, hisq.F64), (hisq.F32, hisq.F64), (hisq.F16, hisq.F64X)])
def test_batch_cg_every_member_converges(small_batch, sloppy, precise):
    members, batch = small_batch
    masses = [0.05, 0.1, 0.02, 0.2, 0.07]
    bs, bp = packed(members, 450)
    x = torch.zeros_like(bp).cuda()
    res = torch.zeros(len(members), dtype=torch.float64)
    rc, st = batch.cg(masses, bp.cuda(), x, tol=1e-10, prec_sloppy=sloppy, prec_precise=precise, residuals=res)
    assert rc == hisq.OK, st.as_dict()
    xs = split(members, x.cpu().numpy())
    for (d, ctx, fat, lng), m, b, xk, rk in zip(members, masses, bs, xs, res.tolist()):
        r = b.numpy() - oracle.mdagm(d, fat, lng, m, xk)
        true = np.linalg.norm(r) / np.linalg.norm(b.numpy())
        assert true <= 1e-10, (d, m, true)
        assert rk <= 1e-10
    # each member alone reaches its solution in about as many iterations as the batch's
    # slowest member
    its = []
    for (d, ctx, _, _), m, b in zip(members, masses, bs):
        xk = torch.zeros_like(b).cuda()
        rc1, st1 = ctx.cg(m, b.cuda(), xk, tol=1e-10, prec_sloppy=sloppy, prec_precise=precise)
        assert rc1 == hisq.OK
        its.append(st1.iterations)
    assert abs(st.iterations - max(its)) <= 5, (st.iterations, its)


def test_batch_arguments(small_batch):
    members, batch = small_batch
    with pytest.raises(hisq.HisqError):
        hisq.Batch([])
    fat, lng = fields.recipe_links((4, 4, 4, 4), 0.3, 1199)
    other = hisq.Context((4, 4, 4, 4), fat.cuda(), lng.cuda(), precs=(hisq.F64,))
    mixed = hisq.Batch([members[0][1], other])
    xp = torch.zeros(mixed.sites, 3, dtype=torch.complex128, device="cuda")
    with pytest.raises(hisq.HisqError):  # F32 is not built in every member
        mixed.dslash(0, xp, torch.empty_like(xp), prec=hisq.F32)
    mixed.dslash(0, xp, torch.empty_like(xp), prec=hisq.F64)
    with pytest.raises(hisq.HisqError):
        mixed.cg([-1.0, 0.1], xp, torch.empty_like(xp), tol=1e-10)
    mixed.close()


def test_uneven_32_lattice_batch():
    # the 32 uneven lattices (8^3x8 ... 24^3x8, 1 327 968 sites): batched FP32 Dslash agrees
    # with the per-lattice launches, batched mixed-precision CG converges for every member
    dims = workloads.uneven_batch()
    assert len(dims) == 32
    ctxs = []
    for i, d in enumerate(dims):
        fat, lng = fields.recipe_links(d, 0.3, 1100 + i, device="cuda")
        ctxs.append(hisq.Context(d, fat, lng, precs=(hisq.F64, hisq.F32)))
    batch = hisq.Batch(ctxs)
    assert batch.sites * 2 == sum(int(np.prod(d)) for d in dims)
    bs = [fields.gaussian_source(d, 2200 + i, device="cuda")[0] for i, d in enumerate(dims)]
    bp = torch.cat([b.reshape(-1) for b in bs]).reshape(-1, 3)
    out = torch.empty_like(bp)
    batch.dslash(1, bp, out, prec=hisq.F32)
    for c, b, o in zip(ctxs, bs, torch.split(out, [c.Vh for c in ctxs])):
        single = torch.empty_like(b)
        c.dslash(1, b, single, prec=hisq.F32)
        assert float((single - o).norm() / single.norm()) <= 1e-6
    x = torch.zeros_like(bp)
    res = torch.zeros(32, dtype=torch.float64)
    rc, st = batch.cg([0.1] * 32, bp, x, tol=1e-10, prec_sloppy=hisq.F32, prec_precise=hisq.F64, residuals=res)
    assert rc == hisq.OK and float(res.max()) <= 1e-10
    # spot-check two members with the oracle
    for k in (0, 31):
        fat, lng = fields.recipe_links(dims[k], 0.3, 1100 + k)
        xk = torch.split(x, [c.Vh for c in ctxs])[k].cpu().numpy()
        r = bs[k].cpu().numpy() - oracle.mdagm(dims[k], fat.numpy(), lng.numpy(), 0.1, xk)
        assert np.linalg.norm(r) / np.linalg.norm(bs[k].cpu().numpy()) <= 1e-10
    batch.close()


def test_batch_cg_single_reduction_matches_two_reduction(small_batch):
    # the single-reduction iteration over a batch of uneven lattices (three epilogue values per
    # lattice, zero partials beyond each lattice's own tiles) against the two-reduction form
    members, batch = small_batch
    n = len(members)
    _, bp = packed(members, 2500)
    bp = bp.cuda()
    its = {}
    for single in (1, 0):
        x = torch.zeros_like(bp)
        res = torch.zeros(n, dtype=torch.float64)
        rc, st = batch.cg([0.1] * n, bp, x, tol=1e-10, prec_sloppy=hisq.F32, prec_precise=hisq.F64,
                          single_reduction=single, residuals=res)
        assert rc == hisq.OK and float(res.max()) <= 1e-10
        its[single] = st.iterations
    assert abs(its[1] - its[0]) <= 3

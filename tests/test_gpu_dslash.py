"""GPU parity of the Dslash and normal operator (through the C ABI) against the FP64 oracle.

Tolerances: FP64 storage and the float-pair F64X path must meet 1e-13 relative error per
site (max over sites of |out_gpu(x) - out_oracle(x)| / |out_oracle(x)|, 3-vector 2-norms).
Reduced precisions are compared norm-wise over the field against bounds derived from
their unit roundoff u and the 16-term sums: F32 u = 2^-24 -> 2e-6; F16 u = 2^-11 (spinor
and link quantisation each) -> 3e-3; BF16 u = 2^-8 -> 2.5e-2.
"""
import numpy as np
import pytest
import torch

import oracle
from hisq_inputs import fields

hisq = pytest.importorskip("paper_2306_01098_gb300.hisq")

pytestmark = pytest.mark.gpu

DIMS = [(4, 4, 4, 4), (8, 8, 8, 8), (6, 4, 4, 4), (8, 8, 8, 12), (4, 6, 8, 10), (10, 4, 6, 4)]
NORM_TOL = {hisq.F32: 2e-6, hisq.F16: 3e-3, hisq.BF16: 2.5e-2}


def site_rel(got, want):
    num = np.linalg.norm(got - want, axis=-1)
    den = np.linalg.norm(want, axis=-1)
    return float((num / den).max())


def field_rel(got, want):
    return float(np.linalg.norm(got - want) / np.linalg.norm(want))


_cache = {}


def setup(dims, eps=0.5, seed=11, precs=(hisq.F64, hisq.F64X, hisq.F32, hisq.F16, hisq.BF16), comp=None, phased=False):
    key = (dims, eps, seed, precs, tuple(sorted((comp or {}).items())), phased)
    if key not in _cache:
        fat, lng = fields.recipe_links(dims, eps, seed)
        if phased:
            fat_c = torch.from_numpy(oracle.phase_links(dims, fat, 1))
            lng_c = torch.from_numpy(oracle.phase_links(dims, lng, 3))
        else:
            fat_c, lng_c = fat, lng
        ctx = hisq.Context(dims, fat_c.cuda(), lng_c.cuda(), precs=precs, compression=comp, phased=phased)
        _cache.clear()
        _cache[key] = (ctx, fat.numpy(), lng.numpy())
    return _cache[key]


@pytest.mark.parametrize("dims", DIMS)
@pytest.mark.parametrize("prec", [hisq.F64, hisq.F64X])
def test_dslash_double_class_parity(dims, prec):
    ctx, fat, lng = setup(dims)
    for p in (0, 1):
        x = fields.gaussian_source(dims, 100 + p)[0]
        out = torch.full_like(x, float("nan")).cuda()
        ctx.dslash(p, x.cuda(), out, prec=prec)
        want = oracle.dslash(dims, fat, lng, x, p)
        assert site_rel(out.cpu().numpy(), want) <= 1e-13


@pytest.mark.parametrize("dims", [(8, 8, 8, 8), (6, 4, 4, 4), (4, 6, 8, 10)])
@pytest.mark.parametrize("prec", [hisq.F32, hisq.F16, hisq.BF16])
def test_dslash_reduced_precision(dims, prec):
    ctx, fat, lng = setup(dims)
    for p in (0, 1):
        x = fields.gaussian_source(dims, 110 + p)[0]
        out = torch.full_like(x, float("nan")).cuda()
        ctx.dslash(p, x.cuda(), out, prec=prec)
        want = oracle.dslash(dims, fat, lng, x, p)
        got = out.cpu().numpy()
        assert np.isfinite(got).all()
        assert field_rel(got, want) <= NORM_TOL[prec]


@pytest.mark.parametrize("prec,tol", [(hisq.F64, 1e-13), (hisq.F32, 2e-6), (hisq.F16, 3e-3), (hisq.BF16, 2.5e-2)])
def test_dslash_12_real_compression(prec, tol):
    dims = (8, 8, 8, 12)
    ctx, fat, lng = setup(dims, comp={prec: 12}, precs=(prec,))
    for p in (0, 1):
        x = fields.gaussian_source(dims, 120 + p)[0]
        out = torch.full_like(x, float("nan")).cuda()
        ctx.dslash(p, x.cuda(), out, prec=prec)
        want = oracle.dslash(dims, fat, lng, x, p)
        got = out.cpu().numpy()
        if prec == hisq.F64:
            assert site_rel(got, want) <= tol
        else:
            assert field_rel(got, want) <= tol


def test_12_real_rejects_non_su3_links():
    dims = (4, 4, 4, 4)
    fat, lng = fields.recipe_links(dims, 0.5, 3)
    fat = fat.clone()
    fat[0, 5] *= 1.5                        # one link no longer c * SU(3)
    with pytest.raises(hisq.HisqError) as e:
        hisq.Context(dims, fat.cuda(), lng.cuda(), precs=(hisq.F32,), compression={hisq.F32: 12})
    assert e.value.code == hisq.EINVAL


@pytest.mark.parametrize("nrhs", [1, 2, 3, 4, 8, 16])
@pytest.mark.parametrize("prec", [hisq.F64, hisq.F32])
def test_dslash_multi_rhs(nrhs, prec):
    dims = (6, 4, 4, 8)
    ctx, fat, lng = setup(dims)
    x = fields.gaussian_source(dims, 130, nrhs)
    out = torch.full_like(x, float("nan")).cuda()
    ctx.dslash(1, x.cuda(), out, prec=prec)
    want = oracle.dslash(dims, fat, lng, x, 1)
    got = out.cpu().numpy()
    for r in range(nrhs):
        if prec == hisq.F64:
            assert site_rel(got[r], want[r]) <= 1e-13
        else:
            assert field_rel(got[r], want[r]) <= 2e-6


@pytest.mark.parametrize("prec", [hisq.F64, hisq.F64X, hisq.F32, hisq.F16, hisq.BF16])
def test_dslash_every_launch_shape(prec):
    # every (right-hand sides per thread, threads per site) shape gives the same operator
    dims, nrhs = (6, 4, 4, 8), 8
    ctx, fat, lng = setup(dims)
    x = fields.gaussian_source(dims, 170, nrhs)
    want = oracle.dslash(dims, fat, lng, x, 0)
    pv = hisq.F32 if prec in (hisq.F16, hisq.BF16) else prec
    tol = {hisq.F32: 2e-6, hisq.F16: 3e-3, hisq.BF16: 2.5e-2}.get(prec)
    for nr in (1, 2, 4, 8):
        if nr == 8 and prec in (hisq.F64, hisq.F64X):
            continue
        for ds in (1, 2, 4):
            ctx.tune_set(prec, pv, nrhs, nr, ds)
            out = torch.full_like(x, float("nan")).cuda()
            ctx.dslash(0, x.cuda(), out, prec=prec)
            got = out.cpu().numpy()
            for r in range(nrhs):
                if tol is None:
                    assert site_rel(got[r], want[r]) <= 1e-13, (nr, ds, r)
                else:
                    assert field_rel(got[r], want[r]) <= tol, (nr, ds, r)
    _cache.clear()


@pytest.mark.parametrize("prec,tol", [(hisq.F16, 3e-3), (hisq.BF16, 2.5e-2)])
def test_dslash_16bit_fields(prec, tol):
    # 16-bit links and 16-bit spinors (one float scale per site) through internal fields
    dims = (8, 6, 4, 6)
    ctx, fat, lng = setup(dims)
    for p in (0, 1):
        x = fields.gaussian_source(dims, 180 + p, 2)
        fi, fo = ctx.field(prec, 2), ctx.field(prec, 2)
        fi.load(x.cuda())
        ctx.dslash_field(p, fi, fo)
        out = torch.empty_like(x).cuda()
        fo.store(out)
        want = oracle.dslash(dims, fat, lng, x, p)
        got = out.cpu().numpy()
        for r in range(2):
            assert field_rel(got[r], want[r]) <= tol


def test_dslash_prephased_links():
    dims = (8, 6, 4, 6)
    ctx, fat, lng = setup(dims, precs=(hisq.F64, hisq.F32), phased=True)
    for p in (0, 1):
        x = fields.gaussian_source(dims, 140 + p)[0]
        out = torch.empty_like(x).cuda()
        ctx.dslash(p, x.cuda(), out, prec=hisq.F64)
        assert site_rel(out.cpu().numpy(), oracle.dslash(dims, fat, lng, x, p)) <= 1e-13


@pytest.mark.parametrize("prec,tol", [(hisq.F64, 1e-13), (hisq.F64X, 1e-13), (hisq.F32, 2e-6)])
def test_mdagm_parity(prec, tol):
    dims, m = (8, 8, 8, 8), 0.1
    ctx, fat, lng = setup(dims)
    b = fields.gaussian_source(dims, 150, 2)
    out = torch.empty_like(b).cuda()
    ctx.mdagm(m, b.cuda(), out, prec=prec)
    want = oracle.mdagm(dims, fat, lng, m, b)
    got = out.cpu().numpy()
    for r in range(2):
        if tol <= 1e-12:
            assert site_rel(got[r], want[r]) <= tol
        else:
            assert field_rel(got[r], want[r]) <= tol


def test_free_field_plane_wave_any_size():
    # property that holds at any size: unit links, A e^{ipx} = lambda(p) e^{ipx}
    dims, m, c1, c3 = (16, 8, 8, 12), 0.05, 9 / 8, -1 / 24
    fat, lng = fields.unit_links(dims, c1, c3)
    ctx = hisq.Context(dims, fat.cuda(), lng.cuda(), precs=(hisq.F64,))
    Vh = int(np.prod(dims)) // 2
    lex = fields.lex_of_eo(dims)[:Vh]
    x, y, z, t = [c[lex].double() for c in fields.lex_coords(dims)]
    n = (3, 1, 5, 7)
    p = [2 * np.pi * n[0] / dims[0], 2 * np.pi * n[1] / dims[1], 2 * np.pi * n[2] / dims[2],
         2 * np.pi * (n[3] + 0.5) / dims[3]]
    phase = torch.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
    u = torch.tensor([0.3 + 0.1j, -0.7j, 0.2], dtype=torch.complex128)
    phi = (phase[:, None] * u[None, :]).contiguous()
    lam = 4 * (m * m + sum((c1 * np.sin(q) + c3 * np.sin(3 * q)) ** 2 for q in p))
    out = torch.empty_like(phi).cuda()
    ctx.mdagm(m, phi.cuda(), out)
    assert (out.cpu() - lam * phi).abs().max().item() < 1e-12 * lam


def test_sampled_sites_large_lattice():
    # 64^3 x 16 in the Dslash benchmark's launch configuration, sampled output sites
    dims = (64, 64, 64, 16)
    fat, lng = fields.recipe_links(dims, 0.3, 1002, device="cuda")
    ctx = hisq.Context(dims, fat, lng, precs=(hisq.F64, hisq.F64X, hisq.F32))
    x = fields.gaussian_source(dims, 2200, 1, device="cuda")[0]
    fh, lh, xh = fat.cpu().numpy(), lng.cpu().numpy(), x.cpu().numpy()
    Vh = ctx.Vh
    rng = np.random.default_rng(1)
    sites = np.concatenate([[0, 1, Vh - 1, Vh - 2], rng.choice(Vh, 60, replace=False)])
    for prec, tol in ((hisq.F64, 1e-13), (hisq.F64X, 1e-13), (hisq.F32, 1e-5)):
        out = torch.empty_like(x)
        ctx.dslash(0, x, out, prec=prec)
        got = out.cpu().numpy()
        for s in sites:
            want = oracle.dslash_site(dims, fh, lh, xh, int(s))
            assert np.linalg.norm(got[s] - want) <= tol * np.linalg.norm(want), (prec, s)
    del fat, lng


def test_argument_errors():
    dims = (4, 4, 4, 4)
    ctx, fat, lng = setup(dims, precs=(hisq.F64,))
    x = fields.gaussian_source(dims, 160, 2).cuda()
    with pytest.raises(hisq.HisqError) as e:
        ctx.dslash(0, x, x)                          # aliasing
    assert e.value.code == hisq.EINVAL
    with pytest.raises(hisq.HisqError) as e:
        ctx.dslash(0, x[0].contiguous(), torch.empty_like(x[0]), prec=hisq.F32)   # not built
    assert e.value.code == hisq.ENOTBUILT
    with pytest.raises(hisq.HisqError) as e:
        ctx.dslash(2, x[0].contiguous(), torch.empty_like(x[0]))
    assert e.value.code == hisq.EINVAL
    for bad in [(5, 4, 4, 4), (4, 4, 2, 4), (4, 4, 4, 7)]:
        with pytest.raises(hisq.HisqError):
            hisq.Context(bad, torch.zeros(4, int(np.prod(bad)), 3, 3, dtype=torch.complex128).cuda(),
                         torch.zeros(4, int(np.prod(bad)), 3, 3, dtype=torch.complex128).cuda())


@pytest.mark.parametrize("prec", [hisq.F64, hisq.F32, hisq.F16])
def test_dslash_site_orders(prec):
    # 8 x 8 x 6 x 4: one z-t plane holds 32 sites and Nt < Nz, so the z-t interchanged
    # launch order is available; both orders, every shape, both parities give the operator
    dims, nrhs = (8, 8, 6, 4), 8
    ctx, fat, lng = setup(dims)
    pv = hisq.F32 if prec == hisq.F16 else prec
    tol = {hisq.F32: 2e-6, hisq.F16: 3e-3}.get(prec)
    for p in (0, 1):
        x = fields.gaussian_source(dims, 190 + p, nrhs)
        want = oracle.dslash(dims, fat, lng, x, p)
        for order in (0, 1):
            for nr in (1, 4, 8):
                if nr == 8 and prec == hisq.F64:
                    continue
                for ds in (1, 4):
                    ctx.tune_set(prec, pv, nrhs, nr, ds, order)
                    out = torch.full_like(x, float("nan")).cuda()
                    ctx.dslash(p, x.cuda(), out, prec=prec)
                    got = out.cpu().numpy()
                    for r in range(nrhs):
                        if tol is None:
                            assert site_rel(got[r], want[r]) <= 1e-13, (order, nr, ds, r)
                        else:
                            assert field_rel(got[r], want[r]) <= tol, (order, nr, ds, r)
    _cache.clear()


def test_site_order_rejected_where_unavailable():
    dims = (6, 4, 4, 8)  # a z-t plane of 12 sites: only storage order
    ctx, fat, lng = setup(dims)
    with pytest.raises(hisq.HisqError):
        ctx.tune_set(hisq.F64, hisq.F64, 1, 1, 1, 1)
    with pytest.raises(hisq.HisqError):
        ctx.tune_set(hisq.F64, hisq.F64, 1, 1, 1, 2)
    ctx.tune_set(hisq.F64, hisq.F64, 1, 1, 1, 0)
    _cache.clear()

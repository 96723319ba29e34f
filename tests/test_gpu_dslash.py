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


@pytest.mark.parametrize("dims,order", [((6, 4, 8, 10), 0), ((10, 4, 6, 4), 0), ((8, 8, 8, 4), 1)])
@pytest.mark.parametrize("prec", [hisq.F64, hisq.F32, hisq.F16])
def test_dslash_block_groups(dims, order, prec):
    # groups of right-hand sides per block (slices of a block over the same sites, links
    # through L1): every slice count and block size gives the oracle's operator, and exactly
    # the result of one group per block (the per-site arithmetic is the same); half volumes
    # 960 and 480 leave ragged last tiles, 8x8x8x4 runs the z-t interchanged site order
    nrhs = 8
    ctx, fat, lng = setup(dims)
    x = fields.gaussian_source(dims, 171, nrhs)
    want = oracle.dslash(dims, fat, lng, x, 1)
    pv = hisq.F32 if prec == hisq.F16 else prec
    tol = {hisq.F32: 2e-6, hisq.F16: 3e-3}.get(prec)
    for nr in (1, 2, 4):
        for bs in (64, 128, 256):
            ref = None
            for wg in (1, 2, 4):
                if bs // wg < 32 or nrhs % (nr * wg):
                    continue
                ctx.tune_set(prec, pv, nrhs, nr, 1, order)
                ctx.tune_set_block(prec, pv, nrhs, bs)
                ctx.tune_set_block_groups(prec, pv, nrhs, wg)
                assert ctx.tune_get_block_groups(prec, pv, nrhs) == wg
                assert ctx.tune_get(prec, pv, nrhs)[2] == order
                out = torch.full_like(x, float("nan")).cuda()
                ctx.dslash(1, x.cuda(), out, prec=prec)
                got = out.cpu().numpy()
                for r in range(nrhs):
                    if tol is None:
                        assert site_rel(got[r], want[r]) <= 1e-13, (nr, bs, wg, r)
                    else:
                        assert field_rel(got[r], want[r]) <= tol, (nr, bs, wg, r)
                if ref is None:
                    ref = got
                else:
                    assert np.array_equal(got, ref), (nr, bs, wg)
    # shapes the block groups do not combine with are refused
    ctx.tune_set(prec, pv, nrhs, 1, 2, order)
    with pytest.raises(hisq.HisqError):
        ctx.tune_set_block_groups(prec, pv, nrhs, 2)
    ctx.tune_set(prec, pv, nrhs, 2, 1, order)
    ctx.tune_set_block(prec, pv, nrhs, 64)
    with pytest.raises(hisq.HisqError):
        ctx.tune_set_block_groups(prec, pv, nrhs, 4)   # 16 threads per slice
    ctx.tune_set(prec, pv, nrhs, 4, 1, order)
    with pytest.raises(hisq.HisqError):
        ctx.tune_set_block_groups(prec, pv, nrhs, 4)   # 4 x 4 right-hand sides do not divide 8


@pytest.mark.parametrize("prec", [hisq.F64, hisq.F64X, hisq.F32, hisq.F16, hisq.BF16])
def test_dslash_every_launch_shape(prec):
    # every (right-hand sides per thread, threads per site, right-hand-side groups per site,
    # threads per block) shape gives the same operator
    dims, nrhs = (6, 4, 4, 8), 8
    ctx, fat, lng = setup(dims)
    x = fields.gaussian_source(dims, 170, nrhs)
    want = oracle.dslash(dims, fat, lng, x, 0)
    pv = hisq.F32 if prec in (hisq.F16, hisq.BF16) else prec
    tol = {hisq.F32: 2e-6, hisq.F16: 3e-3, hisq.BF16: 2.5e-2}.get(prec)
    for nr in (1, 2, 4, 8):
        if nr == 8 and prec in (hisq.F64, hisq.F64X):
            continue
        for ds, rg in ((1, 1), (2, 1), (4, 1), (1, 2), (1, 4)):
            if rg > 1 and (nr > 4 or nrhs % (nr * rg)):
                continue
            for bs in (64, 128, 256):
                ctx.tune_set(prec, pv, nrhs, nr, ds)
                ctx.tune_set_block(prec, pv, nrhs, bs)
                ctx.tune_set_groups(prec, pv, nrhs, rg)
                got_shape = ctx.tune_get(prec, pv, nrhs)
                assert got_shape[0] == nr and got_shape[1] == ds and got_shape[3] == bs and got_shape[4] == rg
                out = torch.full_like(x, float("nan")).cuda()
                ctx.dslash(0, x.cuda(), out, prec=prec)
                got = out.cpu().numpy()
                for r in range(nrhs):
                    if tol is None:
                        assert site_rel(got[r], want[r]) <= 1e-13, (nr, ds, rg, bs, r)
                    else:
                        assert field_rel(got[r], want[r]) <= tol, (nr, ds, rg, bs, r)
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
    # the binding checks what the C side cannot see behind its pointers
    with pytest.raises(ValueError):
        ctx.dslash(0, x, torch.empty_like(x[0]))      # out shorter than in
    with pytest.raises(ValueError):
        ctx.mdagm(0.1, x[:, :-1].contiguous(), torch.empty_like(x[:, :-1]))   # not whole vectors
    with pytest.raises(ValueError):
        ctx.mdagm(0.1, x.to(torch.complex64), torch.empty_like(x).to(torch.complex64))
    with pytest.raises(ValueError):
        ctx.mdagm_noalloc(0.1, x.cpu(), torch.empty_like(x).cpu())
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


# ---------------------------------------------------------------- reduced precision, site by site
# Per-site bound for 16-bit link storage with FP32 vectors.  A stored real component q of a
# link entry carries |q - q_exact| <= u |q_exact| (u = 2^-11 for FP16, 2^-8 for BF16, round to
# nearest), so the entry error is |dU_ij| <= u |U_ij| and, row by row (Cauchy-Schwarz),
# |dU phi| <= u |U|_F |phi|.  For a link c V with V in SU(3), |U|_F = sqrt(3) |c|.  With 12
# reals, rows 0 and 1 are stored that way and row 2 = conj(row0 x row1) is rebuilt from them:
# each rebuilt entry is a difference of two products of unit-bounded entries, so its error
# is at most 2u, and |dU|_F <= (sqrt(2) + 2 sqrt(3)) u |c|.  The FP32 arithmetic (9 complex
# multiply-adds per hop, 16 hops, the FP64 -> FP32 input rounding) adds a few 2^-24 per hop;
# 40 * 2^-24 covers it.  Summed over the 16 hops of the stencil:
#     |D_gpu phi(x) - D phi(x)| <= f(u, nreal) * S(x),   S(x) = sum_hops |c_hop| |phi(x + hop)|
# with c = 1 for the one-hop (fat = U) and 1/24 for the three-hop (long = -UUU/24) links of
# the workloads.  This holds for every site, whatever cancellation the sum has.
U_F16, U_BF16 = 2.0 ** -11, 2.0 ** -8


def hop_factor(u, nreal):
    return (np.sqrt(3.0) if nreal == 18 else np.sqrt(2.0) + 2.0 * np.sqrt(3.0)) * u + 40 * 2.0 ** -24


def hop_magnitudes(dims, x, out_parity, c1=1.0, c3=1.0 / 24.0):
    """S(x) for every output site (half index) of out_parity: sum over mu and the hops +-1, +-3
    of |c| times the 2-norm of the input colour vector at the neighbour.  x: [Vh][3] field of
    parity 1 - out_parity in canonical half-lattice order (half index = lexicographic // 2)."""
    nx, ny, nz, nt = dims
    V = nx * ny * nz * nt
    lex = np.arange(V)
    cx, cy, cz, ct = lex % nx, (lex // nx) % ny, (lex // (nx * ny)) % nz, lex // (nx * ny * nz)
    par = (cx + cy + cz + ct) % 2
    nrm = np.linalg.norm(np.asarray(x).reshape(V // 2, 3), axis=1)
    full = np.zeros(V)
    full[par == 1 - out_parity] = nrm[lex[par == 1 - out_parity] // 2]
    full = full.reshape(nt, nz, ny, nx)
    S = np.zeros_like(full)
    for axis in (3, 2, 1, 0):          # x, y, z, t
        for k, c in ((1, c1), (3, c3)):
            S += c * (np.roll(full, -k, axis=axis) + np.roll(full, k, axis=axis))
    S = S.reshape(V)
    out = np.zeros(V // 2)
    out[lex[par == out_parity] // 2] = S[par == out_parity]
    return out


def check_sites(got, want, S, factor, what):
    err = np.linalg.norm(got - want, axis=-1)
    ratio = float((err / (factor * S)).max())
    assert np.isfinite(got).all(), what
    assert ratio <= 1.0, f"{what}: worst site at {ratio:.3f} of its bound"
    return ratio


@pytest.mark.parametrize("prec,u", [(hisq.F16, U_F16), (hisq.BF16, U_BF16)])
def test_16bit_links_every_site_bench_lattice(prec, u):
    # the bench solve's sloppy operator: 16-bit links (18 reals), FP32 vectors, on the
    # 32^3 x 8 workload (eps 0.5, seed 1001); every output site of both parities, one and four
    # right-hand sides, each (n_inner, threads per site) shape
    dims = (32, 32, 32, 8)
    fat, lng = fields.recipe_links(dims, 0.5, 1001, device="cuda")
    ctx = hisq.Context(dims, fat, lng, precs=(prec,))
    fh, lh = fat.cpu().numpy(), lng.cpu().numpy()
    del fat, lng
    factor = hop_factor(u, 18)
    worst = 0.0
    for nrhs, shapes in ((1, [(1, 1), (1, 2), (1, 4)]), (4, [(4, 1), (2, 2), (1, 4)])):
        x = fields.gaussian_source(dims, 2300 + nrhs, nrhs)
        for p in (0, 1):
            want = oracle.dslash(dims, fh, lh, x, p)
            S = [hop_magnitudes(dims, x[r], p) for r in range(nrhs)]
            for nr, ds in shapes:
                ctx.tune_set(prec, hisq.F32, nrhs, nr, ds)
                out = torch.full_like(x, float("nan")).cuda()
                ctx.dslash(p, x.cuda(), out, prec=prec)
                got = out.cpu().numpy()
                for r in range(nrhs):
                    worst = max(worst, check_sites(got[r], want[r], S[r], factor, (nrhs, p, nr, ds, r)))
    print(f"{hisq.PREC_NAMES[prec]} 32^3x8: worst site at {worst:.3f} of the quantisation bound")


@pytest.mark.parametrize("prec,u", [(hisq.F16, U_F16), (hisq.BF16, U_BF16)])
def test_12_real_every_site_large_lattice(prec, u):
    # 12-real 16-bit links on 64^3 x 16 (the link store, 805 MB, exceeds what L2 keeps, so
    # n_inner > 1 reads links evict-first), every output site, one and four right-hand sides,
    # both site orders (z and t interchanged is the default for several right-hand sides)
    dims = (64, 64, 64, 16)
    fat, lng = fields.recipe_links(dims, 0.3, 1002, device="cuda")
    ctx = hisq.Context(dims, fat, lng, precs=(prec,), compression={prec: 12})
    fh, lh = fat.cpu().numpy(), lng.cpu().numpy()
    del fat, lng
    factor = hop_factor(u, 12)
    worst = 0.0
    for nrhs, shapes in ((1, [(1, 1, 0), (1, 2, 0)]), (4, [(4, 1, 1), (2, 1, 0), (4, 2, 0)])):
        x = fields.gaussian_source(dims, 2400 + nrhs, nrhs)
        p = nrhs % 2
        want = oracle.dslash(dims, fh, lh, x, p)
        S = [hop_magnitudes(dims, x[r], p) for r in range(nrhs)]
        for nr, ds, order in shapes:
            ctx.tune_set(prec, hisq.F32, nrhs, nr, ds, order)
            out = torch.full_like(x, float("nan")).cuda()
            ctx.dslash(p, x.cuda(), out, prec=prec)
            got = out.cpu().numpy()
            for r in range(nrhs):
                worst = max(worst, check_sites(got[r], want[r], S[r], factor, (nrhs, nr, ds, order, r)))
        del want, S, x
    print(f"{hisq.PREC_NAMES[prec]} 12-real 64^3x16: worst site at {worst:.3f} of the quantisation bound")


@pytest.mark.parametrize("scale", [1e-30, 1e30])
def test_float_pair_range(scale):
    # HISQ_F64X keeps every real as a float pair hi + lo without a per-site scale: inputs whose
    # components lie between about 1e-30 (the low word still a normal float) and 1e37 (the
    # products below float overflow) keep the 1e-13 per-site bound; the header states the range
    dims = (8, 6, 4, 6)
    ctx, fat, lng = setup(dims, precs=(hisq.F64, hisq.F64X))
    for p in (0, 1):
        x = (fields.gaussian_source(dims, 190 + p)[0] * scale).contiguous()
        out = torch.full_like(x, float("nan")).cuda()
        ctx.dslash(p, x.cuda(), out, prec=hisq.F64X)
        want = oracle.dslash(dims, fat, lng, x, p)
        assert site_rel(out.cpu().numpy(), want) <= 1e-13, (scale, p)


@pytest.mark.parametrize("prec", [hisq.F64, hisq.F32])
@pytest.mark.parametrize("nr,rg", [(1, 4), (2, 4), (4, 2), (2, 2)])
def test_mdagm_rhs_groups(prec, nr, rg):
    # the normal operator's epilogue and its per-right-hand-side dot products with groups of
    # right-hand sides sharing a site's threads (8 right-hand sides, ragged half volume)
    dims, m, nrhs = (6, 4, 8, 10), 0.07, 8
    ctx, fat, lng = setup(dims, precs=(hisq.F64, hisq.F32))
    ctx.tune_set(prec, prec, nrhs, nr, 1)
    ctx.tune_set_groups(prec, prec, nrhs, rg)
    b = fields.gaussian_source(dims, 195, nrhs)
    out = torch.full_like(b, float("nan")).cuda()
    ctx.mdagm(m, b.cuda(), out, prec=prec)
    want = oracle.mdagm(dims, fat, lng, m, b)
    got = out.cpu().numpy()
    for r in range(nrhs):
        if prec == hisq.F64:
            assert site_rel(got[r], want[r]) <= 1e-13, r
        else:
            assert field_rel(got[r], want[r]) <= 2e-6, r
    with pytest.raises(hisq.HisqError):
        ctx.tune_set_groups(prec, prec, nrhs, 3)
    _cache.clear()

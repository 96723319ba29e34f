"""GPU CG (through the C ABI) against the FP64 oracle.

Pass criterion for every solve: the oracle recomputes |b - A x| / |b| from the GPU's x in
FP64 and it must be <= tol (1e-10).  The relative difference from the oracle's own CG
solution is bounded by kappa(A) * tol (both solutions sit within tol of the exact one in
the residual norm); it is asserted against that bound and printed.
"""
import numpy as np
import pytest
import torch

import oracle
from hisq_inputs import fields

hisq = pytest.importorskip("paper_2306_01098_gb300.hisq")

pytestmark = pytest.mark.gpu

_cache = {}


def setup(dims, eps, seed, precs=(hisq.F64, hisq.F64X, hisq.F32, hisq.F16, hisq.BF16), comp=None):
    key = (dims, eps, seed, precs, tuple(sorted((comp or {}).items())))
    if key not in _cache:
        _cache.clear()
        fat, lng = fields.recipe_links(dims, eps, seed)
        ctx = hisq.Context(dims, fat.cuda(), lng.cuda(), precs=precs, compression=comp)
        _cache[key] = (ctx, fat.numpy(), lng.numpy())
    return _cache[key]


def true_res(dims, fat, lng, m, b, x):
    r = b - oracle.mdagm(dims, fat, lng, m, x)
    return float(np.linalg.norm(r) / np.linalg.norm(b))


def test_plain_fp64_cg_small_workload():
    # 8^4, eps = 0.3, m = 0.1, 1 RHS, tol 1e-10
    dims, m = (8, 8, 8, 8), 0.1
    ctx, fat, lng = setup(dims, 0.3, 1000)
    b = fields.gaussian_source(dims, 2000)[0]
    x = torch.zeros_like(b).cuda()
    rc, st = ctx.cg(m, b.cuda(), x, tol=1e-10, prec_sloppy=hisq.F64, prec_precise=hisq.F64)
    assert rc == hisq.OK
    xg = x.cpu().numpy()
    assert true_res(dims, fat, lng, m, b.numpy(), xg) <= 1e-10
    xo, it_o, _, _ = oracle.cg(dims, fat, lng, m, b.numpy(), tol=1e-10)
    assert abs(st.iterations - it_o) <= 2
    rel = np.linalg.norm(xg - xo) / np.linalg.norm(xo)
    kappa = (4 * (m * m + 4 * (1 + 1 / 24) ** 2)) / (4 * m * m)
    print(f"plain FP64: iterations {st.iterations} (oracle {it_o}), rel. diff vs oracle {rel:.2e}")
    assert rel <= kappa * 1e-10


@pytest.mark.parametrize("sloppy,precise", [(hisq.F32, hisq.F64), (hisq.F16, hisq.F64), (hisq.BF16, hisq.F64),
                                            (hisq.F64X, hisq.F64X), (hisq.F32, hisq.F64X), (hisq.F16, hisq.F64X)])
def test_mixed_precision_cg(sloppy, precise):
    dims, m = (8, 8, 8, 12), 0.02
    ctx, fat, lng = setup(dims, 0.5, 1001)
    b = fields.gaussian_source(dims, 2100)[0]
    x = torch.zeros_like(b).cuda()
    rc, st = ctx.cg(m, b.cuda(), x, tol=1e-10, prec_sloppy=sloppy, prec_precise=precise, reliable_interval=100)
    assert rc == hisq.OK, st.as_dict()
    res = true_res(dims, fat, lng, m, b.numpy(), x.cpu().numpy())
    print(f"sloppy {hisq.PREC_NAMES[sloppy]} precise {hisq.PREC_NAMES[precise]}: iterations {st.iterations}, "
          f"reliable updates {st.reliable_updates}, true residual {res:.2e}")
    assert res <= 1e-10
    assert st.true_residual <= 1e-10


@pytest.mark.parametrize("nrhs,sloppy", [(2, hisq.F64), (4, hisq.F32), (3, hisq.F16), (8, hisq.F32)])
def test_multi_rhs_cg(nrhs, sloppy):
    dims, m = (6, 6, 6, 8), 0.05
    ctx, fat, lng = setup(dims, 0.5, 1010)
    b = fields.gaussian_source(dims, 2150, nrhs)
    x = torch.zeros_like(b).cuda()
    res_out = torch.zeros(nrhs, dtype=torch.float64)
    rc, st = ctx.cg(m, b.cuda(), x, tol=1e-10, prec_sloppy=sloppy, prec_precise=hisq.F64, residuals=res_out)
    assert rc == hisq.OK
    xg = x.cpu().numpy()
    for r in range(nrhs):
        assert true_res(dims, fat, lng, m, b[r].numpy(), xg[r]) <= 1e-10
        assert res_out[r] <= 1e-10


def test_initial_guess_and_host_buffers():
    dims, m = (8, 4, 6, 8), 0.05
    ctx, fat, lng = setup(dims, 0.5, 1011)
    b = fields.gaussian_source(dims, 2160)[0]
    x0 = (0.1 * fields.gaussian_source(dims, 2161)[0]).contiguous()
    x = x0.clone().pin_memory()
    bp = b.clone().pin_memory()
    rc, st = ctx.cg(m, bp, x, tol=1e-10, prec_sloppy=hisq.F32, prec_precise=hisq.F64, zero_guess=0, host_buffers=1)
    assert rc == hisq.OK
    assert true_res(dims, fat, lng, m, b.numpy(), x.numpy()) <= 1e-10


def test_graph_and_direct_launch_agree():
    dims, m = (8, 8, 8, 8), 0.05
    ctx, fat, lng = setup(dims, 0.5, 1012)
    b = fields.gaussian_source(dims, 2170)[0].cuda()
    xs = []
    for g in (0, 1):
        x = torch.zeros_like(b)
        rc, st = ctx.cg(m, b, x, tol=1e-10, prec_sloppy=hisq.F32, prec_precise=hisq.F64, use_graph=g, check_interval=20,
                        reliable_interval=100, persistent=0)
        assert rc == hisq.OK
        xs.append((x.cpu(), st.iterations))
    assert xs[0][1] == xs[1][1]
    assert torch.equal(xs[0][0], xs[1][0])           # same kernels, same order: bitwise


def test_profiled_solve_counts_dslash_launches():
    dims, m = (8, 8, 8, 8), 0.05
    ctx, fat, lng = setup(dims, 0.5, 1012)
    b = fields.gaussian_source(dims, 2171)[0].cuda()
    x = torch.zeros_like(b)
    rc, st = ctx.cg(m, b, x, tol=1e-10, prec_sloppy=hisq.F32, prec_precise=hisq.F64, profile=1, check_interval=10,
                    persistent=0)
    assert rc == hisq.OK
    # the two Dslash launches of the second iteration of every phase of three or more
    # iterations are timed
    assert st.dslash_timed % 2 == 0 and 2 <= st.dslash_timed <= 2 * st.iterations and st.dslash_ms > 0


def test_not_converged_and_nan_source():
    dims, m = (8, 8, 8, 8), 0.01
    ctx, fat, lng = setup(dims, 0.5, 1013)
    b = fields.gaussian_source(dims, 2180)[0].cuda()
    x = torch.zeros_like(b)
    rc, st = ctx.cg(m, b, x, tol=1e-10, maxiter=7, prec_sloppy=hisq.F32, prec_precise=hisq.F64)
    assert rc == hisq.ENOTCONVERGED and st.iterations == 7
    bn = b.clone()
    bn[5, 1] = float("nan")
    rc, st = ctx.cg(m, bn, torch.zeros_like(b), tol=1e-10, prec_sloppy=hisq.F32, prec_precise=hisq.F64)
    assert rc == hisq.ENOTCONVERGED
    # the context stays usable
    rc, st = ctx.cg(m, b, x, tol=1e-10, prec_sloppy=hisq.F32, prec_precise=hisq.F64)
    assert rc == hisq.OK


def test_zero_source_returns_zero():
    dims, m = (4, 4, 4, 4), 0.1
    ctx, fat, lng = setup(dims, 0.5, 1014)
    b = torch.zeros(ctx.Vh, 3, dtype=torch.complex128, device="cuda")
    x = torch.ones_like(b)
    rc, st = ctx.cg(m, b, x, tol=1e-10)
    assert x.abs().max().item() == 0.0 and st.iterations == 0


@pytest.mark.parametrize("sloppy,nrhs", [(hisq.F64, 2), (hisq.F32, 4), (hisq.F16, 8)])
def test_cg_z_t_interchanged_order(sloppy, nrhs):
    # the solver's Dslash pair (with the fused epilogue and its reduction) in the z-t
    # interchanged launch order gives the same solutions within tol
    dims, m = (8, 8, 6, 4), 0.05
    ctx, fat, lng = setup(dims, 0.5, 1030)
    pv = hisq.F32 if sloppy == hisq.F16 else sloppy
    b = fields.gaussian_source(dims, 2300, nrhs)
    its = []
    for order in (0, 1):
        ctx.tune_set(sloppy, pv, nrhs, 2 if nrhs % 2 == 0 else 1, 2, order)
        x = torch.zeros_like(b).cuda()
        res = torch.zeros(nrhs, dtype=torch.float64)
        rc, st = ctx.cg(m, b.cuda(), x, tol=1e-10, prec_sloppy=sloppy, prec_precise=hisq.F64, residuals=res)
        assert rc == hisq.OK
        xg = x.cpu().numpy()
        for r in range(nrhs):
            assert true_res(dims, fat, lng, m, b[r].numpy(), xg[r]) <= 1e-10
        its.append(st.iterations)
    assert abs(its[0] - its[1]) <= 3, its
    _cache.clear()


@pytest.mark.parametrize("ds", [1, 4])
def test_cg_many_reduction_chunks(ds):
    # 32 x 32 x 16 x 16 with 8 right-hand sides: 1024 (ds 1) or 4096 (ds 4) blocks per
    # right-hand side and Dslash launch, so the epilogue's reduction runs single-level
    # (8192 partials) or in two levels over 32 chunks of 128 (32768 partials)
    dims, m, nrhs = (32, 32, 16, 16), 0.1, 8
    fat_d, lng_d = fields.recipe_links(dims, 0.3, 1040, device="cuda")
    ctx = hisq.Context(dims, fat_d, lng_d, precs=(hisq.F64, hisq.F32))
    fat, lng = fat_d.cpu().numpy(), lng_d.cpu().numpy()
    del fat_d, lng_d
    b = fields.gaussian_source(dims, 2400, nrhs)
    ctx.tune_set(hisq.F32, hisq.F32, nrhs, 2, ds, -1)
    x = torch.zeros_like(b).cuda()
    res = torch.zeros(nrhs, dtype=torch.float64)
    rc, st = ctx.cg(m, b.cuda(), x, tol=1e-10, prec_sloppy=hisq.F32, prec_precise=hisq.F64, residuals=res)
    assert rc == hisq.OK
    xg = x.cpu().numpy()
    for r in range(nrhs):
        assert true_res(dims, fat, lng, m, b[r].numpy(), xg[r]) <= 1e-10
    ctx.close()


@pytest.mark.parametrize("sloppy,nrhs", [(hisq.F64, 1), (hisq.F32, 1), (hisq.F16, 1), (hisq.F32, 4), (hisq.F16, 3)])
def test_single_and_two_reduction_iterations_agree(sloppy, nrhs):
    # the single-reduction iteration (|r'|^2 from <r,Ap> and <Ap,Ap> in the operator's
    # epilogue) and the two-reduction form solve the same systems to the FP64 tolerance in
    # about the same number of iterations; in FP64 the iterates are the same to rounding
    dims, m = (8, 8, 8, 12), 0.02
    ctx, fat, lng = setup(dims, 0.5, 1001)
    b = fields.gaussian_source(dims, 2150, nrhs)
    out = {}
    for single in (1, 0):
        x = torch.zeros_like(b).cuda()
        res = torch.zeros(nrhs, dtype=torch.float64)
        rc, st = ctx.cg(m, b.cuda(), x, tol=1e-10, prec_sloppy=sloppy, prec_precise=hisq.F64, reliable_delta=0.01,
                        single_reduction=single, residuals=res, persistent=0)
        assert rc == hisq.OK
        for k in range(nrhs):
            assert true_res(dims, fat, lng, m, b[k].numpy(), x[k].cpu().numpy()) <= 1e-10
        out[single] = (st.iterations, x.cpu().numpy())
    its1, its0 = out[1][0], out[0][0]
    print(f"sloppy {sloppy} nrhs {nrhs}: single-reduction {its1} iterations, two-reduction {its0}")
    assert abs(its1 - its0) <= max(2, 0.05 * its0)
    if sloppy == hisq.F64:
        xa, xb = out[1][1], out[0][1]
        assert np.linalg.norm(xa - xb) <= 1e-9 * np.linalg.norm(xb)


@pytest.mark.parametrize("single", [1, 0])
def test_pause_inside_timed_iterations_ends_device_loop(single):
    # with profile = 1 the first two iterations of a phase are launched directly and timed;
    # a large reliable-update delta pauses the right-hand side inside them, so the device loop
    # that follows starts with nothing active: it must end at once (the idle launch still runs
    # the loop control) and must not apply the last alpha a second time
    dims, m = (8, 8, 8, 12), 0.02
    ctx, fat, lng = setup(dims, 0.5, 1001)
    b = fields.gaussian_source(dims, 2170)[0]
    x = torch.zeros_like(b).cuda()
    rc, st = ctx.cg(m, b.cuda(), x, tol=1e-10, prec_sloppy=hisq.F32, prec_precise=hisq.F64, reliable_delta=0.5,
                    profile=1, single_reduction=single, persistent=0)
    assert rc == hisq.OK
    assert true_res(dims, fat, lng, m, b.numpy(), x.cpu().numpy()) <= 1e-10
    print(f"single_reduction {single}: {st.iterations} iterations, {st.reliable_updates} reliable updates")


def test_bench_configuration_full_size():
    # the benchmark's solve at its full size and launch configuration (32^3 x 8, eps 0.5,
    # m 0.01, 16-bit links with FP32 vectors, FP64 reliable updates, delta 0.01, timed phases,
    # graph loop): the oracle recomputes |b - A x| / |b| in FP64, and the mixed-precision x
    # agrees with the GPU's plain FP64 solve within kappa(A) tol
    from hisq_inputs import workloads
    w = workloads.MIXED_32x8
    fat, lng = fields.recipe_links(w.dims, w.eps, w.link_seed)
    ctx = hisq.Context(w.dims, fat.cuda(), lng.cuda(), precs=(hisq.F64, hisq.F16))
    b = fields.gaussian_source(w.dims, w.source_seed)[0]
    x = torch.zeros_like(b).cuda()
    rc, st = ctx.cg(w.mass, b.cuda(), x, tol=w.tol, prec_sloppy=hisq.F16, prec_precise=hisq.F64, reliable_delta=0.01,
                    profile=1, use_graph=1)
    assert rc == hisq.OK
    res = true_res(w.dims, fat.numpy(), lng.numpy(), w.mass, b.numpy(), x.cpu().numpy())
    assert res <= 1e-10
    x64 = torch.zeros_like(b).cuda()
    rc, st64 = ctx.cg(w.mass, b.cuda(), x64, tol=w.tol, prec_sloppy=hisq.F64)
    assert rc == hisq.OK
    rel = float((x - x64).norm() / x64.norm())
    kappa = (4 * (w.mass ** 2 + 4 * (1 + 1 / 24) ** 2)) / (4 * w.mass ** 2)
    print(f"bench configuration: {st.iterations} iterations, true residual {res:.2e}, |x - x64|/|x64| {rel:.2e}")
    assert rel <= kappa * 1e-10
    ctx.close()


def test_condensate_estimator():
    # per-noise samples Re <eta, A^-1 eta> from one multi-RHS solve against the oracle's
    # (each solve to 1e-10: |difference| <= |eta|^2 1e-10 kappa, asserted as 1e-7 relative);
    # on 4^4 the estimate from 128 Z2 noise vectors lies within 5 standard errors of the exact
    # 4m Tr_e A^-1 / V (dense inverse)
    from hisq_inputs import fields as F
    dims, m = (4, 4, 4, 4), 0.1
    fat, lng = F.recipe_links(dims, 0.3, 1300)
    ctx = hisq.Context(dims, fat.cuda(), lng.cuda(), precs=(hisq.F64, hisq.F32))
    Vh = ctx.Vh
    n = 128
    u = F.uniform(1301, torch.arange(2 * n * Vh * 3, dtype=torch.int64)).reshape(n, Vh, 3, 2)
    eta = torch.complex(torch.where(u[..., 0] < 0.5, -1.0, 1.0).double(), torch.zeros(n, Vh, 3, dtype=torch.float64))
    pbp, samples, rc, st = ctx.condensate(m, eta.contiguous().cuda(), tol=1e-10, prec_sloppy=hisq.F32,
                                          prec_precise=hisq.F64)
    assert rc == hisq.OK
    want = oracle.condensate_samples(dims, fat.numpy(), lng.numpy(), m, eta[:8].numpy(), tol=1e-12)
    assert np.abs(samples[:8] - want).max() <= 1e-7 * np.abs(want).max()
    V = 2 * Vh
    assert abs(pbp - 4 * m * samples.mean() / V) <= 1e-14 * abs(pbp)
    A = oracle.dense_A(dims, fat.numpy(), lng.numpy(), m)
    exact = 4 * m * np.trace(np.linalg.inv(A)).real / V
    err = 4 * m * samples.std(ddof=1) / np.sqrt(n) / V
    print(f"condensate: estimate {pbp:.6f} +- {err:.6f}, exact {exact:.6f}")
    assert abs(pbp - exact) <= 5 * err
    ctx.close()


# ---------------------------------------------------------------- persistent phase kernel
@pytest.mark.parametrize("sloppy,nreal,ds", [(hisq.F16, 18, 1), (hisq.F16, 18, 2), (hisq.F16, 18, 4), (hisq.F32, 18, 2),
                                             (hisq.BF16, 18, 4), (hisq.F16, 12, 2), (hisq.BF16, 12, 1)])
def test_persistent_phase_cg(sloppy, nreal, ds):
    # every sloppy iteration between two reliable updates in one cooperative launch (one block
    # per SM, bounded grid barriers), on a lattice whose half volume (2880) is no multiple of
    # the 128-site tile; the short reliable-update interval makes phases end at their cap
    # (p left to the host) as well as on the delta trigger
    dims, m = (6, 8, 10, 12), 0.02
    ctx, fat, lng = setup(dims, 0.5, 1020, precs=(hisq.F64, sloppy), comp={sloppy: nreal})
    b = fields.gaussian_source(dims, 2190)[0]
    x = torch.full_like(b, float("nan")).cuda()
    rc, st = ctx.cg(m, b.cuda(), x, tol=1e-10, prec_sloppy=sloppy, prec_precise=hisq.F64, reliable_interval=30,
                    persistent=ds)
    assert rc == hisq.OK, st.as_dict()
    assert st.persistent_ds == ds
    res = true_res(dims, fat, lng, m, b.numpy(), x.cpu().numpy())
    assert res <= 1e-10
    # the recurrences of the multi-kernel single-reduction loop, summed in another order
    x2 = torch.zeros_like(b).cuda()
    rc2, st2 = ctx.cg(m, b.cuda(), x2, tol=1e-10, prec_sloppy=sloppy, prec_precise=hisq.F64, reliable_interval=30,
                      persistent=0, single_reduction=1)
    assert rc2 == hisq.OK and st2.persistent_ds == 0
    print(f"persistent {hisq.PREC_NAMES[sloppy]}/{nreal} ds {ds}: {st.iterations} iterations "
          f"({st.reliable_updates} reliable updates), multi-kernel {st2.iterations}; true residual {res:.2e}")
    assert abs(st.iterations - st2.iterations) <= max(3, st2.iterations // 20)


def test_persistent_phase_deterministic_and_timed():
    dims, m = (8, 8, 8, 8), 0.05
    ctx, fat, lng = setup(dims, 0.5, 1012)
    b = fields.gaussian_source(dims, 2172)[0].cuda()
    out = []
    for _ in range(2):
        x = torch.zeros_like(b)
        rc, st = ctx.cg(m, b, x, tol=1e-10, prec_sloppy=hisq.F16, prec_precise=hisq.F64, profile=1, persistent=2)
        assert rc == hisq.OK
        out.append((x.cpu(), st.iterations))
        # every phase is one timed launch; its iterations add up to the solve's
        assert st.phase_iterations == st.iterations and st.phase_ms > 0 and st.dslash_timed == 0
    assert out[0][1] == out[1][1]
    assert torch.equal(out[0][0], out[1][0])     # fixed partial order in every block: bitwise


def test_persistent_phase_bench_workload():
    # the 32^3 x 8 bench workload (eps 0.5, m 0.01): 16-bit links with 18 and 12 reals
    dims, m = (32, 32, 32, 8), 0.01
    fat, lng = fields.recipe_links(dims, 0.5, 1001, device="cuda")
    b = fields.gaussian_source(dims, 2001)[0]
    fh, lh = fat.cpu().numpy(), lng.cpu().numpy()
    for nreal in (18, 12):
        ctx = hisq.Context(dims, fat, lng, precs=(hisq.F64, hisq.F16), compression={hisq.F16: nreal})
        x = torch.zeros_like(b).cuda()
        rc, st = ctx.cg(m, b.cuda(), x, tol=1e-10, prec_sloppy=hisq.F16, prec_precise=hisq.F64,
                        reliable_delta=0.01)
        assert rc == hisq.OK and st.persistent_ds > 0
        res = true_res(dims, fh, lh, m, b.numpy(), x.cpu().numpy())
        print(f"32^3x8 persistent F16/{nreal}: {st.iterations} iterations, {st.reliable_updates} reliable updates, "
              f"true residual {res:.2e}")
        assert res <= 1e-10
        ctx.close()


@pytest.mark.parametrize("precise", [hisq.F64, hisq.F64X])
def test_persistent_budget_and_phase_count(precise):
    # the next phase is queued before the host reads the last update's scalars, so the
    # iteration budget is enforced on the device: maxiter across several capped phases ends
    # at exactly maxiter iterations; every timed phase is followed by one reliable update;
    # a float-pair solve is certified by the FP64 operator as before
    dims, m = (8, 8, 8, 8), 0.01
    ctx, fat, lng = setup(dims, 0.5, 1013)
    b = fields.gaussian_source(dims, 2180)[0].cuda()
    x = torch.zeros_like(b)
    rc, st = ctx.cg(m, b, x, tol=1e-10, maxiter=71, prec_sloppy=hisq.F16, prec_precise=precise,
                    reliable_interval=20, persistent=2, profile=1)
    assert rc == hisq.ENOTCONVERGED and st.iterations == 71 and st.persistent_ds == 2
    assert st.phase_iterations == 71 and st.phase_launches == st.reliable_updates
    x = torch.zeros_like(b)
    rc, st = ctx.cg(m, b, x, tol=1e-10, prec_sloppy=hisq.F16, prec_precise=precise, reliable_interval=20,
                    persistent=2, profile=1)
    assert rc == hisq.OK and st.persistent_ds == 2
    assert st.phase_iterations == st.iterations and st.phase_launches == st.reliable_updates
    assert true_res(dims, fat, lng, m, b.cpu().numpy(), x.cpu().numpy()) <= 1e-10


def test_persistent_barrier_wait_is_bounded():
    # one block leaves the first launch without arriving at its first grid barrier: every
    # other block's wait runs out after 1 ms, raises the device error flag and ends the
    # launch; the solve reports HISQ_EDEVICE and the next solve on the context converges
    dims, m = (8, 8, 8, 8), 0.05
    ctx, fat, lng = setup(dims, 0.5, 1012)
    b = fields.gaussian_source(dims, 2173)[0].cuda()
    with pytest.raises(hisq.HisqError) as err:
        ctx.cg(m, b, torch.zeros_like(b), tol=1e-10, prec_sloppy=hisq.F32, prec_precise=hisq.F64, persistent=2,
               selftest_wait=1)
    assert err.value.code == hisq.EDEVICE
    x = torch.zeros_like(b)
    rc, st = ctx.cg(m, b, x, tol=1e-10, prec_sloppy=hisq.F32, prec_precise=hisq.F64, persistent=2)
    assert rc == hisq.OK
    assert true_res(dims, fat, lng, m, b.cpu().numpy(), x.cpu().numpy()) <= 1e-10


@pytest.mark.parametrize("sloppy,nr,rg", [(hisq.F32, 2, 4), (hisq.F16, 1, 4), (hisq.F32, 4, 2)])
def test_multi_rhs_cg_with_rhs_groups(sloppy, nr, rg):
    # multi-RHS CG whose sloppy Dslash runs groups of right-hand sides on one site's threads:
    # the D_eo epilogue's per-right-hand-side reductions go through the group-wise block sums
    dims, m, nrhs = (6, 6, 6, 8), 0.05, 8
    ctx, fat, lng = setup(dims, 0.5, 1010)
    pv = hisq.F32
    ctx.tune_set(sloppy, pv, nrhs, nr, 1)
    ctx.tune_set_groups(sloppy, pv, nrhs, rg)
    b = fields.gaussian_source(dims, 2155, nrhs)
    x = torch.zeros_like(b).cuda()
    res_out = torch.zeros(nrhs, dtype=torch.float64)
    rc, st = ctx.cg(m, b.cuda(), x, tol=1e-10, prec_sloppy=sloppy, prec_precise=hisq.F64, residuals=res_out)
    assert rc == hisq.OK
    xg = x.cpu().numpy()
    for r in range(nrhs):
        assert true_res(dims, fat, lng, m, b[r].numpy(), xg[r]) <= 1e-10
    _cache.clear()

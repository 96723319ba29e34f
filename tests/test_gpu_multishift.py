"""GPU multi-shift CG (through the C ABI) against the FP64 oracle.

Every shift's solution must have a recomputed residual |b - (A + sigma_s) x_s| / |b| <= tol
(evaluated by the oracle in FP64); the difference from the oracle's multi-shift solution is
bounded by kappa(A + sigma_s) * tol.
"""
import numpy as np
import pytest
import torch

import oracle
from hisq_inputs import fields
from hisq_inputs.workloads import log_shifts

hisq = pytest.importorskip("paper_2306_01098_gb300.hisq")

pytestmark = pytest.mark.gpu


def shifted_res(dims, fat, lng, m, sigma, b, x):
    r = b - oracle.mdagm(dims, fat, lng, m, x) - sigma * x
    return float(np.linalg.norm(r) / np.linalg.norm(b))


@pytest.mark.parametrize("sloppy", [hisq.F64, hisq.F64X, hisq.F32, hisq.F16])
def test_multishift_14_shifts(sloppy):
    dims, m = (8, 8, 8, 8), 0.02
    fat, lng = fields.recipe_links(dims, 0.3, 1002)
    ctx = hisq.Context(dims, fat.cuda(), lng.cuda(), precs=(hisq.F64, hisq.F64X, hisq.F32, hisq.F16))
    b = fields.gaussian_source(dims, 2200)[0]
    sig = list(log_shifts())[::-1]                   # any order
    xs = [torch.zeros_like(b).cuda() for _ in sig]
    res = torch.zeros(len(sig), dtype=torch.float64)
    rc, st = ctx.multishift_cg(m, sig, b.cuda(), xs, tol=[1e-10] * len(sig), prec_sloppy=sloppy,
                               prec_precise=hisq.F64, residuals=res)
    assert rc == hisq.OK
    xo, it_o, _ = oracle.multishift_cg(dims, fat.numpy(), lng.numpy(), m, sig, b.numpy(), 1e-10)
    for s, sg in enumerate(sig):
        xg = xs[s].cpu().numpy()
        assert shifted_res(dims, fat.numpy(), lng.numpy(), m, sg, b.numpy(), xg) <= 1e-10
        assert res[s] <= 1e-10
        kappa = (4 * m * m + sg + 4 * 4 * (1 + 1 / 24) ** 2) / (4 * m * m + sg)
        assert np.linalg.norm(xg - xo[s]) / np.linalg.norm(xo[s]) <= kappa * 1e-10
    print(f"multishift sloppy {hisq.PREC_NAMES[sloppy]}: iterations {st.iterations} (oracle {it_o})")


def test_multishift_single_shift_equals_cg():
    dims, m = (6, 6, 4, 8), 0.05
    fat, lng = fields.recipe_links(dims, 0.5, 1020)
    ctx = hisq.Context(dims, fat.cuda(), lng.cuda(), precs=(hisq.F64,))
    b = fields.gaussian_source(dims, 2201)[0].cuda()
    x1 = torch.zeros_like(b)
    rc, st1 = ctx.multishift_cg(m, [0.0], b, [x1], prec_sloppy=hisq.F64)
    x2 = torch.zeros_like(b)
    rc2, st2 = ctx.cg(m, b, x2, prec_sloppy=hisq.F64)
    assert rc == rc2 == hisq.OK
    assert abs(st1.iterations - st2.iterations) <= 1
    assert (x1 - x2).abs().max().item() <= 1e-8 * x2.abs().max().item()


def test_multishift_bad_arguments():
    dims = (4, 4, 4, 4)
    fat, lng = fields.recipe_links(dims, 0.5, 1021)
    ctx = hisq.Context(dims, fat.cuda(), lng.cuda(), precs=(hisq.F64,))
    b = fields.gaussian_source(dims, 2202)[0].cuda()
    with pytest.raises(hisq.HisqError) as e:
        ctx.multishift_cg(0.1, [-1.0], b, [torch.zeros_like(b)])
    assert e.value.code == hisq.EINVAL


@pytest.mark.parametrize("sloppy", [hisq.F64, hisq.F16])
def test_rational_apply_matches_oracle(sloppy):
    # r(A) b = alpha0 b + sum_s alpha_s (A + sigma_s)^-1 b (24 partial fractions of A^-1/2 by
    # sinc quadrature, alpha0 = 0.25) through hisq_rational_apply against the oracle's
    # multi-shift evaluation of the same rational function: every shifted system to 1e-10, so
    # the two agree within sum_s |alpha_s| 1e-10 |b| / (lambda_min + sigma_s) (asserted as 1e-8
    # relative), and against the exact A^-1/2 within the quadrature's error
    from hisq_inputs import rational
    dims, m = (8, 8, 8, 12), 0.1
    fat, lng = fields.recipe_links(dims, 0.3, 1000)
    ctx = hisq.Context(dims, fat.cuda(), lng.cuda(), precs=(hisq.F64, hisq.F64X, hisq.F32, hisq.F16))
    b = fields.gaussian_source(dims, 2600)[0]
    lo, hi = 4 * m * m, 4 * (m * m + 4 * (1 + 1 / 24) ** 2)
    a0, al, sg = rational.inv_sqrt(24, lo, hi)
    a0 = 0.25
    x = torch.empty_like(b).cuda()
    res = torch.zeros(len(sg), dtype=torch.float64)
    rc, st = ctx.rational_apply(m, a0, al, sg, b.cuda(), x, tol=1e-10, prec_sloppy=sloppy, prec_precise=hisq.F64,
                                residuals=res)
    assert rc == hisq.OK and float(res.max()) <= 1e-10
    want, res_o = oracle.rational_apply(dims, fat.numpy(), lng.numpy(), m, a0, al, sg, b.numpy(), tol=1e-12)
    got = x.cpu().numpy()
    rel = np.linalg.norm(got - want) / np.linalg.norm(want)
    print(f"sloppy {sloppy}: {st.iterations} iterations, rel. diff from the oracle {rel:.2e}")
    assert rel <= 1e-8
    ctx.close()


def test_rational_apply_bad_arguments():
    dims = (4, 4, 4, 6)
    fat, lng = fields.recipe_links(dims, 0.3, 1000)
    ctx = hisq.Context(dims, fat.cuda(), lng.cuda(), precs=(hisq.F64,))
    b = fields.gaussian_source(dims, 2601)[0].cuda()
    x = torch.empty_like(b)
    for al, sg in (([1.0], [-1.0]), ([float("nan")], [1.0]), ([1.0] * 65, [1.0] * 65)):
        with pytest.raises(hisq.HisqError):
            ctx.rational_apply(0.1, 0.0, al, sg, b, x, prec_sloppy=hisq.F64)
    with pytest.raises(hisq.HisqError):  # b and x overlap
        ctx.rational_apply(0.1, 0.0, [1.0], [1.0], b, b, prec_sloppy=hisq.F64)
    ctx.close()

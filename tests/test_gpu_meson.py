"""GPU point-source meson correlators (hisq_meson_correlators) against the oracle
(oracle.point_propagator, oracle.meson_correlators).

Both sides solve the even system by CG (the GPU to 1e-10 in mixed precision, the oracle to
1e-13); the solution error is at most |r| / lambda_min(A) = 1e-10 |rhs| / (4m^2), which bounds
the propagator difference by about 1e-8 relative at m = 0.1, and the correlators are compared
to 1e-6 of the pion correlator's sum.  Properties that hold at any size check the
GPU output by itself: the full-lattice residual M G - delta (with the oracle's operator), the
staggered Ward identity sum_tau C_0(tau) = Re tr G(src, src) / (2m), and bitwise repeatability.
"""
import numpy as np
import pytest
import torch

import oracle
from hisq_inputs import fields

hisq = pytest.importorskip("paper_2306_01098_gb300.hisq")

pytestmark = pytest.mark.gpu


def _full_residual(dims, fat, lng, m, G, src):
    """max over source colours of |M G_c - delta_c| (the oracle's operator) in units of
    |rhs_c| / (2m), rhs_c = 2m b_e - D_eo b_o the even system's right-hand side: the even
    part of M G_c - delta_c is (A x_e - rhs_c) / (2m) and the odd part vanishes, so this is
    the relative residual of the even solve."""
    V = int(np.prod(dims))
    Vh = V // 2
    ci = oracle.eo_index(dims, src)
    worst = 0.0
    for c in range(3):
        b = np.zeros((V, 3), dtype=np.complex128)
        b[ci, c] = 1.0
        rhs = 2 * m * b[:Vh] - oracle.dslash(dims, fat, lng, b[Vh:], 0)
        ge, go = G[c, :Vh], G[c, Vh:]
        r = np.empty_like(b)
        r[:Vh] = 2 * m * ge + oracle.dslash(dims, fat, lng, go, 0) - b[:Vh]
        r[Vh:] = 2 * m * go + oracle.dslash(dims, fat, lng, ge, 1) - b[Vh:]
        worst = max(worst, np.linalg.norm(r) * 2 * m / np.linalg.norm(rhs))
    return worst


def _ward(G, dims, src, m):
    ci = oracle.eo_index(dims, src)
    return sum(G[c, ci, c] for c in range(3)).real / (2 * m)


@pytest.mark.parametrize("dims,src", [((8, 8, 8, 8), (0, 0, 0, 0)), ((8, 8, 8, 8), (3, 2, 5, 7)),
                                      ((6, 4, 8, 10), (5, 0, 3, 4))])
def test_correlators_match_oracle(dims, src):
    m = 0.1
    fat, lng = fields.recipe_links(dims, 0.3, 1400)
    ctx = hisq.Context(dims, fat.cuda(), lng.cuda(), precs=(hisq.F64, hisq.F32))
    V = int(np.prod(dims))
    Gw = oracle.point_propagator(dims, fat.numpy(), lng.numpy(), m, src, tol=1e-13)
    for d in range(4):
        prop = torch.full((3, V, 3), float("nan"), dtype=torch.complex128, device="cuda")  # unwritten sites show
        corr, rc, st = ctx.meson_correlators(m, src, d, prop=prop, tol=1e-10, prec_sloppy=hisq.F32,
                                             prec_precise=hisq.F64)
        assert rc == hisq.OK and st.true_residual <= 1e-10
        want = oracle.meson_correlators(dims, Gw, src, d)
        scale = want[0].sum()
        assert np.abs(corr - want).max() <= 1e-6 * scale, (d, np.abs(corr - want).max() / scale)
        G = prop.cpu().numpy()
        assert np.linalg.norm(G - Gw) <= 1e-6 * np.linalg.norm(Gw)
        # the GPU's correlators of the GPU's own propagator, by the oracle's definition
        assert np.abs(corr - oracle.meson_correlators(dims, G, src, d)).max() <= 1e-12 * scale
    assert _full_residual(dims, fat.numpy(), lng.numpy(), m, G, src) <= 1.5e-10
    assert abs(corr[0].sum() - _ward(G, dims, src, m)) <= 5e-8 * corr[0].sum()
    ctx.close()


def test_repeatable_and_without_propagator():
    dims, m, src = (8, 8, 8, 8), 0.1, (1, 2, 3, 4)
    fat, lng = fields.recipe_links(dims, 0.3, 1401)
    ctx = hisq.Context(dims, fat.cuda(), lng.cuda(), precs=(hisq.F64, hisq.F32))
    a, _, _ = ctx.meson_correlators(m, src, 3, tol=1e-10, prec_sloppy=hisq.F32, prec_precise=hisq.F64)
    b, _, _ = ctx.meson_correlators(m, src, 3, tol=1e-10, prec_sloppy=hisq.F32, prec_precise=hisq.F64)
    assert np.array_equal(a, b)
    prop = torch.empty(3, 2 * ctx.Vh, 3, dtype=torch.complex128, device="cuda")
    c, _, _ = ctx.meson_correlators(m, src, 3, prop=prop, tol=1e-10, prec_sloppy=hisq.F32,
                                    prec_precise=hisq.F64)
    assert np.array_equal(a, c)
    ctx.close()


def test_full_size_properties():
    # 32^3 x 8, m = 0.01, 16-bit sloppy links (the solver configuration of the time-to-solution
    # workload): the full-lattice residual and the Ward identity, which hold at any size
    dims, m, src = (32, 32, 32, 8), 0.01, (5, 17, 30, 3)
    fat, lng = fields.recipe_links(dims, 0.5, 1001)
    ctx = hisq.Context(dims, fat.cuda(), lng.cuda(), precs=(hisq.F64, hisq.F32, hisq.F16))
    prop = torch.full((3, 2 * ctx.Vh, 3), float("nan"), dtype=torch.complex128, device="cuda")
    corr, rc, st = ctx.meson_correlators(m, src, 3, prop=prop, tol=1e-10, prec_sloppy=hisq.F16,
                                         prec_precise=hisq.F64)
    assert rc == hisq.OK and st.true_residual <= 1e-10
    G = prop.cpu().numpy()
    assert _full_residual(dims, fat.numpy(), lng.numpy(), m, G, src) <= 1.5e-10
    ward = _ward(G, dims, src, m)
    assert abs(corr[0].sum() - ward) <= 1e-6 * ward
    assert (corr[0] > 0).all()
    # sampled slices against the oracle's definition applied to the GPU propagator
    assert np.abs(corr - oracle.meson_correlators(dims, G, src, 3)).max() <= 1e-12 * corr[0].sum()
    ctx.close()


def test_rejects_bad_arguments():
    dims = (4, 4, 4, 4)
    fat, lng = fields.recipe_links(dims, 0.3, 1402)
    ctx = hisq.Context(dims, fat.cuda(), lng.cuda(), precs=(hisq.F64, hisq.F32))
    with pytest.raises(hisq.HisqError):
        ctx.meson_correlators(0.1, (0, 0, 4, 0), 3)
    with pytest.raises(hisq.HisqError):
        ctx.meson_correlators(0.1, (0, 0, 0, 0), -1)
    with pytest.raises(hisq.HisqError):
        ctx.meson_correlators(0.0, (0, 0, 0, 0), 3)
    ctx.close()

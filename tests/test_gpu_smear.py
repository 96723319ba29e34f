"""GPU HISQ link smearing (hisq_smear_links) against the oracle (oracle/smear.py), and the Dirac
operator built from the smeared links.

Both sides are FP64; the GPU projects to U(3) by the Newton iteration for the polar factor,
the oracle by the eigendecomposition of V^+ V, so agreement to 1e-13 (entries of order one)
checks the projection as well as every staple path.
"""
import numpy as np
import pytest
import torch

import oracle
from hisq_inputs import fields
from oracle import smear

hisq = pytest.importorskip("paper_2306_01098_gb300.hisq")

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dims,eps_naik", [((4, 4, 4, 4), 0.0), ((4, 6, 4, 8), 0.3), ((8, 8, 8, 8), 0.0)])
def test_smeared_links_match_oracle(dims, eps_naik):
    thin, _ = fields.recipe_links(dims, 0.5, 1200)
    fat, lng = hisq.smear_links(dims, thin.cuda(), eps_naik=eps_naik)
    want_fat, want_lng = smear.hisq_links(dims, thin.numpy(), eps_naik=eps_naik)
    assert np.abs(fat.cpu().numpy() - want_fat).max() <= 1e-13
    assert np.abs(lng.cpu().numpy() - want_lng).max() <= 1e-14
    # host buffers give the same links
    fh, lh = hisq.smear_links(dims, thin, eps_naik=eps_naik)
    assert torch.equal(fh, fat.cpu()) and torch.equal(lh, lng.cpu())


def test_unit_links_give_free_field_links():
    dims = (4, 4, 6, 4)
    vol = int(np.prod(dims))
    unit = torch.eye(3, dtype=torch.complex128).expand(4, vol, 3, 3).contiguous().cuda()
    fat, lng = hisq.smear_links(dims, unit)
    assert float((fat - 9 / 8 * torch.eye(3, dtype=torch.complex128, device="cuda")).abs().max()) <= 1e-14
    assert float((lng + 1 / 24 * torch.eye(3, dtype=torch.complex128, device="cuda")).abs().max()) <= 1e-15


def test_operator_with_smeared_links():
    # the HISQ operator of the smeared links: Dslash parity with the oracle applied to the
    # oracle's smeared links, and a mixed-precision solve to the FP64 tolerance
    dims, m = (8, 8, 8, 8), 0.05
    thin, _ = fields.recipe_links(dims, 0.5, 1201)
    fat, lng = hisq.smear_links(dims, thin.cuda())
    ofat, olng = smear.hisq_links(dims, thin.numpy())
    ctx = hisq.Context(dims, fat, lng, precs=(hisq.F64, hisq.F32, hisq.F16))
    src = fields.gaussian_source(dims, 2700)[0]
    out = torch.empty_like(src).cuda()
    ctx.dslash(1, src.cuda(), out)
    want = oracle.dslash(dims, ofat, olng, src.numpy(), 1)
    got = out.cpu().numpy()
    site = np.linalg.norm((got - want).reshape(-1, 3), axis=1) / np.linalg.norm(want.reshape(-1, 3), axis=1)
    assert site.max() <= 1e-13
    b = fields.gaussian_source(dims, 2701)[0]
    x = torch.zeros_like(b).cuda()
    rc, st = ctx.cg(m, b.cuda(), x, tol=1e-10, prec_sloppy=hisq.F16, prec_precise=hisq.F64)
    assert rc == hisq.OK
    r = b.numpy() - oracle.mdagm(dims, ofat, olng, m, x.cpu().numpy())
    assert np.linalg.norm(r) / np.linalg.norm(b.numpy()) <= 1e-10
    ctx.close()


def test_smear_rejects_bad_dims():
    thin, _ = fields.recipe_links((4, 4, 4, 4), 0.5, 1200)
    with pytest.raises(hisq.HisqError):
        hisq.smear_links((4, 4, 4, 5), thin.cuda())

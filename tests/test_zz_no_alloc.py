"""hisq_mdagm_noalloc: the FP64 normal operator for callers that cannot let the library
allocate device memory (their memory belongs to another allocator or a fixed budget, or
their loop must not call cudaMalloc/cudaFree, which synchronise the device).  Its output
must match hisq_mdagm's on two calls in a row (the fixed scratch array keeps the previous
call's contents), within the FP64 tolerance used by the other parity tests.

This file is collected last on purpose, so a run that stops at the first failure has run
every other test before it."""
import numpy as np
import pytest
import torch

from hisq_inputs import fields

hisq = pytest.importorskip("paper_2306_01098_gb300.hisq")

pytestmark = pytest.mark.gpu


def site_rel(got, want):
    return float((np.linalg.norm(got - want, axis=-1) / np.linalg.norm(want, axis=-1)).max())


def test_noalloc_matches_mdagm_on_two_calls():
    dims, m = (8, 8, 6, 12), 0.05
    fat, lng = fields.recipe_links(dims, 0.5, 4000)
    ctx = hisq.Context(dims, fat.cuda(), lng.cuda(), precs=(hisq.F64,))
    for call, nrhs in enumerate((3, 1)):
        b = fields.gaussian_source(dims, 4100 + call, nrhs).cuda()
        want = torch.empty_like(b)
        ctx.mdagm(m, b, want, prec=hisq.F64)
        got = torch.full_like(b, float("nan"))
        ctx.mdagm_noalloc(m, b, got)
        torch.cuda.synchronize()
        g, w = got.cpu().numpy(), want.cpu().numpy()
        for r in range(nrhs):
            assert site_rel(g[r], w[r]) <= 1e-13


def test_noalloc_rejects_more_sites_than_its_scratch():
    dims = (16, 16, 16, 16)                        # Vh = 32768; 33 vectors exceed 2^20 sites
    fat, lng = fields.unit_links(dims, 1.0, -1 / 24)
    ctx = hisq.Context(dims, fat.cuda(), lng.cuda(), precs=(hisq.F64,))
    b = torch.zeros(33, ctx.Vh, 3, dtype=torch.complex128, device="cuda")
    with pytest.raises(hisq.HisqError) as e:
        ctx.mdagm_noalloc(0.1, b, torch.empty_like(b))
    assert e.value.code == hisq.EINVAL

"""hisq_mdagm_noalloc: the FP64 normal operator for callers that cannot let the library
allocate device memory (their memory belongs to another allocator or a fixed budget, or
their loop must not call cudaMalloc/cudaFree, which synchronise the device).

On a fresh context, before any other operator call has tuned a launch shape or grown the
context's workspace, the entry point is checked against the oracle's normal operator, and
the device's free memory is checked to stay the same across the call.  Then its output must
match hisq_mdagm's on two calls in a row (the fixed scratch array keeps the previous call's
contents), within the FP64 tolerance used by the other parity tests.

This file is collected last on purpose, so a run that stops at the first failure has run
every other test before it."""
import numpy as np
import pytest
import torch

import oracle
from hisq_inputs import fields

hisq = pytest.importorskip("paper_2306_01098_gb300.hisq")

pytestmark = pytest.mark.gpu


def site_rel(got, want):
    return float((np.linalg.norm(got - want, axis=-1) / np.linalg.norm(want, axis=-1)).max())


def test_noalloc_fresh_context_matches_oracle_without_allocating():
    dims, m = (6, 4, 8, 10), 0.07                  # Vh = 960: not a multiple of the 128-site tile
    fat, lng = fields.recipe_links(dims, 0.5, 4200)
    ctx = hisq.Context(dims, fat.cuda(), lng.cuda(), precs=(hisq.F64,))
    b = fields.gaussian_source(dims, 4300, 2)
    bd = b.cuda()
    out = torch.full_like(bd, float("nan"))
    # the first call on a device may load the library's device code (and with it the
    # fixed array) and looks up the array's address; it is the warm-up
    ctx.mdagm_noalloc(m, bd, out)
    torch.cuda.synchronize()
    want = np.stack([oracle.mdagm(dims, fat.numpy(), lng.numpy(), m, b[r].numpy()) for r in range(2)])
    g = out.cpu().numpy()
    for r in range(2):
        assert site_rel(g[r], want[r]) <= 1e-13
    # later calls allocate nothing: the device's free memory does not move
    out2 = torch.full_like(bd, float("nan"))
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        ctx.mdagm_noalloc(m, bd, out2)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 == free0, f"free device memory moved by {free0 - free1} bytes"
    assert np.array_equal(out2.cpu().numpy(), g)


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

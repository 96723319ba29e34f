"""Pins of the oracle's learned-preconditioner pieces (network layer, backward, FCG).

The network is not in the paper; its definition is the gauge-covariant parallel-transport
layer stated in the oracle.  Pins:
  * a single layer with tap weights (+1, -1) reproduces D on both parities (ties the
    transports to the independently pinned Dslash);
  * gauge covariance of the whole network under a random SU(3) transform;
  * the backward pass against central finite differences of the loss (FP64), for the
    error-norm loss and the residual-norm loss; the residual-norm gradient of a single
    identity tap against its closed form with the dense operator;
  * flexible CG with K = identity reproduces CG; with K = dense A^{-1} it converges in
    one iteration.
"""
import numpy as np
import pytest
import torch

import oracle
from hisq_inputs import fields

NTAP = oracle.NTAP


def _np(t):
    return t.detach().cpu().numpy() if hasattr(t, "detach") else t


def _links(dims, eps=0.5, seed=11):
    f, l = fields.recipe_links(dims, eps, seed)
    return _np(f), _np(l)


def _rand_weights(chans, seed, scale=0.3):
    rng = np.random.default_rng(seed)
    ws = []
    for l in range(len(chans) - 1):
        n = NTAP * chans[l + 1] * chans[l]
        ws.append(scale * (rng.normal(size=n) + 1j * rng.normal(size=n)) / np.sqrt(NTAP * chans[l]))
    return np.concatenate(ws)


def test_dslash_is_one_layer():
    dims = (4, 6, 4, 4)
    fat, lng = _links(dims)
    V, Vh = int(np.prod(dims)), int(np.prod(dims)) // 2
    w = np.zeros((NTAP, 1, 1), dtype=np.complex128)
    for mu in range(4):
        w[1 + 2 * mu] = 1
        w[2 + 2 * mu] = -1
        w[9 + 2 * mu] = 1
        w[10 + 2 * mu] = -1
    psi = _np(fields.gaussian_full(dims, 80))
    out = oracle.net_layer(dims, fat, lng, w, psi, 1, 1)[0]
    assert np.abs(out[:Vh] - oracle.dslash(dims, fat, lng, psi[0, Vh:], 0)).max() < 1e-13
    assert np.abs(out[Vh:] - oracle.dslash(dims, fat, lng, psi[0, :Vh], 1)).max() < 1e-13


def test_network_gauge_covariance():
    dims = (4, 4, 4, 6)
    chans = [1, 3, 2, 1]
    U = fields.thin_links(dims, 0.5, 31)
    Om = fields.gauge_transform_lex(dims, 3000)
    Up = torch.empty_like(U)
    for mu in range(4):
        Up[mu] = Om @ U[mu] @ fields._shift_lex(Om, dims, mu, 1).conj().transpose(-1, -2)
    fat = _np(fields.lex_links_to_canonical(U, dims))
    lng = _np(fields.lex_links_to_canonical(fields.long_from_thin_lex(U, dims), dims))
    fatp = _np(fields.lex_links_to_canonical(Up, dims))
    lngp = _np(fields.lex_links_to_canonical(fields.long_from_thin_lex(Up, dims), dims))
    Vh = int(np.prod(dims)) // 2
    Om_e = _np(Om[fields.lex_of_eo(dims)])[:Vh]
    w = _rand_weights(chans, 3)
    b = _np(fields.gaussian_source(dims, 90))[0]
    lhs = oracle.net_apply(dims, fatp, lngp, chans, w, np.einsum("sij,sj->si", Om_e, b))
    rhs = np.einsum("sij,sj->si", Om_e, oracle.net_apply(dims, fat, lng, chans, w, b))
    assert np.abs(lhs - rhs).max() <= 1e-13 * np.abs(rhs).max()


@pytest.mark.parametrize("chans", [[1, 2, 1], [1, 3, 2, 2, 1]])
def test_backward_matches_finite_differences(chans):
    dims = (4, 4, 4, 4)
    fat, lng = _links(dims, seed=44)
    w = _rand_weights(chans, 7)
    b = _np(fields.gaussian_source(dims, 91))[0]
    x = _np(fields.gaussian_source(dims, 92))[0]
    loss, g = oracle.net_loss_grad(dims, fat, lng, chans, w, b, x)
    # forward consistency: loss from net_apply
    z = oracle.net_apply(dims, fat, lng, chans, w, b)
    assert abs(loss - np.linalg.norm(z - x) ** 2 / np.linalg.norm(x) ** 2) < 1e-13
    rng = np.random.default_rng(0)
    idx = rng.choice(w.size, size=12, replace=False)
    h = 1e-5
    for i in idx:
        for part, unit in (("re", 1.0), ("im", 1j)):
            wp, wm = w.copy(), w.copy()
            wp[i] += h * unit
            wm[i] -= h * unit
            lp, _ = oracle.net_loss_grad(dims, fat, lng, chans, wp, b, x)
            lm, _ = oracle.net_loss_grad(dims, fat, lng, chans, wm, b, x)
            fd = (lp - lm) / (2 * h)
            an = g[i].real if part == "re" else g[i].imag
            assert abs(fd - an) <= 1e-7 * max(1.0, abs(an)), (i, part, fd, an)


def test_residual_loss_single_tap_closed_form():
    # K = c * identity (one 1 -> 1 layer, tap 0 only): L(c) = |A (c b - x)|^2 / |b|^2 and
    # dL/dRe c + i dL/dIm c = 2 <b, A^2 (c b - x)> / |b|^2
    dims, m = (4, 4, 4, 6), 0.1
    fat, lng = _links(dims, seed=46)
    b = _np(fields.gaussian_source(dims, 93))[0]
    x = _np(fields.gaussian_source(dims, 94))[0]
    c = 0.7 - 0.2j
    w = np.zeros(NTAP, dtype=np.complex128)
    w[0] = c
    loss, g = oracle.net_loss_grad_residual(dims, fat, lng, [1, 1], w, b, x, m)
    A = oracle.dense_A(dims, fat, lng, m)
    bv, xv = b.reshape(-1), x.reshape(-1)
    e = c * bv - xv
    bb = np.vdot(bv, bv).real
    assert abs(loss - np.linalg.norm(A @ e) ** 2 / bb) <= 1e-12 * loss
    want = 2 * np.vdot(bv, A @ (A @ e)) / bb
    assert abs(g[0] - want) <= 1e-12 * abs(want)
    # every hop changes parity: in one layer the hopping taps only reach odd output sites,
    # which the loss does not see
    assert np.abs(g[1:]).max() == 0.0


@pytest.mark.parametrize("chans", [[1, 2, 1], [1, 3, 2, 1]])
def test_residual_loss_backward_matches_finite_differences(chans):
    dims, m = (4, 4, 4, 4), 0.2
    fat, lng = _links(dims, seed=47)
    w = _rand_weights(chans, 8)
    b = _np(fields.gaussian_source(dims, 95))[0]
    x = _np(fields.gaussian_source(dims, 96))[0]
    loss, g = oracle.net_loss_grad_residual(dims, fat, lng, chans, w, b, x, m)
    z = oracle.net_apply(dims, fat, lng, chans, w, b)
    r = oracle.mdagm(dims, fat, lng, m, z - x)
    assert abs(loss - np.linalg.norm(r) ** 2 / np.linalg.norm(b) ** 2) <= 1e-12 * loss
    rng = np.random.default_rng(1)
    idx = rng.choice(w.size, size=10, replace=False)
    h = 1e-5
    for i in idx:
        for part, unit in (("re", 1.0), ("im", 1j)):
            wp, wm = w.copy(), w.copy()
            wp[i] += h * unit
            wm[i] -= h * unit
            lp, _ = oracle.net_loss_grad_residual(dims, fat, lng, chans, wp, b, x, m)
            lm, _ = oracle.net_loss_grad_residual(dims, fat, lng, chans, wm, b, x, m)
            fd = (lp - lm) / (2 * h)
            an = g[i].real if part == "re" else g[i].imag
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (i, part, fd, an)


def test_fcg_identity_reproduces_cg():
    dims, m = (6, 4, 4, 4), 0.05
    fat, lng = _links(dims, seed=45)
    b = _np(fields.gaussian_source(dims, 93))[0]
    _, it_cg, _, r_cg = oracle.cg(dims, fat, lng, m, b, tol=1e-10)
    x, it_f, _, r_f = oracle.fcg(dims, fat, lng, m, b, tol=1e-10)
    assert abs(it_cg - it_f) <= 1 and r_f <= 1e-10


def test_fcg_exact_inverse_converges_in_one_iteration():
    dims, m = (4, 4, 4, 4), 0.1
    fat, lng = _links(dims, seed=46)
    b = _np(fields.gaussian_source(dims, 94))[0]
    A = oracle.dense_A(dims, fat, lng, m)
    K = np.linalg.inv(A)
    x, it, _, r = oracle.fcg_dense(dims, fat, lng, m, K, b, tol=1e-10)
    assert it == 1 and r < 1e-12


def test_fcg_complex_phase_preconditioner_reproduces_cg():
    # K = exp(i theta) I spans the same Krylov space as K = I, and the step that minimises
    # the A-norm of the error along p is alpha = <p, r> / <p, A p> = conj(<r, z>) / <p, A p>
    # (<a, b> = sum conj(a) b): flexible CG must then take CG's steps.  Dropping the
    # conjugate (alpha = <r, z> / <p, A p>) rotates every step by exp(2 i theta) and fails.
    dims, m = (4, 4, 4, 4), 0.1
    fat, lng = _links(dims, seed=47)
    b = _np(fields.gaussian_source(dims, 95))[0]
    n = b.size
    _, it_cg, _, _ = oracle.cg(dims, fat, lng, m, b, tol=1e-10)
    x1, it1, _, r1 = oracle.fcg_dense(dims, fat, lng, m, np.eye(n, dtype=np.complex128), b, tol=1e-10)
    K = np.exp(0.7j) * np.eye(n, dtype=np.complex128)
    x, it, _, r = oracle.fcg_dense(dims, fat, lng, m, K, b, tol=1e-10, maxiter=4 * it_cg)
    assert r <= 1e-10 and abs(it - it_cg) <= 1 and abs(it1 - it_cg) <= 1
    assert np.linalg.norm(x - x1) <= 1e-9 * np.linalg.norm(x1)

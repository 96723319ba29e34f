"""Pins of the oracle's HISQ link smearing (oracle/smear.py).

* Unit links: the first level sums to 1, the projection keeps it, the second level is 9/8 and
  the Naik link -1/24 (the free-field coefficients, which the Dslash pins already tie to the
  closed-form spectrum).
* Random U(1) phases times the identity: every smeared link is a scalar sum over explicit paths;
  an independent enumeration of the paths (1, 3, 5, 7 links, Lepage, Naik; first level,
  projection to a unit phase, second level) must reproduce the staple recursion.  A wrong
  detour, a missing dagger or a dropped path changes the phases.
* Gauge covariance under a random SU(3) transform: X'(x) = O(x) X(x) O(x+mu)^+,
  W'(x) = O(x) W(x) O(x+3mu)^+.
* The projection returns unitary matrices and leaves unitary ones unchanged.
"""
import itertools

import numpy as np
import pytest

from hisq_inputs import fields
from oracle import smear


def _links(dims, eps, seed):
    f, _ = fields.recipe_links(dims, eps, seed)
    return f.numpy()


def test_unit_links_give_the_free_field_coefficients():
    dims = (4, 4, 4, 6)
    vol = int(np.prod(dims))
    unit = np.broadcast_to(np.eye(3, dtype=np.complex128), (4, vol, 3, 3)).copy()
    x, w = smear.hisq_links(dims, unit)
    assert np.abs(x - 9 / 8 * np.eye(3)).max() < 1e-14
    assert np.abs(w + 1 / 24 * np.eye(3)).max() < 1e-15
    x2, w2 = smear.hisq_links(dims, unit, eps_naik=0.4)
    assert np.abs(w2 - (-1 / 24 + 0.4 / 8) * np.eye(3)).max() < 1e-15
    assert np.abs(x2 - x).max() == 0.0


def _paths(mu):
    """(coefficient name, list of (direction, sign)) of the paths from x to x + mu."""
    others = [d for d in range(4) if d != mu]
    yield "c1", [(mu, 1)]
    for nu in others:
        for s in (1, -1):
            yield "c3", [(nu, s), (mu, 1), (nu, -s)]
            yield "cl", [(nu, s), (nu, s), (mu, 1), (nu, -s), (nu, -s)]
    for nu, rho in itertools.permutations(others, 2):
        for s, t in itertools.product((1, -1), repeat=2):
            yield "c5", [(rho, t), (nu, s), (mu, 1), (nu, -s), (rho, -t)]
    for nu, rho, sig in itertools.permutations(others, 3):
        for s, t, u in itertools.product((1, -1), repeat=3):
            yield "c7", [(sig, u), (rho, t), (nu, s), (mu, 1), (nu, -s), (rho, -t), (sig, -u)]


def _path_product(phase, dims, start, steps):
    """product of the U(1) link values along the path (phase[mu][t, z, y, x] = e^{i theta})."""
    pos = list(start)  # (x, y, z, t)
    val = 1.0 + 0j
    for d, s in steps:
        if s > 0:
            val *= phase[d][pos[3], pos[2], pos[1], pos[0]]
            pos[d] = (pos[d] + 1) % dims[d]
        else:
            pos[d] = (pos[d] - 1) % dims[d]
            val *= np.conj(phase[d][pos[3], pos[2], pos[1], pos[0]])
    return val


def _smear_scalar(phase, dims, coef):
    nx, ny, nz, nt = dims
    out = np.zeros_like(phase)
    for mu in range(4):
        paths = list(_paths(mu))
        for t, z, y, x in itertools.product(range(nt), range(nz), range(ny), range(nx)):
            acc = 0j
            for name, steps in paths:
                if coef[name] != 0.0:
                    acc += coef[name] * _path_product(phase, dims, (x, y, z, t), steps)
            out[mu][t, z, y, x] = acc
    return out


def test_abelian_links_match_explicit_path_sums():
    dims = (4, 4, 4, 4)
    nx, ny, nz, nt = dims
    rng = np.random.default_rng(7)
    theta = rng.uniform(-np.pi, np.pi, size=(4, nt, nz, ny, nx))
    phase = np.exp(1j * theta)
    u4 = phase[..., None, None] * np.eye(3)
    thin = smear.from_4d(dims, u4)
    x, w = smear.hisq_links(dims, thin)
    x4, w4 = smear.to_4d(dims, x), smear.to_4d(dims, w)
    # brute force, scalar
    lev1 = _smear_scalar(phase, dims, dict(c1=1 / 8, c3=1 / 16, c5=1 / 64, c7=1 / 384, cl=0.0))
    proj = lev1 / np.abs(lev1)
    lev2 = _smear_scalar(proj, dims, dict(c1=1.0, c3=1 / 16, c5=1 / 64, c7=1 / 384, cl=-1 / 8))
    naik = np.zeros_like(proj)
    for mu in range(4):
        naik[mu] = -1 / 24 * proj[mu] * smear.shift(proj[mu], mu, 1) * smear.shift(proj[mu], mu, 2)
    assert np.abs(x4 - lev2[..., None, None] * np.eye(3)).max() < 1e-13
    assert np.abs(w4 - naik[..., None, None] * np.eye(3)).max() < 1e-14


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (4, 6, 4, 6)])
def test_gauge_covariance(dims):
    thin = _links(dims, 0.5, 91)
    x, w = smear.hisq_links(dims, thin)
    nx, ny, nz, nt = dims
    om = fields.gauge_transform_lex(dims, 3000).numpy().reshape(nt, nz, ny, nx, 3, 3)  # lexicographic = 4D order
    u4 = smear.to_4d(dims, thin)
    ut = np.empty_like(u4)
    for mu in range(4):
        ut[mu] = smear.mm(smear.mm(om, u4[mu]), smear.dag(smear.shift(om, mu, 1)))
    xt, wt = smear.hisq_links(dims, smear.from_4d(dims, ut))
    x4, w4, xt4, wt4 = (smear.to_4d(dims, a) for a in (x, w, xt, wt))
    for mu in range(4):
        want_x = smear.mm(smear.mm(om, x4[mu]), smear.dag(smear.shift(om, mu, 1)))
        want_w = smear.mm(smear.mm(om, w4[mu]), smear.dag(smear.shift(om, mu, 3)))
        assert np.abs(xt4[mu] - want_x).max() < 1e-13
        assert np.abs(wt4[mu] - want_w).max() < 1e-14


def test_projection_is_unitary_and_idempotent():
    dims = (4, 4, 4, 4)
    thin = _links(dims, 0.5, 93)
    u4 = smear.to_4d(dims, thin)
    v = smear.smear_level(u4, u4, **smear.LEVEL1)
    w = smear.project_u3(v)
    eye = np.eye(3)
    assert np.abs(smear.mm(smear.dag(w), w) - eye).max() < 1e-13
    assert np.abs(smear.project_u3(w) - w).max() < 1e-13
    assert np.abs(smear.project_u3(u4) - u4).max() < 1e-13
    # the polar factor: V = W H with H = W^+ V Hermitian positive definite
    h = smear.mm(smear.dag(w), v)
    assert np.abs(h - smear.dag(h)).max() < 1e-13
    assert np.linalg.eigvalsh(0.5 * (h + smear.dag(h))).min() > 0.0

"""Pins of the oracle's point-source propagator and meson correlators (oracle.point_propagator,
oracle.meson_correlators; hadronic correlators with point sources, Sec. 3.3).

* Site coordinates of the canonical layout against the C oracle's index inverse, which the
  golden index table pins (Sec. 4.3).
* The propagator equals the source columns of the dense inverse of the full M = 2m + D on 4^4,
  for an even and an odd source: pins the even-odd reconstruction (the 2m and the sign of the
  odd part) independently of it.
* Ward identity of the staggered action: sum_x |G(x, y)|^2 = (M^-1 M^-+)(y, y)
  = Re tr G(y, y) / (2m) (M^+ M = M M^+ = 4m^2 - D^2, whose inverse is parity-diagonal, and
  M^-1 = (2m - D)(4m^2 - D^2)^-1 has no D part on the diagonal): the pion correlator summed over
  the slices against the propagator's own diagonal, in every direction.
* Sign bookkeeping of the eight channels: the Walsh-Hadamard combination
  sum_S (-1)^|S & T| C_S(tau) = 8 x (the |G|^2 summed over the slice sites whose transverse
  offsets have parity pattern T), the right side summed site by site in a plain loop.
* Gauge invariance (random SU(3) transform) and invariance under translation of links and
  source by two sites.
"""
import numpy as np
import pytest
import torch

import oracle
from hisq_inputs import fields


def _np(t):
    return t.detach().cpu().numpy() if hasattr(t, "detach") else t


def _links(dims, eps, seed):
    fat, lng = fields.recipe_links(dims, eps, seed)
    return _np(fat), _np(lng)


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 8, 4)])
def test_site_coords_match_index_inverse(dims):
    c = oracle.site_coords_all(dims)
    V = int(np.prod(dims))
    for i in range(0, V, max(1, V // 97)):
        assert tuple(c[i]) == oracle.coords(dims, i)
    assert tuple(c[V - 1]) == oracle.coords(dims, V - 1)


@pytest.mark.parametrize("src", [(1, 2, 3, 0), (0, 1, 3, 2)])  # odd, even
def test_propagator_matches_dense_inverse_4x4(src):
    dims, m = (4, 4, 4, 4), 0.1
    fat, lng = _links(dims, 0.3, 61)
    G = oracle.point_propagator(dims, fat, lng, m, src, tol=1e-13)
    Minv = np.linalg.inv(oracle.dense_M(dims, fat, lng, m))
    ci = oracle.eo_index(dims, src)
    V = int(np.prod(dims))
    for c in range(3):
        want = Minv[:, 3 * ci + c].reshape(V, 3)
        assert np.abs(G[c] - want).max() <= 1e-10 * np.abs(want).max()


@pytest.mark.parametrize("dims,src", [((4, 4, 4, 8), (1, 0, 2, 5)), ((6, 4, 4, 6), (2, 3, 0, 0))])
def test_ward_identity(dims, src):
    m = 0.07
    fat, lng = _links(dims, 0.5, 62)
    G = oracle.point_propagator(dims, fat, lng, m, src, tol=1e-13)
    ci = oracle.eo_index(dims, src)
    diag = sum(G[c, ci, c] for c in range(3))
    want = diag.real / (2 * m)
    assert abs(diag.imag) <= 1e-9 * abs(diag)
    for d in range(4):
        C = oracle.meson_correlators(dims, G, src, d)
        assert C.shape == (8, dims[d])
        assert abs(C[0].sum() - want) <= 1e-9 * want
        assert (C[0] > 0).all()


def test_channel_signs_walsh_hadamard():
    dims, m, src = (4, 6, 4, 4), 0.1, (3, 2, 1, 1)
    fat, lng = _links(dims, 0.5, 63)
    G = oracle.point_propagator(dims, fat, lng, m, src, tol=1e-12)
    V = int(np.prod(dims))
    w = np.zeros(V)
    for i in range(V):
        w[i] = sum(abs(G[c, i, a]) ** 2 for c in range(3) for a in range(3))
    for d in (1, 3):
        C = oracle.meson_correlators(dims, G, src, d)
        trans = [mu for mu in range(4) if mu != d]
        want = np.zeros((8, dims[d]))
        for i in range(V):
            x = oracle.coords(dims, i)
            tau = (x[d] - src[d]) % dims[d]
            T = 0
            for k, mu in enumerate(trans):
                if (x[mu] - src[mu]) % 2:
                    T |= 1 << k
            want[T, tau] += w[i]
        for T in range(8):
            comb = sum((-1) ** bin(S & T).count("1") * C[S] for S in range(8))
            assert np.abs(comb - 8 * want[T]).max() <= 1e-12 * C[0].max()


def _gauge_rotate(dims, U, Om):
    out = torch.empty_like(U)
    for mu in range(4):
        out[mu] = Om @ U[mu] @ fields._shift_lex(Om, dims, mu, 1).conj().transpose(-1, -2)
    return out


def test_gauge_invariance():
    dims, m, src = (4, 4, 6, 4), 0.1, (2, 1, 3, 0)
    U = fields.thin_links(dims, 0.5, 64)
    Up = _gauge_rotate(dims, U, fields.gauge_transform_lex(dims, 3001))
    corr = []
    for u in (U, Up):
        fat = _np(fields.lex_links_to_canonical(u, dims))
        lng = _np(fields.lex_links_to_canonical(fields.long_from_thin_lex(u, dims), dims))
        G = oracle.point_propagator(dims, fat, lng, m, src, tol=1e-13)
        corr.append(np.stack([oracle.meson_correlators(dims, G, src, d)[:, :4] for d in range(4)]))
    assert np.abs(corr[0] - corr[1]).max() <= 1e-9 * np.abs(corr[0]).max()


@pytest.mark.parametrize("mu", [1, 3])
def test_translation_by_two(mu):
    # links U'(x) = U(x + 2 mu) with source s give the correlators of U with source s + 2 mu
    # (a wrap in t flips the sign of G on some sites, which |G|^2 does not see)
    dims, m, src = (4, 6, 4, 6), 0.1, (1, 1, 2, 3)
    U = fields.thin_links(dims, 0.5, 65)
    Us = torch.stack([fields._shift_lex(U[nu], dims, mu, 2) for nu in range(4)])
    src2 = list(src)
    src2[mu] = (src2[mu] + 2) % dims[mu]
    res = []
    for u, s in ((Us, src), (U, tuple(src2))):
        fat = _np(fields.lex_links_to_canonical(u, dims))
        lng = _np(fields.lex_links_to_canonical(fields.long_from_thin_lex(u, dims), dims))
        G = oracle.point_propagator(dims, fat, lng, m, s, tol=1e-13)
        res.append(np.stack([oracle.meson_correlators(dims, G, s, d)[:, :4] for d in range(4)]))
    assert np.abs(res[0] - res[1]).max() <= 1e-9 * np.abs(res[0]).max()

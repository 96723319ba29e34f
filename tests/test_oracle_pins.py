"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each pin is chosen so that a plausible mistake in the oracle fails it:
  * index formula (Sec. 4.3): hand-evaluated golden indices, bijection, even sites first;
  * operation counts (Sec. 5.1): 1146 flop, 288 + 96 + 6 words per site, intensities;
  * free field (unit links): dense spectrum on 4^4 and plane waves on 8^4 against the
    closed form 4[m^2 + sum_mu (c1 sin p_mu + c3 sin 3p_mu)^2], antiperiodic in t
    -> pins the hop lengths, coefficients, staggered phases and time boundary sign;
  * anti-Hermiticity D_oe = -D_eo^+ -> pins the daggers and signs of backward hops;
  * gauge covariance under random SU(3) -> pins which site's link each hop uses;
  * translation by two sites commutes with D;
  * CG / multi-shift CG against dense solves, multi-shift with one shift = CG.
"""
import math
import os

import numpy as np
import pytest
import torch

import oracle
from hisq_inputs import fields

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _np(t):
    return t.detach().cpu().numpy() if hasattr(t, "detach") else t


def test_rng_matches_published_splitmix64():
    # the torch generator must reproduce the published splitmix64 sequence bit for bit
    for seed in (0, 1, 1000, 2**40 + 7):
        n = torch.tensor([0, 1, 2, 12345, 2**33 + 5, 2**50 + 1], dtype=torch.int64)
        got = fields.random_bits(seed, n)
        key = fields.splitmix64_ref(seed, 0)
        for i, c in enumerate(n.tolist()):
            want = fields.splitmix64_ref(key, c)
            assert (int(got[i]) & ((1 << 64) - 1)) == want


def test_su3_generator_is_special_unitary():
    U = fields.thin_links((4, 4, 4, 4), 0.5, 7)
    U = U.reshape(-1, 3, 3)
    eye = torch.eye(3, dtype=torch.complex128)
    assert (U.conj().transpose(-1, -2) @ U - eye).abs().max() < 1e-14
    assert (torch.linalg.det(U) - 1).abs().max() < 1e-14


def test_eo_index_golden_and_bijection():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "eo_index.txt")) if l.strip() and not l.startswith("#")]
    assert len(rows) >= 10
    for r in rows:
        v = [int(a) for a in r]
        dims, x, want = v[:4], v[4:8], v[8]
        assert oracle.eo_index(dims, x) == want
        assert oracle.coords(dims, want) == tuple(x)
    dims = (6, 4, 4, 8)
    V = int(np.prod(dims))
    seen = set()
    for t in range(dims[3]):
        for z in range(dims[2]):
            for y in range(dims[1]):
                for x in range(dims[0]):
                    i = oracle.eo_index(dims, (x, y, z, t))
                    assert (i < V // 2) == ((x + y + z + t) % 2 == 0)
                    seen.add(i)
    assert seen == set(range(V))


def test_operation_counts_match_paper():
    vals = {}
    for l in open(os.path.join(GOLDEN, "paper_counts.txt")):
        if l.strip() and not l.startswith("#"):
            k, v = l.split()
            vals[k] = float(v)
    dims = (4, 4, 4, 4)
    fat, lng = fields.recipe_links(dims, 0.3, 1000)
    src = fields.gaussian_source(dims, 2000)[0]
    for site in (0, 17, 127):
        fl, lw, nw, ow = oracle.count_site(dims, fat, lng, src, site)
        assert fl == vals["flops"] and lw == vals["link_words"]
        assert nw == vals["neighbour_words"] and ow == vals["output_words"]
    words = vals["link_words"] + vals["neighbour_words"] + vals["output_words"]
    assert round(vals["flops"] / (4 * words), 2) == vals["intensity_fp32"]
    assert math.floor(100 * vals["flops"] / (8 * words)) / 100 == vals["intensity_fp64"]


def _free_spectrum(dims, m, c1, c3):
    ps = []
    for mu, n in enumerate(dims):
        k = np.arange(n)
        p = 2 * np.pi * (k + (0.5 if mu == 3 else 0.0)) / n
        ps.append((c1 * np.sin(p) + c3 * np.sin(3 * p)) ** 2)
    tot = ps[0][:, None, None, None] + ps[1][None, :, None, None] + ps[2][None, None, :, None] + ps[3][None, None, None, :]
    lam = 4 * (m * m + tot.ravel())
    return np.sort(np.repeat(lam, 3))


@pytest.mark.parametrize("c1,c3", [(9 / 8, -1 / 24), (1.0, -1 / 24), (1.0, 0.0)])
def test_free_field_dense_spectrum_4x4(c1, c3):
    dims, m = (4, 4, 4, 4), 0.1
    fat, lng = fields.unit_links(dims, c1, c3)
    A = oracle.dense_A(dims, fat, lng, m)
    ev = np.sort(np.linalg.eigvalsh(A))
    full = _free_spectrum(dims, m, c1, c3)
    want = full[::2]
    assert np.abs(full[0::2] - full[1::2]).max() < 1e-12   # even/odd blocks are isospectral
    assert np.abs(ev - want).max() < 1e-12


def test_free_field_plane_waves_8x4():
    dims, m, c1, c3 = (8, 8, 8, 8), 0.1, 9 / 8, -1 / 24
    fat, lng = fields.unit_links(dims, c1, c3)
    V, Vh = 8 ** 4, 8 ** 4 // 2
    lex = fields.lex_of_eo(dims)[:Vh]
    x, y, z, t = [c[lex].numpy() for c in fields.lex_coords(dims)]
    rng = np.random.default_rng(5)
    for n in [(0, 0, 0, 0), (1, 2, 3, 4), (7, 0, 5, 2), (3, 3, 1, 7)]:
        p = [2 * np.pi * n[0] / 8, 2 * np.pi * n[1] / 8, 2 * np.pi * n[2] / 8, 2 * np.pi * (n[3] + 0.5) / 8]
        phase = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
        u = rng.normal(size=3) + 1j * rng.normal(size=3)
        phi = phase[:, None] * u[None, :]
        lam = 4 * (m * m + sum((c1 * math.sin(q) + c3 * math.sin(3 * q)) ** 2 for q in p))
        Aphi = oracle.mdagm(dims, fat, lng, m, phi)
        assert np.abs(Aphi - lam * phi).max() < 1e-12 * lam


def _random_links(dims, eps=0.5, seed=11):
    fat, lng = fields.recipe_links(dims, eps, seed)
    return _np(fat), _np(lng)


def test_anti_hermiticity_dense_4x4():
    dims = (4, 4, 4, 4)
    fat, lng = _random_links(dims)
    Deo = oracle.dense_D(dims, fat, lng, 0)
    Doe = oracle.dense_D(dims, fat, lng, 1)
    assert np.abs(Doe + Deo.conj().T).max() < 1e-14


@pytest.mark.parametrize("dims", [(6, 4, 4, 4), (8, 8, 8, 8), (4, 6, 8, 10)])
def test_anti_hermiticity_random_vectors(dims):
    fat, lng = _random_links(dims, seed=12)
    psi = _np(fields.gaussian_source(dims, 21))[0]
    phi = _np(fields.gaussian_source(dims, 22))[0]
    lhs = np.vdot(psi, oracle.dslash(dims, fat, lng, phi, 0))     # <psi_e, D_eo phi_o>
    rhs = np.vdot(oracle.dslash(dims, fat, lng, psi, 1), phi)     # <D_oe psi_e, phi_o>
    assert abs(lhs + rhs) <= 1e-14 * abs(lhs)


def _gauge_rotate(dims, U_lex, Om_lex):
    """U'_mu(x) = Om(x) U_mu(x) Om(x+mu)^+ on lexicographic fields."""
    out = torch.empty_like(U_lex)
    for mu in range(4):
        out[mu] = Om_lex @ U_lex[mu] @ fields._shift_lex(Om_lex, dims, mu, 1).conj().transpose(-1, -2)
    return out


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 4, 8)])
def test_gauge_covariance(dims):
    U = fields.thin_links(dims, 0.5, 31)
    Om = fields.gauge_transform_lex(dims, 3000)
    Up = _gauge_rotate(dims, U, Om)
    fat = _np(fields.lex_links_to_canonical(U, dims))
    lng = _np(fields.lex_links_to_canonical(fields.long_from_thin_lex(U, dims), dims))
    fatp = _np(fields.lex_links_to_canonical(Up, dims))
    lngp = _np(fields.lex_links_to_canonical(fields.long_from_thin_lex(Up, dims), dims))
    Om_c = _np(Om[fields.lex_of_eo(dims)])                      # canonical order
    Vh = int(np.prod(dims)) // 2
    for p in (0, 1):
        phi = _np(fields.gaussian_source(dims, 40 + p))[0]      # parity 1-p
        Om_in = Om_c[(1 - p) * Vh:(2 - p) * Vh]
        Om_out = Om_c[p * Vh:(p + 1) * Vh]
        lhs = oracle.dslash(dims, fatp, lngp, np.einsum("sij,sj->si", Om_in, phi), p)
        rhs = np.einsum("sij,sj->si", Om_out, oracle.dslash(dims, fat, lng, phi, p))
        assert np.abs(lhs - rhs).max() <= 1e-13 * np.abs(rhs).max()


def test_translation_by_two_commutes():
    dims = (6, 4, 8, 4)
    U = fields.thin_links(dims, 0.5, 33)
    lng = fields.long_from_thin_lex(U, dims)
    phi_full = fields.gaussian_full(dims, 50)[0]        # canonical order, all sites
    lex_of = fields.lex_of_eo(dims)
    eo_of = fields.eo_of_lex(dims)
    Vh = int(np.prod(dims)) // 2
    for mu in (0, 1, 2):
        Us = torch.stack([fields._shift_lex(U[nu], dims, mu, 2) for nu in range(4)])
        Ls = torch.stack([fields._shift_lex(lng[nu], dims, mu, 2) for nu in range(4)])
        phi_lex = phi_full[eo_of]                         # lexicographic
        phis = fields._shift_lex(phi_lex, dims, mu, 2)[lex_of]
        a = oracle.dslash(dims, fields.lex_links_to_canonical(Us, dims), fields.lex_links_to_canonical(Ls, dims),
                          phis[Vh:].numpy(), 0)
        full_out = np.zeros((2 * Vh, 3), dtype=np.complex128)
        full_out[:Vh] = oracle.dslash(dims, fields.lex_links_to_canonical(U, dims),
                                      fields.lex_links_to_canonical(lng, dims), phi_full[Vh:].numpy(), 0)
        shifted = fields._shift_lex(torch.from_numpy(full_out)[eo_of], dims, mu, 2)[lex_of]
        assert np.abs(a - shifted[:Vh].numpy()).max() < 1e-13


def test_phased_links_reproduce_operator():
    dims = (4, 6, 4, 6)
    fat, lng = _random_links(dims, seed=14)
    fp, lp = oracle.phase_links(dims, fat, 1), oracle.phase_links(dims, lng, 3)
    phi = _np(fields.gaussian_source(dims, 60))[0]
    for p in (0, 1):
        assert np.abs(oracle.dslash(dims, fp, lp, phi, p, phased=True) - oracle.dslash(dims, fat, lng, phi, p)).max() < 1e-15


def test_normal_operator_is_hpd_above_4m2():
    dims, m = (4, 4, 4, 4), 0.05
    fat, lng = _random_links(dims, seed=15)
    A = oracle.dense_A(dims, fat, lng, m)
    assert np.abs(A - A.conj().T).max() < 1e-14
    ev = np.linalg.eigvalsh(A)
    assert ev.min() >= 4 * m * m * (1 - 1e-12)


def test_cg_matches_dense_solve_4x4():
    dims, m = (4, 4, 4, 4), 0.1
    fat, lng = _random_links(dims, eps=0.3, seed=1000)
    b = _np(fields.gaussian_source(dims, 2000))[0]
    A = oracle.dense_A(dims, fat, lng, m)
    import scipy.linalg as sl
    xd = sl.cho_solve(sl.cho_factor(A), b.reshape(-1)).reshape(b.shape)
    x, it, rit, rtrue = oracle.cg(dims, fat, lng, m, b, tol=1e-10)
    assert rtrue <= 1e-10 and it > 5
    kappa = np.linalg.cond(A)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) <= kappa * 1e-10


def test_multishift_matches_dense_solves_4x4():
    dims, m = (4, 4, 4, 4), 0.05
    fat, lng = _random_links(dims, eps=0.5, seed=16)
    b = _np(fields.gaussian_source(dims, 70))[0]
    A = oracle.dense_A(dims, fat, lng, m)
    sig = np.exp(np.linspace(np.log(1e-5), 0, 14))[::-1].copy()      # any order
    x, it, res = oracle.multishift_cg(dims, fat, lng, m, sig, b, 1e-11)
    assert (res <= 1e-10).all()
    n = A.shape[0]
    for s, sg in enumerate(sig):
        xd = np.linalg.solve(A + sg * np.eye(n), b.reshape(-1))
        assert np.linalg.norm(x[s].reshape(-1) - xd) / np.linalg.norm(xd) < 1e-9


def test_multishift_single_shift_is_cg():
    dims, m = (6, 4, 4, 4), 0.1
    fat, lng = _random_links(dims, seed=17)
    b = _np(fields.gaussian_source(dims, 71))[0]
    x1, it1, res = oracle.multishift_cg(dims, fat, lng, m, [0.0], b, 1e-10)
    x2, it2, _, _ = oracle.cg(dims, fat, lng, m, b, tol=1e-10)
    assert it1 == it2
    # identical recurrences; OpenMP reduction order differs between the two runs, so the
    # iterates agree to the solve tolerance rather than to the last bit
    assert np.linalg.norm(x1[0] - x2) < 1e-9 * np.linalg.norm(x2)


def test_multishift_vs_independent_cg_6x4():
    dims, m = (6, 6, 6, 4), 0.02
    fat, lng = _random_links(dims, seed=18)
    b = _np(fields.gaussian_source(dims, 72))[0]
    sig = [0.0, 1e-3, 0.1, 1.0]
    x, it, res = oracle.multishift_cg(dims, fat, lng, m, sig, b, 1e-11)
    for s, sg in enumerate(sig):
        # (A + sigma) = A at mass m' with 4m'^2 = 4m^2 + sigma
        ms = math.sqrt(m * m + sg / 4)
        xs, _, _, rt = oracle.cg(dims, fat, lng, ms, b, tol=1e-11)
        assert np.linalg.norm(x[s] - xs) / np.linalg.norm(xs) < 1e-8


def test_rational_apply_matches_dense_spectral_evaluation():
    # r(A) b = alpha0 b + sum_s alpha_s (A + sigma_s)^-1 b from one multi-shift solve, against
    # V r(Lambda) V^+ b with the dense eigendecomposition of A on 4^4 (a dropped coefficient,
    # a shift applied with the wrong sign or to the wrong term fails it)
    from hisq_inputs import rational
    dims, m = (4, 4, 4, 4), 0.1
    fat, lng = fields.recipe_links(dims, 0.3, 48)
    fat, lng = fat.numpy(), lng.numpy()
    b = fields.gaussian_source(dims, 96)[0].numpy()
    A = oracle.dense_A(dims, fat, lng, m)
    lam, V = np.linalg.eigh(A)
    a0, al, sg = rational.inv_sqrt(24, 0.9 * lam[0], 1.1 * lam[-1])
    a0 = 0.25  # exercise the constant term as well
    x, res = oracle.rational_apply(dims, fat, lng, m, a0, al, sg, b, tol=1e-13)
    assert res.max() <= 1e-12
    r_lam = a0 + sum(a / (lam + s) for a, s in zip(al, sg))
    want = V @ (r_lam * (V.conj().T @ b.reshape(-1)))
    assert np.linalg.norm(x.reshape(-1) - want) <= 1e-11 * np.linalg.norm(want)
    # and r approximates A^-1/2 to the quadrature's accuracy on this spectrum
    exact = V @ ((lam ** -0.5) * (V.conj().T @ b.reshape(-1)))
    err = np.linalg.norm((x.reshape(-1) - a0 * b.reshape(-1)) - exact) / np.linalg.norm(exact)
    assert err <= 2e-3


def test_condensate_trace_identity_4x4():
    # Tr M^-1 over the full lattice (dense M = 2m + D) = 4 m Tr_e A^-1 (even sites)
    dims, m = (4, 4, 4, 4), 0.1
    fat, lng = _random_links(dims, 0.3, 49)
    M = oracle.dense_M(dims, fat, lng, m)
    A = oracle.dense_A(dims, fat, lng, m)
    full = np.trace(np.linalg.inv(M))
    want = 4 * m * np.trace(np.linalg.inv(A))
    assert abs(full.imag) <= 1e-12 * abs(full) and abs(full - want) <= 1e-11 * abs(want)


def test_condensate_free_field_closed_form():
    # unit links: Tr_e A^-1 = sum over the even block's free spectrum 4 [m^2 + sum (c1 sin p + c3 sin 3p)^2]
    dims, m, c1, c3 = (4, 4, 4, 4), 0.1, 9 / 8, -1 / 24
    fat, lng = fields.unit_links(dims, c1, c3)
    A = oracle.dense_A(dims, fat.numpy(), lng.numpy(), m)
    lam = _free_spectrum(dims, m, c1, c3)[::2]
    assert abs(np.trace(np.linalg.inv(A)).real - np.sum(1.0 / lam)) <= 1e-11 * np.sum(1.0 / lam)


def test_condensate_basis_noise_gives_exact_trace():
    # the estimator with every unit vector of the even sites as "noise" is the exact trace
    dims, m = (4, 4, 4, 4), 0.1
    fat, lng = _random_links(dims, 0.3, 50)
    Vh = 128
    eta = np.eye(3 * Vh, dtype=np.complex128).reshape(3 * Vh, Vh, 3)
    s = oracle.condensate_samples(dims, fat, lng, m, eta, tol=1e-13)
    A = oracle.dense_A(dims, fat, lng, m)
    exact = np.trace(np.linalg.inv(A)).real
    assert abs(s.sum() - exact) <= 1e-10 * exact

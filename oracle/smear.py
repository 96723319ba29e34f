"""HISQ link smearing (two levels with a U(3) projection between them), plain numpy FP64.

TEST INFRASTRUCTURE ONLY, like the rest of oracle/.  Follows the paper's description of the HISQ
link treatment (Sec. 3.1): a first level with coefficients c1 = 1/8 for the link and c3 = 1/16,
c5 = 1/64, c7 = 1/384 for the 3-, 5- and 7-link staples, projection of the result to U(3),
and a second level on the projected links with c1 = 1, the same staple coefficients, the Lepage
term c_L = -1/8, and the Naik term c_N = -1/24 + eps/8 built from the projected links.

Staples (my statement of the standard definitions): for a field F_mu(x) of 3x3 matrices that
connects x to x + mu, and nu != mu,
  stap_nu[F]_mu(x) = U_nu(x) F_mu(x+nu) U_nu(x+mu)^+ + U_nu(x-nu)^+ F_mu(x-nu) U_nu(x-nu+mu)
  S3 = sum_nu stap_nu[U]                      (6 paths)
  S5 = sum_{rho} stap_rho[ sum_{nu != rho} stap_nu[U] ]          (24 paths)
  S7 = sum_{sig} stap_sig[ sum_{rho != sig} stap_rho[ sum_{nu != rho, sig} stap_nu[U] ] ]  (48)
  Lepage = sum_nu lep_nu[U], lep_nu the staple whose detour is two steps along nu
  Naik_mu(x) = c_N W_mu(x) W_mu(x+mu) W_mu(x+2mu)
(all sums over directions different from mu).  With unit links the first level is
1/8 + 6/16 + 24/64 + 48/384 = 1, the second 1 + 3/8 + 3/8 + 1/8 - 6/8 = 9/8 and the Naik
link -1/24: the tree-level coefficients of the improved free-field operator.
U(3) projection: W = V (V^+ V)^(-1/2), the unitary factor of the polar decomposition, with the
inverse square root from the eigendecomposition of the Hermitian V^+ V (numpy eigh).

Layout in: links [4][V][3][3] complex128 in the canonical even-odd order of Sec. 4.3 (the
library's input layout).  Internally 4D arrays [Nt][Nz][Ny][Nx][3][3] with periodic shifts.
"""
from __future__ import annotations

import numpy as np

LEVEL1 = dict(c1=1 / 8, c3=1 / 16, c5=1 / 64, c7=1 / 384, cl=0.0)
LEVEL2 = dict(c1=1.0, c3=1 / 16, c5=1 / 64, c7=1 / 384, cl=-1 / 8)


def _eo_perm(dims):
    """lexicographic site index (x fastest) -> canonical even-odd index (Sec. 4.3)."""
    nx, ny, nz, nt = dims
    t, z, y, x = np.meshgrid(np.arange(nt), np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    lex = (x + nx * (y + ny * (z + nz * t))).reshape(-1)
    par = ((x + y + z + t) % 2).reshape(-1)
    vol = nx * ny * nz * nt
    return lex // 2 + (vol // 2) * par  # indexed by lex (the meshgrid order is lexicographic)


def to_4d(dims, links):
    """[4][V][3][3] canonical -> [4][Nt][Nz][Ny][Nx][3][3]."""
    nx, ny, nz, nt = dims
    eo = _eo_perm(dims)
    return np.ascontiguousarray(links[:, eo]).reshape(4, nt, nz, ny, nx, 3, 3)


def from_4d(dims, u4):
    nx, ny, nz, nt = dims
    vol = nx * ny * nz * nt
    eo = _eo_perm(dims)
    out = np.empty((4, vol, 3, 3), dtype=np.complex128)
    out[:, eo] = u4.reshape(4, vol, 3, 3)
    return out


# direction mu = 0..3 is x, y, z, t; in the 4D arrays the axes are (t, z, y, x) = (0, 1, 2, 3)
_AXIS = {0: 3, 1: 2, 2: 1, 3: 0}


def shift(f, mu, n):
    """g(x) = f(x + n mu) (periodic)."""
    return np.roll(f, -n, axis=_AXIS[mu])


def mm(a, b):
    return np.einsum("...ij,...jk->...ik", a, b)


def dag(a):
    return np.conj(np.swapaxes(a, -1, -2))


def stap(u4, f, mu, nu, hops=1):
    """stap_nu[F]_mu(x) for a field F connecting x to x + mu; `hops` steps along nu."""
    un = u4[nu]
    fwd = un
    for k in range(1, hops):
        fwd = mm(fwd, shift(un, nu, k))               # U_nu(x) ... U_nu(x+(hops-1)nu)
    up = mm(mm(fwd, shift(f, nu, hops)), dag(shift(fwd, mu, 1)))
    down_leg = shift(fwd, nu, -hops)                    # U_nu(x-hops nu) ... U_nu(x-nu)
    down = mm(mm(dag(down_leg), shift(f, nu, -hops)), shift(down_leg, mu, 1))
    return up + down


def smear_level(u4, f4, c1, c3, c5, c7, cl):
    """c1 F + c3 S3 + c5 S5 + c7 S7 + cl Lepage, staples built from the links u4 around F = f4."""
    out = np.empty_like(f4)
    for mu in range(4):
        others = [d for d in range(4) if d != mu]
        f = f4[mu]
        acc = c1 * f
        t3 = {nu: stap(u4, f, mu, nu) for nu in others}
        for nu in others:
            acc = acc + c3 * t3[nu]
        for rho in others:
            inner = sum(t3[nu] for nu in others if nu != rho)
            acc = acc + c5 * stap(u4, inner, mu, rho)
        for sig in others:
            inner7 = 0
            for rho in others:
                if rho == sig:
                    continue
                inner5 = sum(t3[nu] for nu in others if nu not in (rho, sig))
                inner7 = inner7 + stap(u4, inner5, mu, rho)
            acc = acc + c7 * stap(u4, inner7, mu, sig)
        if cl != 0.0:
            for nu in others:
                acc = acc + cl * stap(u4, f, mu, nu, hops=2)
        out[mu] = acc
    return out


def project_u3(v):
    """W = V (V^+ V)^(-1/2) for every 3x3 matrix of the array."""
    q = mm(dag(v), v)
    lam, vec = np.linalg.eigh(q)
    inv_sqrt = mm(vec * (lam[..., None, :] ** -0.5), dag(vec))
    return mm(v, inv_sqrt)


def hisq_links(dims, thin, eps_naik=0.0):
    """(fat X, long W) in the canonical [4][V][3][3] layout from thin links U (unphased)."""
    u4 = to_4d(dims, np.asarray(thin, dtype=np.complex128))
    v = smear_level(u4, u4, **LEVEL1)
    w = project_u3(v)
    x = smear_level(w, w, **LEVEL2)
    cn = -1.0 / 24.0 + eps_naik / 8.0
    naik = np.empty_like(w)
    for mu in range(4):
        naik[mu] = cn * mm(mm(w[mu], shift(w[mu], mu, 1)), shift(w[mu], mu, 2))
    return from_4d(dims, x), from_4d(dims, naik)

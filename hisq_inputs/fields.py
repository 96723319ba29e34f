"""Seeded synthetic inputs for the HISQ Dslash and solver workloads.

This module is shared by the FP64 oracle tests and by the GPU library's tests and
benchmarks.  It holds no Dslash or solver arithmetic: only

* a counter-based random number generator (splitmix64 finaliser, Box-Muller),
* random SU(3) matrices U = exp(i eps H) with H = sum_a h_a lambda_a / 2,
* the workload link recipe: fat = c1 U, long = c3 U_mu(x) U_mu(x+mu) U_mu(x+2mu)
  (the synthetic stand-in for HISQ smeared links; c3 = -1/24 is the Naik
  coefficient of the second smearing level, Sec. 3.1),
* Gaussian complex sources on one parity,
* the canonical even-odd site ordering of Sec. 4.3 used to lay those out.

Layouts (all complex128 torch tensors):
  links   [4][V][3][3]   index mu*V + eo(x), row-major 3x3  (Sec. 4.3, link index)
  vectors [nrhs][Vh][3]  one parity, eo half-index           (Sec. 4.3, site index)
where eo(x) = floor(lex/2) + (V/2) * ((x+y+z+t) mod 2) and
lex = x + Nx (y + Ny (z + Nz t)); mu = 0,1,2,3 is x,y,z,t.

Everything is a pure function of (dims, seed, ...), independent of device and
thread order: the value drawn for item n of a stream is splitmix64 output n.
"""
from __future__ import annotations

import math

import torch

_GOLDEN = 0x9E3779B97F4A7C15
_MIX1 = 0xBF58476D1CE4E5B9
_MIX2 = 0x94D049BB133111EB
_M64 = (1 << 64) - 1


def _s64(c: int) -> int:
    """Two's-complement int64 value of an unsigned 64-bit constant."""
    c &= _M64
    return c - (1 << 64) if c >= (1 << 63) else c


def _lsr(z: torch.Tensor, k: int) -> torch.Tensor:
    """Logical right shift of int64 bit patterns."""
    return (z >> k) & ((1 << (64 - k)) - 1)


def splitmix64_mix(z: torch.Tensor) -> torch.Tensor:
    """splitmix64 output finaliser on int64 bit patterns (wrapping arithmetic)."""
    z = (z ^ _lsr(z, 30)) * _s64(_MIX1)
    z = (z ^ _lsr(z, 27)) * _s64(_MIX2)
    return z ^ _lsr(z, 31)


def splitmix64_ref(seed: int, n: int) -> int:
    """Pure-Python splitmix64: output number n (0-based) of the generator seeded with `seed`."""
    z = (seed + (n + 1) * _GOLDEN) & _M64
    z = ((z ^ (z >> 30)) * _MIX1) & _M64
    z = ((z ^ (z >> 27)) * _MIX2) & _M64
    return z ^ (z >> 31)


def _stream_key(seed: int) -> int:
    # decorrelate small consecutive seeds: the key is splitmix64 output 0 of `seed`
    return splitmix64_ref(seed, 0)


def random_bits(seed: int, counters: torch.Tensor) -> torch.Tensor:
    """Output number `counters` of splitmix64 keyed by `seed` (int64 bit patterns)."""
    key = _stream_key(seed)
    z = _s64(key) + (counters + 1) * _s64(_GOLDEN)
    return splitmix64_mix(z)


def uniform(seed: int, counters: torch.Tensor) -> torch.Tensor:
    """Uniform doubles in (0, 1]: top 53 bits of the stream, plus one ulp."""
    b = _lsr(random_bits(seed, counters), 11)
    return (b.to(torch.float64) + 1.0) * (2.0 ** -53)


def normal(seed: int, counters: torch.Tensor) -> torch.Tensor:
    """Standard normal doubles; normal number n uses uniforms 2n and 2n+1 (Box-Muller)."""
    u1 = uniform(seed, 2 * counters)
    u2 = uniform(seed, 2 * counters + 1)
    return torch.sqrt(-2.0 * torch.log(u1)) * torch.cos(2.0 * math.pi * u2)


# ----------------------------------------------------------------------------- lattice order

def volume(dims) -> int:
    nx, ny, nz, nt = dims
    return nx * ny * nz * nt


def check_dims(dims) -> None:
    if len(dims) != 4 or any(int(n) < 4 or int(n) % 2 for n in dims):
        raise ValueError(f"lattice dims must be four even extents >= 4, got {dims}")


def lex_coords(dims, device="cpu"):
    """Coordinates (x, y, z, t) of every site in lexicographic order, x fastest."""
    nx, ny, nz, nt = dims
    lex = torch.arange(volume(dims), device=device, dtype=torch.int64)
    x = lex % nx
    y = (lex // nx) % ny
    z = (lex // (nx * ny)) % nz
    t = lex // (nx * ny * nz)
    return x, y, z, t


def eo_of_lex(dims, device="cpu") -> torch.Tensor:
    """Canonical even-odd index of every lexicographic site (Sec. 4.3)."""
    x, y, z, t = lex_coords(dims, device)
    lex = torch.arange(volume(dims), device=device, dtype=torch.int64)
    par = (x + y + z + t) % 2
    return lex // 2 + par * (volume(dims) // 2)


def lex_of_eo(dims, device="cpu") -> torch.Tensor:
    """Inverse permutation: lexicographic index of every canonical even-odd slot."""
    eo = eo_of_lex(dims, device)
    inv = torch.empty_like(eo)
    inv[eo] = torch.arange(eo.numel(), device=device, dtype=torch.int64)
    return inv


# ----------------------------------------------------------------------------- SU(3)

def gell_mann(device="cpu") -> torch.Tensor:
    """The eight Gell-Mann matrices, [8][3][3] complex128."""
    lam = torch.zeros(8, 3, 3, dtype=torch.complex128)
    lam[0, 0, 1] = lam[0, 1, 0] = 1
    lam[1, 0, 1] = -1j
    lam[1, 1, 0] = 1j
    lam[2, 0, 0] = 1
    lam[2, 1, 1] = -1
    lam[3, 0, 2] = lam[3, 2, 0] = 1
    lam[4, 0, 2] = -1j
    lam[4, 2, 0] = 1j
    lam[5, 1, 2] = lam[5, 2, 1] = 1
    lam[6, 1, 2] = -1j
    lam[6, 2, 1] = 1j
    s3 = 1.0 / math.sqrt(3.0)
    lam[7, 0, 0] = lam[7, 1, 1] = s3
    lam[7, 2, 2] = -2 * s3
    return lam.to(device)


def su3_from_counters(seed: int, counters: torch.Tensor, eps: float) -> torch.Tensor:
    """exp(i eps H) with H = sum_a h_a lambda_a/2, h_a = normal(seed, 8*counter + a).

    `counters` is a 1-D int64 tensor of matrix numbers; returns [n][3][3] complex128.
    """
    dev = counters.device
    a = torch.arange(8, device=dev, dtype=torch.int64)
    h = normal(seed, counters[:, None] * 8 + a[None, :])          # [n][8]
    H = torch.einsum("na,aij->nij", h.to(torch.complex128), gell_mann(dev)) * 0.5
    out = torch.empty_like(H)
    chunk = 1 << 22
    for i in range(0, H.shape[0], chunk):
        out[i:i + chunk] = torch.linalg.matrix_exp(1j * eps * H[i:i + chunk])
    return out


# ----------------------------------------------------------------------------- fields

def _lex_to_canonical_links(lex_links: torch.Tensor, dims) -> torch.Tensor:
    """[4][V][3][3] lexicographic -> canonical even-odd order."""
    perm = lex_of_eo(dims, lex_links.device)
    return lex_links[:, perm].contiguous()


def thin_links(dims, eps: float, seed: int, device="cpu") -> torch.Tensor:
    """Random SU(3) links U_mu(x), lexicographic order [4][V][3][3]; matrix number mu*V + lex."""
    check_dims(dims)
    V = volume(dims)
    out = torch.empty(4, V, 3, 3, dtype=torch.complex128, device=device)
    for mu in range(4):
        cnt = torch.arange(V, device=device, dtype=torch.int64) + mu * V
        out[mu] = su3_from_counters(seed, cnt, eps)
    return out


def _shift_lex(field: torch.Tensor, dims, mu: int, k: int) -> torch.Tensor:
    """field(x + k mu^) for a [V][...] lexicographic field (periodic)."""
    nx, ny, nz, nt = dims
    shaped = field.reshape(nt, nz, ny, nx, *field.shape[1:])
    axis = 3 - mu                    # mu=0 (x) is the fastest axis
    return torch.roll(shaped, shifts=-k, dims=axis).reshape(field.shape)


def recipe_links(dims, eps: float, seed: int, c1: float = 1.0, c3: float = -1.0 / 24.0,
                 device="cpu"):
    """Workload link recipe: (fat, long) canonical [4][V][3][3] complex128, no phases.

    fat_mu(x) = c1 U_mu(x);  long_mu(x) = c3 U_mu(x) U_mu(x+mu) U_mu(x+2mu).
    """
    U = thin_links(dims, eps, seed, device)
    fat = U * c1
    lng = torch.empty_like(U)
    for mu in range(4):
        u1 = _shift_lex(U[mu], dims, mu, 1)
        u2 = _shift_lex(U[mu], dims, mu, 2)
        lng[mu] = c3 * (U[mu] @ u1 @ u2)
        del u1, u2
    return _lex_to_canonical_links(fat, dims), _lex_to_canonical_links(lng, dims)


def long_from_thin_lex(U: torch.Tensor, dims, c3: float = -1.0 / 24.0) -> torch.Tensor:
    """The recipe's long links from arbitrary lexicographic thin links U (used for gauge checks)."""
    lng = torch.empty_like(U)
    for mu in range(4):
        lng[mu] = c3 * (U[mu] @ _shift_lex(U[mu], dims, mu, 1) @ _shift_lex(U[mu], dims, mu, 2))
    return lng


def lex_links_to_canonical(lex_links: torch.Tensor, dims) -> torch.Tensor:
    return _lex_to_canonical_links(lex_links, dims)


def unit_links(dims, c1: float, c3: float, device="cpu"):
    """Free field: fat = c1 * 1, long = c3 * 1 (canonical layout)."""
    V = volume(dims)
    eye = torch.eye(3, dtype=torch.complex128, device=device)
    fat = (c1 * eye).expand(4, V, 3, 3).contiguous()
    lng = (c3 * eye).expand(4, V, 3, 3).contiguous()
    return fat, lng


def gaussian_source(dims, seed: int, nrhs: int = 1, device="cpu") -> torch.Tensor:
    """Gaussian complex 3-vectors on one parity: [nrhs][Vh][3]; Re and Im each N(0,1)."""
    check_dims(dims)
    Vh = volume(dims) // 2
    n = torch.arange(nrhs * Vh * 6, device=device, dtype=torch.int64)
    g = normal(seed, n).reshape(nrhs, Vh, 3, 2)
    return torch.complex(g[..., 0], g[..., 1]).contiguous()


def gaussian_full(dims, seed: int, nvec: int = 1, device="cpu") -> torch.Tensor:
    """Gaussian complex 3-vectors on all sites, canonical order: [nvec][V][3]."""
    check_dims(dims)
    V = volume(dims)
    n = torch.arange(nvec * V * 6, device=device, dtype=torch.int64)
    g = normal(seed, n).reshape(nvec, V, 3, 2)
    return torch.complex(g[..., 0], g[..., 1]).contiguous()


def gauge_transform_lex(dims, seed: int, eps: float = 1.0, device="cpu") -> torch.Tensor:
    """Random SU(3) Omega(x), lexicographic [V][3][3]."""
    V = volume(dims)
    return su3_from_counters(seed, torch.arange(V, device=device, dtype=torch.int64), eps)

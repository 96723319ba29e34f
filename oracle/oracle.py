"""ctypes binding of the FP64 C oracle (hisq_oracle.c) plus a few dense numpy checks.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Arrays are numpy complex128 in
the canonical layouts of Sec. 4.3: links [4][V][3][3], half-lattice vectors
[nrhs][Vh][3], full-lattice fields [C][V][3].
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hisq_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libhisq_oracle.so")
_lock = threading.Lock()
_lib = None

__all__ = [
    "build", "lib", "dslash", "dslash_site", "mdagm", "cg", "cg_fixed", "multishift_cg", "rational_apply",
    "condensate_samples", "dense_M", "site_coords_all", "point_propagator", "meson_correlators",
    "phase_links", "eo_index", "coords", "count_site", "net_layer", "net_layer_backward",
    "net_apply", "net_loss_grad", "net_loss_grad_residual", "fcg", "fcg_dense", "dense_A", "dense_D", "NTAP",
    "set_threads",
]

NTAP = 17


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, -O2, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            _declare(_lib)
    return _lib


def set_threads(n: int) -> None:
    """Number of OpenMP threads the oracle uses (it must be called before the first solve)."""
    os.environ["OMP_NUM_THREADS"] = str(int(n))
    try:
        omp = ctypes.CDLL("libgomp.so.1")
        omp.omp_set_num_threads(ctypes.c_int(int(n)))
    except OSError:
        pass


_P = ctypes.c_void_p
_I = ctypes.c_int
_L = ctypes.c_long
_D = ctypes.c_double


def _declare(L):
    L.ho_dslash.argtypes = [_P, _P, _P, _I, _I, _P, _P, _I]
    L.ho_dslash_site.argtypes = [_P, _P, _P, _I, _P, _L, _P]
    L.ho_count_site.argtypes = [_P, _P, _P, _P, _L, _P]
    L.ho_phase_links.argtypes = [_P, _P, _P, _I]
    L.ho_eo_index.argtypes = [_P, _P, _P]
    L.ho_coords.argtypes = [_P, _L, _P]
    L.ho_mdagm.argtypes = [_P, _P, _P, _I, _D, _P, _P, _I]
    L.ho_cg.argtypes = [_P, _P, _P, _I, _D, _P, _P, _D, _I, _P]
    L.ho_cg.restype = _I
    L.ho_cg_fixed.argtypes = [_P, _P, _P, _D, _P, _P, _I]
    L.ho_cg_fixed.restype = _D
    L.ho_multishift_cg.argtypes = [_P, _P, _P, _I, _D, _I, _P, _P, _P, _P, _I, _P]
    L.ho_multishift_cg.restype = _I
    L.ho_net_layer.argtypes = [_P, _P, _P, _I, _I, _I, _P, _P, _P]
    L.ho_net_layer_backward.argtypes = [_P, _P, _P, _I, _I, _I, _P, _P, _P, _P, _P]
    L.ho_net_apply.argtypes = [_P, _P, _P, _I, _I, _P, _P, _P, _P]
    L.ho_net_loss_grad.argtypes = [_P, _P, _P, _I, _I, _P, _P, _P, _P, _P]
    L.ho_net_loss_grad.restype = _D
    L.ho_fcg.argtypes = [_P, _P, _P, _I, _D, _I, _P, _P, _P, _P, _D, _I, _P]
    L.ho_fcg.restype = _I
    L.ho_fcg_dense.argtypes = [_P, _P, _P, _I, _D, _P, _P, _P, _D, _I, _P]
    L.ho_fcg_dense.restype = _I


def _c(a, dtype=np.complex128):
    """Contiguous numpy array (accepts torch CPU tensors)."""
    if hasattr(a, "detach"):
        a = a.detach().cpu().numpy()
    return np.ascontiguousarray(a, dtype=dtype)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _dims(dims):
    return np.ascontiguousarray(dims, dtype=np.int32)


def _vol(dims):
    return int(np.prod(dims))


def dslash(dims, fat, lng, inp, out_parity, phased=False):
    """out = D_{p,1-p} in for a [nrhs][Vh][3] (or [Vh][3]) half-lattice field."""
    d, F, W, x = _dims(dims), _c(fat), _c(lng), _c(inp)
    Vh = _vol(dims) // 2
    nrhs = x.size // (Vh * 3)
    out = np.empty_like(x)
    lib().ho_dslash(_ptr(d), _ptr(F), _ptr(W), int(phased), int(out_parity), _ptr(x), _ptr(out), nrhs)
    return out


def dslash_site(dims, fat, lng, inp, out_index, phased=False):
    """One output site (canonical index, including the parity offset) of D applied to `inp`."""
    d, F, W, x = _dims(dims), _c(fat), _c(lng), _c(inp)
    out = np.empty(3, dtype=np.complex128)
    lib().ho_dslash_site(_ptr(d), _ptr(F), _ptr(W), int(phased), _ptr(x), int(out_index), _ptr(out))
    return out


def count_site(dims, fat, lng, inp, out_index=0):
    """(flops, link words, neighbour words, output words) for one output site."""
    d, F, W, x = _dims(dims), _c(fat), _c(lng), _c(inp)
    counts = np.zeros(4, dtype=np.int64)
    lib().ho_count_site(_ptr(d), _ptr(F), _ptr(W), _ptr(x), int(out_index), _ptr(counts))
    return tuple(int(c) for c in counts)


def phase_links(dims, links, naik_hops):
    d, U = _dims(dims), _c(links)
    out = np.empty_like(U)
    lib().ho_phase_links(_ptr(d), _ptr(U), _ptr(out), int(naik_hops))
    return out


def eo_index(dims, x):
    d = _dims(dims)
    xx = np.ascontiguousarray(x, dtype=np.int32)
    r = ctypes.c_long(0)
    lib().ho_eo_index(_ptr(d), _ptr(xx), ctypes.byref(r))
    return r.value


def coords(dims, idx):
    d = _dims(dims)
    x = np.zeros(4, dtype=np.int32)
    lib().ho_coords(_ptr(d), int(idx), _ptr(x))
    return tuple(int(v) for v in x)


def mdagm(dims, fat, lng, m, inp, phased=False):
    """(4 m^2 - D_eo D_oe) in on even sites."""
    d, F, W, x = _dims(dims), _c(fat), _c(lng), _c(inp)
    Vh = _vol(dims) // 2
    out = np.empty_like(x)
    lib().ho_mdagm(_ptr(d), _ptr(F), _ptr(W), int(phased), float(m), _ptr(x), _ptr(out), x.size // (Vh * 3))
    return out


def cg(dims, fat, lng, m, b, tol=1e-10, maxiter=100000, x0=None, phased=False):
    """Textbook CG on A x = b. Returns (x, iterations, iterated rel. res., true rel. res.)."""
    d, F, W, bb = _dims(dims), _c(fat), _c(lng), _c(b)
    x = np.zeros_like(bb) if x0 is None else _c(x0).copy()
    st = np.zeros(3)
    lib().ho_cg(_ptr(d), _ptr(F), _ptr(W), int(phased), float(m), _ptr(bb), _ptr(x), float(tol),
                int(maxiter), _ptr(st))
    return x, int(st[0]), float(st[1]), float(st[2])


def cg_fixed(dims, fat, lng, m, b, iters):
    """`iters` CG iterations from x = 0 (timing sample); returns (x, iterated rel. res.)."""
    d, F, W, bb = _dims(dims), _c(fat), _c(lng), _c(b)
    x = np.zeros_like(bb)
    rr = lib().ho_cg_fixed(_ptr(d), _ptr(F), _ptr(W), float(m), _ptr(bb), _ptr(x), int(iters))
    return x, rr


def multishift_cg(dims, fat, lng, m, sigma, b, tol, maxiter=100000, phased=False):
    """Multi-shift CG. Returns (x [nshift][Vh][3], iterations, true rel. residual per shift)."""
    d, F, W, bb = _dims(dims), _c(fat), _c(lng), _c(b)
    sig = np.ascontiguousarray(sigma, dtype=np.float64)
    ns = sig.size
    tols = np.ascontiguousarray(np.broadcast_to(np.asarray(tol, dtype=np.float64), (ns,)))
    x = np.zeros((ns,) + bb.shape, dtype=np.complex128)
    st = np.zeros(1 + ns)
    lib().ho_multishift_cg(_ptr(d), _ptr(F), _ptr(W), int(phased), float(m), ns, _ptr(sig), _ptr(bb),
                           _ptr(x), _ptr(tols), int(maxiter), _ptr(st))
    return x, int(st[0]), st[1:].copy()


def rational_apply(dims, fat, lng, m, alpha0, alpha, sigma, b, tol=1e-12, phased=False):
    """r(A) b = alpha0 b + sum_s alpha_s (A + sigma_s)^-1 b with the (A + sigma_s)^-1 b of one
    multi-shift CG solve (the way RHMC uses the solver, Sec. 3.2).  Returns (x, true residual
    of every shifted system)."""
    xs, _, res = multishift_cg(dims, fat, lng, m, sigma, b, tol, phased=phased)
    out = alpha0 * np.asarray(b, dtype=np.complex128)
    for a, x in zip(alpha, xs):
        out = out + a * x
    return out, res


def condensate_samples(dims, fat, lng, m, eta, tol=1e-12, phased=False):
    """Re <eta_k, A^-1 eta_k> for noise vectors eta_k on even sites, one CG solve each.  Their
    mean estimates Tr_e A^-1, and (1/V) Tr M^-1 = 4 m Tr_e A^-1 / V for M = 2m + D (the diagonal
    blocks of M^-1 = M^+ (M M^+)^-1 are 2m (4m^2 - D^2)^-1, whose even and odd blocks have the
    same spectrum)."""
    eta = np.asarray(eta, dtype=np.complex128)
    out = np.empty(eta.shape[0])
    for k in range(eta.shape[0]):
        x, _, _, _ = cg(dims, fat, lng, m, eta[k], tol=tol, phased=phased)
        out[k] = np.vdot(eta[k], x).real
    return out


def site_coords_all(dims):
    """[V][4] integer (x, y, z, t) of every canonical full-lattice index (Sec. 4.3: the
    lexicographic index, x fastest, halved, with the odd sites after the Vh even ones)."""
    nx, ny, nz, nt = dims
    V = nx * ny * nz * nt
    lex = np.arange(V)
    x = lex % nx
    y = (lex // nx) % ny
    z = (lex // (nx * ny)) % nz
    t = lex // (nx * ny * nz)
    canon = lex // 2 + (V // 2) * ((x + y + z + t) % 2)
    out = np.empty((V, 4), dtype=np.int64)
    out[canon] = np.stack([x, y, z, t], axis=1)
    return out


def point_propagator(dims, fat, lng, m, src, tol=1e-12, phased=False):
    """G = M^-1 on the three colour point sources at site `src` = (x, y, z, t), M = 2m + D on
    the full lattice: [3][V][3] complex (source colour, canonical site, sink colour).

    Solves through the even-odd reduction that the paper's solvers use (Sec. 3.2): for
    M (x_e, x_o) = (b_e, b_o), the even part obeys A x_e = 2m b_e - D_eo b_o with
    A = 4m^2 - D_eo D_oe, and the odd part follows as x_o = (b_o - D_oe x_e) / (2m).
    The even system is solved by the oracle's CG to `tol`."""
    Vh = _vol(dims) // 2
    ci = eo_index(dims, src)
    p, s = divmod(ci, Vh)
    b = np.zeros((2, 3, Vh, 3), dtype=np.complex128)  # [parity][source colour][site][colour]
    for c in range(3):
        b[p, c, s, c] = 1.0
    rhs = 2 * m * b[0] - dslash(dims, fat, lng, b[1], 0, phased)
    G = np.empty((3, 2 * Vh, 3), dtype=np.complex128)
    for c in range(3):
        xe, _, _, _ = cg(dims, fat, lng, m, rhs[c], tol=tol, phased=phased)
        G[c, :Vh] = xe
        G[c, Vh:] = (b[1, c] - dslash(dims, fat, lng, xe, 1, phased)) / (2 * m)
    return G


def meson_correlators(dims, G, src, direction):
    """Point-source staggered meson correlators along `direction` (0..3 = x, y, z, t) from a
    propagator G [3][V][3] of point_propagator (the hadronic correlators of Sec. 3.3, "along
    any direction", with point sources):

      C[S][tau] = sum over sites x with (x_d - src_d) mod N_d = tau of
                  (-1)^(sum over i in S of (x_{e_i} - src_{e_i})) * sum_{a,b} |G_ab(x, src)|^2,

    where e_0 < e_1 < e_2 are the three directions other than d and bit i of S = 0..7
    selects e_i.  These are the eight local staggered meson channels (sign factors from the
    spin-taste phases of the transverse directions); S = 0 is the Goldstone pion.
    Returns [8][N_d] float64."""
    coords = site_coords_all(dims)
    w = np.sum(np.abs(np.asarray(G)) ** 2, axis=(0, 2))  # per canonical site
    d = int(direction)
    trans = [mu for mu in range(4) if mu != d]
    nd = dims[d]
    tau = (coords[:, d] - src[d]) % nd
    out = np.zeros((8, nd))
    for S in range(8):
        parity = np.zeros(len(w), dtype=np.int64)
        for i, mu in enumerate(trans):
            if S >> i & 1:
                parity += coords[:, mu] - src[mu]
        sign = np.where(parity % 2 == 0, 1.0, -1.0)
        out[S] = np.bincount(tau, weights=sign * w, minlength=nd)
    return out


def dense_M(dims, fat, lng, m, phased=False):
    """Dense M = 2m + D on the full lattice, even sites first: [[2m, D_eo], [D_oe, 2m]]."""
    Deo = dense_D(dims, fat, lng, 0, phased)
    Doe = dense_D(dims, fat, lng, 1, phased)
    n = Deo.shape[0]
    eye = np.eye(n, dtype=np.complex128)
    return np.block([[2 * m * eye, Deo], [Doe, 2 * m * eye]])


def net_layer(dims, fat, lng, w, inp, cin, cout, phased=False):
    d, F, W, ww, x = _dims(dims), _c(fat), _c(lng), _c(w), _c(inp)
    out = np.zeros((cout, _vol(dims), 3), dtype=np.complex128)
    lib().ho_net_layer(_ptr(d), _ptr(F), _ptr(W), int(phased), cin, cout, _ptr(ww), _ptr(x), _ptr(out))
    return out


def net_layer_backward(dims, fat, lng, w, inp, gout, cin, cout, phased=False, want_gin=True):
    d, F, W, ww, x, g = _dims(dims), _c(fat), _c(lng), _c(w), _c(inp), _c(gout)
    gw = np.zeros((NTAP, cout, cin), dtype=np.complex128)
    gin = np.zeros((cin, _vol(dims), 3), dtype=np.complex128) if want_gin else None
    lib().ho_net_layer_backward(_ptr(d), _ptr(F), _ptr(W), int(phased), cin, cout, _ptr(ww), _ptr(x),
                                _ptr(g), _ptr(gin) if want_gin else None, _ptr(gw))
    return gin, gw


def net_apply(dims, fat, lng, chans, w, b_even, phased=False):
    d, F, W, ww, b = _dims(dims), _c(fat), _c(lng), _c(w), _c(b_even)
    ch = np.ascontiguousarray(chans, dtype=np.int32)
    z = np.zeros_like(b)
    lib().ho_net_apply(_ptr(d), _ptr(F), _ptr(W), int(phased), len(chans) - 1, _ptr(ch), _ptr(ww),
                       _ptr(b), _ptr(z))
    return z


def net_loss_grad(dims, fat, lng, chans, w, b_even, x_even, phased=False):
    d, F, W, ww, b, x = _dims(dims), _c(fat), _c(lng), _c(w), _c(b_even), _c(x_even)
    ch = np.ascontiguousarray(chans, dtype=np.int32)
    gw = np.zeros_like(ww)
    loss = lib().ho_net_loss_grad(_ptr(d), _ptr(F), _ptr(W), int(phased), len(chans) - 1, _ptr(ch),
                                  _ptr(ww), _ptr(b), _ptr(x), _ptr(gw))
    return loss, gw


def net_loss_grad_residual(dims, fat, lng, chans, w, b_even, x_even, m, phased=False):
    """Residual-norm loss |A (K b - x)|^2 / |b|^2 of one pair and its weight gradient.

    A = 4 m^2 - D_eo D_oe.  The forward pass runs the layers on the full lattice (b on the
    even sites, zero on the odd ones) and keeps the even sites of the output, z = K b.
    With e = z - x the gradient with respect to the output is 2 A^2 e / |b|^2 (A is
    Hermitian), zero on odd sites, and is carried back through the layers with
    net_layer_backward.  Gradients use the convention d/dRe + i d/dIm, as net_loss_grad.
    """
    V = _vol(dims)
    Vh = V // 2
    b = np.asarray(b_even, dtype=np.complex128).reshape(Vh, 3)
    x = np.asarray(x_even, dtype=np.complex128).reshape(Vh, 3)
    w = np.asarray(w, dtype=np.complex128)
    nl = len(chans) - 1
    acts = [np.zeros((1, V, 3), dtype=np.complex128)]
    acts[0][0, :Vh] = b
    ws, off = [], 0
    for l in range(nl):
        n = NTAP * chans[l + 1] * chans[l]
        ws.append(w[off:off + n].reshape(NTAP, chans[l + 1], chans[l]))
        off += n
        acts.append(net_layer(dims, fat, lng, ws[l], acts[l], chans[l], chans[l + 1], phased))
    e = acts[-1][0, :Vh] - x
    Ae = mdagm(dims, fat, lng, m, e, phased=phased)
    A2e = mdagm(dims, fat, lng, m, Ae, phased=phased)
    bb = float(np.vdot(b, b).real)
    loss = float(np.vdot(Ae, Ae).real) / bb
    g = np.zeros((1, V, 3), dtype=np.complex128)
    g[0, :Vh] = 2.0 * A2e / bb
    grads = [None] * nl
    for l in reversed(range(nl)):
        gin, gw = net_layer_backward(dims, fat, lng, ws[l], acts[l], g, chans[l], chans[l + 1], phased,
                                     want_gin=l > 0)
        grads[l] = gw.reshape(-1)
        g = gin
    return loss, np.concatenate(grads)


def fcg(dims, fat, lng, m, b, chans=None, w=None, tol=1e-10, maxiter=100000, phased=False):
    """Flexible CG with the network preconditioner (chans/w) or the identity (chans None)."""
    d, F, W, bb = _dims(dims), _c(fat), _c(lng), _c(b)
    x = np.zeros_like(bb)
    st = np.zeros(3)
    if chans is None:
        nl, ch, ww = 0, np.zeros(1, dtype=np.int32), np.zeros(1, dtype=np.complex128)
    else:
        nl, ch, ww = len(chans) - 1, np.ascontiguousarray(chans, dtype=np.int32), _c(w)
    lib().ho_fcg(_ptr(d), _ptr(F), _ptr(W), int(phased), float(m), nl, _ptr(ch), _ptr(ww), _ptr(bb),
                 _ptr(x), float(tol), int(maxiter), _ptr(st))
    return x, int(st[0]), float(st[1]), float(st[2])


def fcg_dense(dims, fat, lng, m, K, b, tol=1e-10, maxiter=1000, phased=False):
    d, F, W, bb, KK = _dims(dims), _c(fat), _c(lng), _c(b), _c(K)
    x = np.zeros_like(bb)
    st = np.zeros(3)
    lib().ho_fcg_dense(_ptr(d), _ptr(F), _ptr(W), int(phased), float(m), _ptr(KK), _ptr(bb), _ptr(x),
                       float(tol), int(maxiter), _ptr(st))
    return x, int(st[0]), float(st[1]), float(st[2])


def dense_D(dims, fat, lng, out_parity, phased=False):
    """Dense matrix of D_{p,1-p}: [3Vh][3Vh] complex, built column by column."""
    Vh = _vol(dims) // 2
    n = 3 * Vh
    cols = np.eye(n, dtype=np.complex128).reshape(n, Vh, 3)
    out = dslash(dims, fat, lng, cols, out_parity, phased)
    return out.reshape(n, n).T.copy()


def dense_A(dims, fat, lng, m, phased=False):
    """Dense A = 4 m^2 - D_eo D_oe on even sites: [3Vh][3Vh]."""
    Vh = _vol(dims) // 2
    n = 3 * Vh
    cols = np.eye(n, dtype=np.complex128).reshape(n, Vh, 3)
    out = mdagm(dims, fat, lng, m, cols, phased)
    return out.reshape(n, n).T.copy()

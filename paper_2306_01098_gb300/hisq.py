"""ctypes binding of libhisq.so: the C ABI of include/hisq.h, argument marshalling only.

Vectors and links are torch tensors (complex128, contiguous) whose device pointers are
passed straight to the library; every step of the computation runs in the library's CUDA
kernels.  There is no CPU fallback: importing works without a GPU, but every call needs
the built library and a CUDA device, and raises otherwise.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.path.join(HERE, "libhisq.so")

F64, F64X, F32, F16, BF16 = 0, 1, 2, 3, 4
PREC_NAMES = {F64: "f64", F64X: "f64x", F32: "f32", F16: "f16", BF16: "bf16"}
NPREC = 5

OK, EINVAL, ENOMEM, ECUDA, ENOTCONVERGED, ETIMEOUT, EDEVICE, ENOTBUILT = range(8)

_lib = None


class HisqError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"hisq error {code}: {msg}")
        self.code = code


class Opts(ctypes.Structure):
    _fields_ = [("links_on_device", ctypes.c_int), ("links_phased", ctypes.c_int),
                ("prec_mask", ctypes.c_uint), ("compression", ctypes.c_int * NPREC),
                ("device", ctypes.c_int), ("autotune", ctypes.c_int)]


class SolveOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("maxiter", ctypes.c_int), ("prec_sloppy", ctypes.c_int),
                ("prec_precise", ctypes.c_int), ("reliable_interval", ctypes.c_int),
                ("reliable_delta", ctypes.c_double), ("zero_guess", ctypes.c_int),
                ("host_buffers", ctypes.c_int), ("check_interval", ctypes.c_int),
                ("use_graph", ctypes.c_int), ("profile", ctypes.c_int), ("l2_persist", ctypes.c_int),
                ("stream", ctypes.c_void_p), ("single_reduction", ctypes.c_int), ("persistent", ctypes.c_int),
                ("selftest_wait", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("reliable_updates", ctypes.c_int),
                ("true_residual", ctypes.c_double), ("iterated_residual", ctypes.c_double),
                ("seconds", ctypes.c_double), ("dslash_calls", ctypes.c_long),
                ("dslash_ms", ctypes.c_double), ("dslash_timed", ctypes.c_long),
                ("bytes_moved", ctypes.c_double), ("kernels", ctypes.c_long), ("phase_ms", ctypes.c_double),
                ("phase_iterations", ctypes.c_long), ("phase_launches", ctypes.c_long),
                ("persistent_ds", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class NetOpts(ctypes.Structure):
    _fields_ = [("nlayer", ctypes.c_int), ("channels", ctypes.c_int), ("link_prec", ctypes.c_int),
                ("epochs", ctypes.c_int), ("batch", ctypes.c_int), ("lr", ctypes.c_double),
                ("beta1", ctypes.c_double), ("beta2", ctypes.c_double), ("eps", ctypes.c_double),
                ("init_hop", ctypes.c_double), ("seed", ctypes.c_ulonglong), ("loss", ctypes.c_int),
                ("mass", ctypes.c_double), ("tensor_cores", ctypes.c_int), ("selftest_wait", ctypes.c_int)]


class Peaks(ctypes.Structure):
    _fields_ = [("fp32_tflops", ctypes.c_double), ("fp64_tflops", ctypes.c_double),
                ("l2_read_gbs", ctypes.c_double), ("hbm_read_gbs", ctypes.c_double),
                ("launch_us", ctypes.c_double), ("grid_barrier_us", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_P, _I, _D, _L = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_long

_SIGS = {
    "hisq_opts_default": (None, [ctypes.POINTER(Opts)]),
    "hisq_create": (_I, [ctypes.POINTER(_P), ctypes.POINTER(_I), _P, _P, ctypes.POINTER(Opts)]),
    "hisq_destroy": (None, [_P]),
    "hisq_get_last_error": (_I, [_P]),
    "hisq_last_error_message": (ctypes.c_char_p, [_P]),
    "hisq_strerror": (ctypes.c_char_p, [_I]),
    "hisq_half_volume": (_L, [_P]),
    "hisq_field_create": (_I, [_P, _I, _I, ctypes.POINTER(_P)]),
    "hisq_field_destroy": (None, [_P]),
    "hisq_field_import": (_I, [_P, _P, _P]),
    "hisq_field_export": (_I, [_P, _P, _P]),
    "hisq_field_bytes": (ctypes.c_size_t, [_P]),
    "hisq_dslash": (_I, [_P, _I, _P, _P, _I, _I, _P]),
    "hisq_condensate": (_I, [_P, _D, _I, _P, ctypes.POINTER(SolveOpts), _P, ctypes.POINTER(_D),
                             ctypes.POINTER(Stats)]),
    "hisq_meson_correlators": (_I, [_P, _D, ctypes.POINTER(_I), _I, ctypes.POINTER(SolveOpts), _P, _P,
                                    ctypes.POINTER(Stats)]),
    "hisq_smear_links": (_I, [ctypes.POINTER(_I), _P, _P, _P, _D, _I, _P]),
    "hisq_rational_apply": (_I, [_P, _D, _I, ctypes.POINTER(_D), ctypes.POINTER(_D), _D, _P, _P,
                                 ctypes.POINTER(SolveOpts), ctypes.POINTER(Stats), _P]),
    "hisq_dslash_field": (_I, [_P, _I, _P, _P, _P]),
    "hisq_mdagm": (_I, [_P, _D, _P, _P, _I, _I, _P]),
    "hisq_mdagm_noalloc": (_I, [_P, _D, _P, _P, _I, _P]),
    "hisq_tune_set": (_I, [_P, _I, _I, _I, _I, _I, _I]),
    "hisq_tune_set_block": (_I, [_P, _I, _I, _I, _I]),
    "hisq_tune_set_groups": (_I, [_P, _I, _I, _I, _I]),
    "hisq_tune_get": (_I, [_P, _I, _I, _I, ctypes.POINTER(_I)]),
    "hisq_tune_set_block_groups": (_I, [_P, _I, _I, _I, _I]),
    "hisq_tune_get_block_groups": (_I, [_P, _I, _I, _I, ctypes.POINTER(_I)]),
    "hisq_solve_opts_default": (None, [ctypes.POINTER(SolveOpts)]),
    "hisq_cg": (_I, [_P, _D, _P, _P, _I, ctypes.POINTER(SolveOpts), ctypes.POINTER(Stats), _P]),
    "hisq_multishift_cg": (_I, [_P, _D, _I, _P, _P, _P, _P, ctypes.POINTER(SolveOpts), ctypes.POINTER(Stats), _P]),
    "hisq_batch_create": (_I, [ctypes.POINTER(_P), _I, _P]),
    "hisq_batch_destroy": (None, [_P]),
    "hisq_batch_sites": (_L, [_P]),
    "hisq_batch_last_error_message": (ctypes.c_char_p, [_P]),
    "hisq_batch_dslash": (_I, [_P, _I, _P, _P, _I, _P]),
    "hisq_batch_cg": (_I, [_P, _P, _P, _P, ctypes.POINTER(SolveOpts), ctypes.POINTER(Stats), _P]),
    "hisq_net_opts_default": (None, [ctypes.POINTER(NetOpts)]),
    "hisq_net_create": (_I, [_P, ctypes.POINTER(NetOpts), ctypes.POINTER(_P)]),
    "hisq_net_destroy": (None, [_P]),
    "hisq_net_num_weights": (_L, [_P]),
    "hisq_net_get_weights": (_I, [_P, _P]),
    "hisq_net_set_weights": (_I, [_P, _P]),
    "hisq_net_apply": (_I, [_P, _P, _P, _P]),
    "hisq_net_loss_grad": (_I, [_P, _P, _P, ctypes.POINTER(_D), _P]),
    "hisq_net_train": (_I, [_P, _I, _P, _P, _P]),
    "hisq_precond_train": (_I, [_P, ctypes.POINTER(NetOpts), _I, _P, _P, ctypes.POINTER(_P)]),
    "hisq_net_save": (_I, [_P, ctypes.c_char_p]),
    "hisq_net_load": (_I, [_P, ctypes.c_char_p, ctypes.POINTER(_P)]),
    "hisq_fcg": (_I, [_P, _D, _P, _P, _P, ctypes.POINTER(SolveOpts), ctypes.POINTER(Stats)]),
    "hisq_dd_create": (_I, [ctypes.POINTER(_P), ctypes.POINTER(_I), _I, _I, _P, _P, ctypes.POINTER(Opts)]),
    "hisq_dd_destroy": (None, [_P]),
    "hisq_dd_last_error_message": (ctypes.c_char_p, [_P]),
    "hisq_dd_half_volume": (_L, [_P]),
    "hisq_dd_halo_sites": (_L, [_P]),
    "hisq_dd_pack": (_I, [_P, _P, _P, _P, _P]),
    "hisq_dd_dslash": (_I, [_P, _I, _P, _P, _P, _P, _P]),
    "hisq_measure_peaks": (_I, [_I, ctypes.POINTER(Peaks)]),
}


def measure_peaks(device=0):
    """Measured FMA throughput, L2/HBM read bandwidth, launch and grid-barrier times
    (hisq_measure_peaks) as a dict."""
    p = Peaks()
    rc = lib().hisq_measure_peaks(int(device), ctypes.byref(p))
    if rc != OK:
        raise HisqError(rc, lib().hisq_strerror(rc).decode())
    return p.as_dict()


def exported_symbols():
    return sorted(_SIGS)


def lib():
    """Load libhisq.so (built in-tree by build()); raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIBPATH):
            raise RuntimeError(f"{LIBPATH} is not built; run __graft_entry__.build()")
        L = ctypes.CDLL(LIBPATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ptr(t):
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        if not t.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(t.data_ptr())
    return ctypes.c_void_p(t)


def _stream(stream):
    if stream is None:
        return None
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


class Context:
    """One lattice with its links prepared on the device (hisq_create)."""

    def __init__(self, dims, fat, lng, precs=(F64, F64X, F32, F16), compression=None, phased=False, device=0,
                 autotune=True):
        L = lib()
        o = Opts()
        L.hisq_opts_default(ctypes.byref(o))
        o.links_on_device = int(fat.is_cuda)
        o.links_phased = int(phased)
        o.prec_mask = sum(1 << p for p in precs)
        o.device = device
        o.autotune = int(autotune)
        for p, c in (compression or {}).items():
            o.compression[p] = c
        d = (ctypes.c_int * 4)(*dims)
        h = ctypes.c_void_p()
        rc = L.hisq_create(ctypes.byref(h), d, _ptr(fat), _ptr(lng), ctypes.byref(o))
        if rc != OK:
            raise HisqError(rc, L.hisq_strerror(rc).decode())
        self.h = h
        self.dims = tuple(dims)
        self.device = int(device)
        self.Vh = L.hisq_half_volume(h)

    def close(self):
        if getattr(self, "h", None):
            lib().hisq_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self, rc):
        if rc not in (OK, ENOTCONVERGED):
            raise HisqError(rc, lib().hisq_last_error_message(self.h).decode())
        return rc

    # ------------------------------------------------------------------ operators
    def _nrhs(self, inp, out):
        """Right-hand sides of an (in, out) pair of canonical [nrhs][Vh][3] complex128 vectors.
        The C side receives only pointers, so sizes, dtypes and devices are checked here."""
        import torch
        for name, t in (("in", inp), ("out", out)):
            if t.dtype != torch.complex128:
                raise ValueError(f"{name}: complex128 expected, got {t.dtype}")
            if not t.is_cuda or t.device.index != self.device:
                raise ValueError(f"{name}: must live on cuda:{self.device}, the context's device")
        n = self.Vh * 3
        if inp.numel() == 0 or inp.numel() % n:
            raise ValueError(f"in: {inp.numel()} elements is not a whole number of [Vh={self.Vh}][3] vectors")
        if out.numel() != inp.numel():
            raise ValueError(f"out has {out.numel()} elements, in has {inp.numel()}")
        return inp.numel() // n

    def dslash(self, out_parity, inp, out, prec=F64, stream=None):
        nrhs = self._nrhs(inp, out)
        return self.check(lib().hisq_dslash(self.h, out_parity, _ptr(inp), _ptr(out), nrhs, prec, _stream(stream)))

    def mdagm(self, m, inp, out, prec=F64, stream=None):
        nrhs = self._nrhs(inp, out)
        return self.check(lib().hisq_mdagm(self.h, float(m), _ptr(inp), _ptr(out), nrhs, prec, _stream(stream)))

    def mdagm_noalloc(self, m, inp, out, stream=None):
        """FP64 normal operator without device allocation (fixed scratch array)."""
        nrhs = self._nrhs(inp, out)
        return self.check(lib().hisq_mdagm_noalloc(self.h, float(m), _ptr(inp), _ptr(out), nrhs, _stream(stream)))

    def tune_set(self, prec_links, prec_vectors, nrhs, n_inner, threads_per_site, site_order=-1):
        return self.check(lib().hisq_tune_set(self.h, prec_links, prec_vectors, nrhs, n_inner, threads_per_site,
                                              site_order))

    def tune_set_block(self, prec_links, prec_vectors, nrhs, threads_per_block):
        return self.check(lib().hisq_tune_set_block(self.h, prec_links, prec_vectors, nrhs, threads_per_block))

    def tune_set_groups(self, prec_links, prec_vectors, nrhs, rhs_groups):
        return self.check(lib().hisq_tune_set_groups(self.h, prec_links, prec_vectors, nrhs, rhs_groups))

    def tune_set_block_groups(self, prec_links, prec_vectors, nrhs, block_groups):
        return self.check(lib().hisq_tune_set_block_groups(self.h, prec_links, prec_vectors, nrhs, block_groups))

    def tune_get_block_groups(self, prec_links, prec_vectors, nrhs):
        """Groups of right-hand sides per block stored for the key, or None."""
        g = ctypes.c_int(0)
        rc = lib().hisq_tune_get_block_groups(self.h, prec_links, prec_vectors, nrhs, ctypes.byref(g))
        return g.value if rc == OK else None

    def tune_get(self, prec_links, prec_vectors, nrhs):
        """(n_inner, threads_per_site, site_order, threads_per_block, rhs_groups) stored for the
        key, or None."""
        sh = (ctypes.c_int * 5)()
        rc = lib().hisq_tune_get(self.h, prec_links, prec_vectors, nrhs, sh)
        return tuple(sh) if rc == OK else None

    def field(self, prec, nrhs=1):
        return Field(self, prec, nrhs)

    def dslash_field(self, out_parity, fin, fout, stream=None):
        return self.check(lib().hisq_dslash_field(self.h, out_parity, fin.h, fout.h, _stream(stream)))

    # ------------------------------------------------------------------ solvers
    @staticmethod
    def solve_opts(**kw):
        o = SolveOpts()
        lib().hisq_solve_opts_default(ctypes.byref(o))
        for k, v in kw.items():
            if k == "stream":
                v = _stream(v)
            setattr(o, k, v)
        return o

    def cg(self, m, b, x, opts=None, residuals=None, **kw):
        o = opts or self.solve_opts(**kw)
        st = Stats()
        nrhs = b.numel() // (self.Vh * 3)
        rc = self.check(lib().hisq_cg(self.h, float(m), _ptr(b), _ptr(x), nrhs, ctypes.byref(o), ctypes.byref(st),
                                      _ptr(residuals)))
        return rc, st

    def multishift_cg(self, m, sigma, b, xs, tol=None, opts=None, residuals=None, **kw):
        o = opts or self.solve_opts(**kw)
        st = Stats()
        n = len(sigma)
        sig = (ctypes.c_double * n)(*sigma)
        xp = (ctypes.c_void_p * n)(*[x.data_ptr() for x in xs])
        tp = (ctypes.c_double * n)(*tol) if tol is not None else None
        rc = self.check(lib().hisq_multishift_cg(self.h, float(m), n, sig, _ptr(b), xp, tp, ctypes.byref(o),
                                                 ctypes.byref(st), _ptr(residuals)))
        return rc, st


    def condensate(self, m, eta, opts=None, **kw):
        """(pbp, samples, rc, stats): (1/V) Tr M^-1 estimated from noise vectors (hisq_condensate)."""
        import numpy as np
        o = opts or self.solve_opts(**kw)
        st = Stats()
        n = eta.numel() // (self.Vh * 3)
        samples = np.zeros(n)
        pbp = ctypes.c_double()
        rc = self.check(lib().hisq_condensate(self.h, float(m), n, _ptr(eta), ctypes.byref(o),
                                              samples.ctypes.data_as(ctypes.c_void_p), ctypes.byref(pbp),
                                              ctypes.byref(st)))
        return pbp.value, samples, rc, st

    def meson_correlators(self, m, src, direction, prop=None, opts=None, **kw):
        """(corr [8][N_d], rc, stats): point-source staggered meson correlators along
        `direction` (hisq_meson_correlators); `prop` (device [3][V][3] complex128) receives G."""
        import numpy as np
        o = opts or self.solve_opts(**kw)
        st = Stats()
        corr = np.zeros((8, self.dims[direction]))
        s = (ctypes.c_int * 4)(*[int(v) for v in src])
        rc = self.check(lib().hisq_meson_correlators(self.h, float(m), s, int(direction), ctypes.byref(o),
                                                     corr.ctypes.data_as(ctypes.c_void_p), _ptr(prop),
                                                     ctypes.byref(st)))
        return corr, rc, st

    def rational_apply(self, m, alpha0, alpha, sigma, b, x, opts=None, residuals=None, **kw):
        """x = alpha0 b + sum_s alpha_s (A + sigma_s)^-1 b (hisq_rational_apply)."""
        o = opts or self.solve_opts(**kw)
        st = Stats()
        n = len(sigma)
        al = (ctypes.c_double * n)(*[float(v) for v in alpha])
        sg = (ctypes.c_double * n)(*[float(v) for v in sigma])
        rc = self.check(lib().hisq_rational_apply(self.h, float(m), n, al, sg, float(alpha0), _ptr(b), _ptr(x),
                                                  ctypes.byref(o), ctypes.byref(st), _ptr(residuals)))
        return rc, st


def smear_links(dims, thin, eps_naik=0.0, stream=None):
    """(fat, long) HISQ links from thin links (hisq_smear_links); tensors on thin's device."""
    import torch
    fat = torch.empty_like(thin)
    lng = torch.empty_like(thin)
    d = (ctypes.c_int * 4)(*[int(v) for v in dims])
    rc = lib().hisq_smear_links(d, _ptr(thin), _ptr(fat), _ptr(lng), float(eps_naik), int(thin.is_cuda),
                                _stream(stream))
    if rc != OK:
        raise HisqError(rc, lib().hisq_strerror(rc).decode())
    return fat, lng


class Batch:
    """Lattices of different sizes in single launches (hisq_batch_*).  Vectors are packed:
    lattice k's [Vh_k][3] complex sites follow those of lattices 0..k-1."""

    def __init__(self, ctxs):
        self.ctxs = list(ctxs)  # the batch borrows the contexts
        arr = (ctypes.c_void_p * len(self.ctxs))(*[c.h.value for c in self.ctxs])
        h = ctypes.c_void_p()
        rc = lib().hisq_batch_create(ctypes.byref(h), len(self.ctxs), arr)
        if rc != OK:
            raise HisqError(rc, lib().hisq_strerror(rc).decode())
        self.h = h
        self.sites = lib().hisq_batch_sites(h)
        self.offsets = []
        off = 0
        for c in self.ctxs:
            self.offsets.append(off)
            off += c.Vh

    def close(self):
        if getattr(self, "h", None):
            lib().hisq_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self, rc):
        if rc not in (OK, ENOTCONVERGED):
            raise HisqError(rc, lib().hisq_batch_last_error_message(self.h).decode())
        return rc

    def dslash(self, out_parity, inp, out, prec=F64, stream=None):
        return self.check(lib().hisq_batch_dslash(self.h, out_parity, _ptr(inp), _ptr(out), prec, _stream(stream)))

    def cg(self, masses, b, x, opts=None, residuals=None, **kw):
        o = opts or Context.solve_opts(**kw)
        st = Stats()
        m = (ctypes.c_double * len(self.ctxs))(*[float(v) for v in masses])
        rc = self.check(lib().hisq_batch_cg(self.h, m, _ptr(b), _ptr(x), ctypes.byref(o), ctypes.byref(st),
                                            _ptr(residuals)))
        return rc, st


class Net:
    """Learned preconditioner (hisq_net_*): gauge-covariant parallel-transport network."""

    def __init__(self, ctx: Context, handle=None, **opts):
        self.ctx = ctx
        if handle is not None:
            self.h = handle
        else:
            o = NetOpts()
            lib().hisq_net_opts_default(ctypes.byref(o))
            for k, v in opts.items():
                setattr(o, k, v)
            h = ctypes.c_void_p()
            ctx.check(lib().hisq_net_create(ctx.h, ctypes.byref(o), ctypes.byref(h)))
            self.h = h
        self.nw = lib().hisq_net_num_weights(self.h)

    @classmethod
    def trained(cls, ctx: Context, B, X, **opts):
        """A network created and trained on the (b, x) pairs in one call (hisq_precond_train)."""
        o = NetOpts()
        lib().hisq_net_opts_default(ctypes.byref(o))
        for k, v in opts.items():
            setattr(o, k, v)
        h = ctypes.c_void_p()
        ctx.check(lib().hisq_precond_train(ctx.h, ctypes.byref(o), B.shape[0], _ptr(B), _ptr(X), ctypes.byref(h)))
        return cls(ctx, handle=h)

    @classmethod
    def load(cls, ctx: Context, path: str):
        h = ctypes.c_void_p()
        ctx.check(lib().hisq_net_load(ctx.h, path.encode(), ctypes.byref(h)))
        return cls(ctx, handle=h)

    def save(self, path: str):
        self.ctx.check(lib().hisq_net_save(self.h, path.encode()))

    def get_weights(self):
        import numpy as np
        w = np.zeros(2 * self.nw)
        self.ctx.check(lib().hisq_net_get_weights(self.h, w.ctypes.data_as(ctypes.c_void_p)))
        return w[0::2] + 1j * w[1::2]

    def set_weights(self, w):
        import numpy as np
        w = np.asarray(w, dtype=np.complex128).ravel()
        a = np.ascontiguousarray(np.stack([w.real, w.imag], axis=1).ravel())
        self.ctx.check(lib().hisq_net_set_weights(self.h, a.ctypes.data_as(ctypes.c_void_p)))

    def apply(self, b, z, stream=None):
        self.ctx.check(lib().hisq_net_apply(self.h, _ptr(b), _ptr(z), _stream(stream)))

    def loss_grad(self, b, x):
        import numpy as np
        loss = ctypes.c_double()
        g = np.zeros(2 * self.nw)
        self.ctx.check(lib().hisq_net_loss_grad(self.h, _ptr(b), _ptr(x), ctypes.byref(loss),
                                                 g.ctypes.data_as(ctypes.c_void_p)))
        return loss.value, g[0::2] + 1j * g[1::2]

    def train(self, B, X, epochs):
        import numpy as np
        losses = np.zeros(max(epochs, 1))
        npairs = B.shape[0]
        self.ctx.check(lib().hisq_net_train(self.h, npairs, _ptr(B), _ptr(X), losses.ctypes.data_as(ctypes.c_void_p)))
        return losses[:epochs]

    def close(self):
        if getattr(self, "h", None):
            lib().hisq_net_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fcg(ctx: Context, m, b, x, net=None, opts=None, **kw):
    """Flexible CG with the network preconditioner (hisq_fcg)."""
    o = opts or ctx.solve_opts(**kw)
    st = Stats()
    rc = ctx.check(lib().hisq_fcg(ctx.h, float(m), net.h if net is not None else None, _ptr(b), _ptr(x),
                                  ctypes.byref(o), ctypes.byref(st)))
    return rc, st


class Field:
    """Internal-layout vectors of one precision (hisq_field_*)."""

    def __init__(self, ctx: Context, prec: int, nrhs: int = 1):
        self.ctx = ctx
        h = ctypes.c_void_p()
        ctx.check(lib().hisq_field_create(ctx.h, prec, nrhs, ctypes.byref(h)))
        self.h, self.prec, self.nrhs = h, prec, nrhs

    def load(self, src, stream=None):
        self.ctx.check(lib().hisq_field_import(self.h, _ptr(src), _stream(stream)))

    def store(self, dst, stream=None):
        self.ctx.check(lib().hisq_field_export(self.h, _ptr(dst), _stream(stream)))

    def nbytes(self):
        return lib().hisq_field_bytes(self.h)

    def close(self):
        if getattr(self, "h", None):
            lib().hisq_field_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Domain:
    """One time slab [t0, t0 + lt) of a domain-decomposed lattice (hisq_dd_*): its Dslash
    takes the opposite-parity field on the slab plus the two received halos (three time
    slices each).  Links: the GLOBAL unphased canonical fields (host or device)."""

    def __init__(self, global_dims, t0, lt, fat, lng, device=0):
        L = lib()
        o = Opts()
        L.hisq_opts_default(ctypes.byref(o))
        o.links_on_device = int(fat.is_cuda)
        o.device = device
        d = (ctypes.c_int * 4)(*global_dims)
        h = ctypes.c_void_p()
        rc = L.hisq_dd_create(ctypes.byref(h), d, int(t0), int(lt), _ptr(fat), _ptr(lng), ctypes.byref(o))
        if rc != OK:
            raise HisqError(rc, L.hisq_strerror(rc).decode())
        self.h, self.t0, self.lt, self.device = h, int(t0), int(lt), int(device)
        self.global_dims = tuple(global_dims)
        self.Vh = L.hisq_dd_half_volume(h)
        self.halo = L.hisq_dd_halo_sites(h)

    def check(self, rc):
        if rc != OK:
            raise HisqError(rc, lib().hisq_dd_last_error_message(self.h).decode())
        return rc

    def _vec(self, t, n, name):
        import torch
        if t.dtype != torch.complex128 or not t.is_cuda or t.device.index != self.device or t.numel() != 3 * n:
            raise ValueError(f"{name}: complex128 [{n}][3] on cuda:{self.device} expected")

    def halo_buffers(self):
        """(send_lo, send_hi, recv_lo, recv_hi) device buffers of [3 F][3] complex128."""
        import torch
        return tuple(torch.empty(self.halo, 3, dtype=torch.complex128, device=f"cuda:{self.device}") for _ in range(4))

    def pack(self, inp, send_lo, send_hi, stream=None):
        """The three lowest and three highest time slices of `inp` (one parity)."""
        self._vec(inp, self.Vh, "in")
        self._vec(send_lo, self.halo, "send_lo")
        self._vec(send_hi, self.halo, "send_hi")
        return self.check(lib().hisq_dd_pack(self.h, _ptr(inp), _ptr(send_lo), _ptr(send_hi), _stream(stream)))

    def dslash(self, out_parity, inp, recv_lo, recv_hi, out, stream=None):
        self._vec(inp, self.Vh, "in")
        self._vec(out, self.Vh, "out")
        self._vec(recv_lo, self.halo, "recv_lo")
        self._vec(recv_hi, self.halo, "recv_hi")
        return self.check(lib().hisq_dd_dslash(self.h, int(out_parity), _ptr(inp), _ptr(recv_lo), _ptr(recv_hi),
                                               _ptr(out), _stream(stream)))

    def close(self):
        if getattr(self, "h", None):
            lib().hisq_dd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

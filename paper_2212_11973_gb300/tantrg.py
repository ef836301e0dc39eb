"""ctypes binding of libtantrg.so (include/tantrg.h): argument marshalling only.

Every name mirrors the C ABI.  All numerical work happens inside the library's
CUDA kernels; this module never computes anything itself and raises if the
library is missing (there is no CPU fallback).  PyTorch supplies the CUDA
stream and, optionally, its caching allocator for device memory.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libtantrg.so")

TT_OK = 0
STATUS = {0: "TT_OK", 1: "TT_ERR_INVALID_ARG", 2: "TT_ERR_OOM", 3: "TT_ERR_CUDA",
          4: "TT_ERR_NUMERIC", 5: "TT_ERR_TIMEOUT", 6: "TT_ERR_STATE"}
TT_PREC_FP64 = 0
TT_PREC_MIXED_BF16X3 = 1
TT_PREC_MIXED_BF16X6 = 2


class TTError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)


class tt_alloc_cb(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", C.c_void_p)]


class tt_model(C.Structure):
    _fields_ = [("Lx", C.c_int), ("Wy", C.c_int), ("bc_y_periodic", C.c_int),
                ("t", C.c_double), ("tp", C.c_double), ("U", C.c_double), ("mu", C.c_double),
                ("interaction_form", C.c_int)]


class tt_run_opts(C.Structure):
    _fields_ = [("D_max", C.c_int), ("krylov_dim", C.c_int), ("precision", C.c_int),
                ("growth_precision", C.c_int), ("svd_cut", C.c_double), ("degen_tol", C.c_double),
                ("env_precision", C.c_int)]


class tt_obs(C.Structure):
    _fields_ = [("beta", C.c_double), ("energy_per_site", C.c_double), ("density", C.c_double),
                ("double_occ", C.c_double), ("free_energy_per_site", C.c_double), ("lnZ", C.c_double),
                ("max_bond", C.c_int), ("krylov_resid_max", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class tt_stats(C.Structure):
    _fields_ = [("heff_flops", C.c_double), ("heff_ms", C.c_double), ("heff_launches", C.c_longlong),
                ("env_flops", C.c_double), ("env_ms", C.c_double), ("bond_ms", C.c_double),
                ("gather_ms", C.c_double), ("gather_launches", C.c_longlong),
                ("step_flops", C.c_double), ("step_ms", C.c_double), ("launches", C.c_longlong),
                ("n_sites", C.c_int), ("max_bond", C.c_int), ("n_sectors_max", C.c_int),
                ("qr_ms", C.c_double), ("bond_flops", C.c_double), ("qr_sectors", C.c_longlong), ("qr_fallbacks", C.c_longlong),
                ("site_exp_ms", C.c_double), ("bond_exp_ms", C.c_double), ("env_update_ms", C.c_double),
                ("absorb_ms", C.c_double), ("gauge_ms", C.c_double),
                ("tuned_tc128", C.c_longlong), ("tuned_tcp128x64", C.c_longlong), ("tuned_mma64", C.c_longlong),
                ("qr_gemm_ms", C.c_double), ("qr_gemm_flops", C.c_double), ("qr_chol_ms", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_P = C.c_void_p
_PI = C.POINTER(C.c_int)
_PD = C.POINTER(C.c_double)
_PL = C.POINTER(C.c_int64)

SIGNATURES = {
    "tt_ctx_create": (C.c_int, [C.POINTER(tt_alloc_cb), _P, C.POINTER(_P)]),
    "tt_ctx_destroy": (None, [_P]),
    "tt_last_error": (C.c_char_p, [_P]),
    "tt_ctx_set_wait_limit": (C.c_int, [_P, C.c_double]),
    "tt_hubbard_mpo_create": (C.c_int, [_P, C.POINTER(tt_model), C.POINTER(_P)]),
    "tt_mpo_destroy": (None, [_P]),
    "tt_mpo_num_sites": (C.c_int, [_P]),
    "tt_mpo_bond_dim": (C.c_int, [_P, C.c_int]),
    "tt_mpo_channel_charge": (C.c_int, [_P, C.c_int, C.c_int, _PI, _PI]),
    "tt_rho_create": (C.c_int, [_P, _P, C.c_double, C.c_int, C.POINTER(tt_run_opts), C.POINTER(_P)]),
    "tt_rho_destroy": (None, [_P]),
    "tt_rho_grow": (C.c_int, [_P, _P, C.c_double, C.c_double, _PD]),
    "tt_rho_grow_exp": (C.c_int, [_P, _P, C.c_double, C.c_double, _PD]),
    "tt_tdvp_step": (C.c_int, [_P, _P, C.c_double, C.c_int]),
    "tt_rho_pad": (C.c_int, [_P, _P, C.c_int]),
    "tt_measure": (C.c_int, [_P, _P, C.POINTER(tt_obs)]),
    "tt_stats_get": (C.c_int, [_P, C.POINTER(tt_stats)]),
    "tt_rho_set_profiling": (C.c_int, [_P, C.c_int]),
    "tt_rho_bond_dims": (C.c_int, [_P, _PI, C.c_int]),
    "tt_rho_bond_sectors": (C.c_int, [_P, C.c_int, _PI, _PI, _PI, C.c_int, _PI]),
    "tt_rho_save": (C.c_int, [_P, C.c_char_p]),
    "tt_rho_load": (C.c_int, [_P, _P, C.c_char_p, C.POINTER(tt_run_opts), C.POINTER(_P)]),
    "tt_layout_sizes": (C.c_int, [_P, C.c_int, _PI, _PI, _PI, _PI, _PL, _PL, _PL]),
    "tt_heff_apply_host": (C.c_int, [_P, _P, C.c_int, C.c_int, _PI, _PI, _PI, _PI, _PD, _PD, _PD, _PD]),
    "tt_heff_apply_terms_host": (C.c_int, [_P, C.c_int, _PI, _PI, C.c_int, _PI, _PI, C.c_int, _PI, _PI, _PI, _PI,
                                           _PD, C.c_int, _PI, _PI, _PI, _PI, _PD, _PD, _PD, _PD]),
    "tt_layout_sizes_terms": (C.c_int, [C.c_int, _PI, _PI, C.c_int, _PI, _PI, _PI, _PI, _PI, _PI, _PL, _PL, _PL]),
    "tt_qr_device": (C.c_int, [_P, _P, C.c_int, C.c_int, _P, _P]),
    "tt_qr_device_noalloc": (C.c_int, [_P, C.c_int, C.c_int, _P, _P, _P]),
    "tt_batch_create": (C.c_int, [_P, C.c_int, C.POINTER(tt_model), _PI, C.c_double, C.POINTER(tt_run_opts),
                                  C.POINTER(_P)]),
    "tt_batch_destroy": (None, [_P]),
    "tt_batch_size": (C.c_int, [_P]),
    "tt_batch_grow": (C.c_int, [_P, C.c_double, C.c_double]),
    "tt_batch_pad": (C.c_int, [_P]),
    "tt_batch_step": (C.c_int, [_P, C.c_double, C.c_int]),
    "tt_batch_measure": (C.c_int, [_P, C.POINTER(tt_obs)]),
    "tt_batch_stats": (C.c_int, [_P, C.c_int, C.POINTER(tt_stats)]),
    "tt_batch_set_profiling": (C.c_int, [_P, C.c_int]),
}

_lib = None


def load_library(path: str = LIB_PATH):
    """Load libtantrg.so and declare the C signatures; raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libtantrg.so not found at {path}: run __graft_entry__.build() first "
                           "(the CUDA library is required; there is no fallback)")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(ctx, status):
    if status != TT_OK:
        msg = load_library().tt_last_error(ctx).decode() if ctx else ""
        raise TTError(status, msg)


class Context:
    """tt_ctx on the current torch CUDA stream; device memory from torch's caching
    allocator unless use_torch_allocator=False (then cudaMallocAsync)."""

    def __init__(self, stream=None, use_torch_allocator: bool = True):
        import torch
        lib = load_library()
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        handle = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        self._cb = None
        cbp = None
        if use_torch_allocator:
            dev = torch.cuda.current_device()

            def _alloc(nbytes, strm, user):
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), dev, int(strm or 0))
                except Exception:
                    return None

            def _free(ptr, nbytes, strm, user):
                torch.cuda.caching_allocator_delete(int(ptr))

            self._cb = tt_alloc_cb(ALLOC_FN(_alloc), FREE_FN(_free), None)
            cbp = C.byref(self._cb)
        h = C.c_void_p()
        st = lib.tt_ctx_create(cbp, C.c_void_p(handle), C.byref(h))
        if st != TT_OK:
            raise TTError(st, "tt_ctx_create failed")
        self.h = h

    def set_wait_limit(self, seconds: float):
        _check(self.h, load_library().tt_ctx_set_wait_limit(self.h, float(seconds)))

    def close(self):
        if getattr(self, "h", None):
            load_library().tt_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Mpo:
    def __init__(self, ctx: Context, Lx, Wy, periodic, t=1.0, U=0.0, mu=0.0, form=1, tp=0.0):
        lib = load_library()
        self.ctx = ctx
        self.model = tt_model(Lx, Wy, int(periodic), t, tp, U, mu, form)
        h = C.c_void_p()
        _check(ctx.h, lib.tt_hubbard_mpo_create(ctx.h, C.byref(self.model), C.byref(h)))
        self.h = h
        self.N = lib.tt_mpo_num_sites(h)

    def bond_dim(self, k):
        return load_library().tt_mpo_bond_dim(self.h, k)

    def channel_charges(self, k):
        lib = load_library()
        out = []
        for w in range(self.bond_dim(k)):
            a, b = C.c_int(), C.c_int()
            _check(self.ctx.h, lib.tt_mpo_channel_charge(self.h, k, w, C.byref(a), C.byref(b)))
            out.append((a.value, b.value))
        return out

    def close(self):
        if getattr(self, "h", None):
            load_library().tt_mpo_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def run_opts(D_max, krylov_dim=8, precision=TT_PREC_FP64, growth_precision=-1, svd_cut=1e-12, degen_tol=1e-10,
             env_precision=0):
    return tt_run_opts(D_max, krylov_dim, precision, growth_precision, svd_cut, degen_tol, env_precision)


class Rho:
    def __init__(self, ctx: Context, mpo: Mpo, beta0: float, opts: tt_run_opts, handle=None, taylor_order: int = 1):
        lib = load_library()
        self.ctx, self.mpo, self.opts = ctx, mpo, opts
        if handle is None:
            h = C.c_void_p()
            _check(ctx.h, lib.tt_rho_create(ctx.h, mpo.h, beta0, taylor_order, C.byref(opts), C.byref(h)))
            handle = h
        self.h = handle

    @classmethod
    def load(cls, ctx, mpo, path, opts):
        h = C.c_void_p()
        _check(ctx.h, load_library().tt_rho_load(ctx.h, mpo.h, path.encode(), C.byref(opts), C.byref(h)))
        return cls(ctx, mpo, 0.0, opts, handle=h)

    def grow(self, dtau, beta_max):
        b = C.c_double()
        _check(self.ctx.h, load_library().tt_rho_grow(self.h, self.mpo.h, dtau, beta_max, C.byref(b)))
        return b.value

    def grow_exp(self, ratio, beta_max):
        b = C.c_double()
        _check(self.ctx.h, load_library().tt_rho_grow_exp(self.h, self.mpo.h, ratio, beta_max, C.byref(b)))
        return b.value

    def pad(self, D_target):
        _check(self.ctx.h, load_library().tt_rho_pad(self.h, self.mpo.h, D_target))

    def step(self, dtau, n_steps=1):
        _check(self.ctx.h, load_library().tt_tdvp_step(self.h, self.mpo.h, dtau, n_steps))

    def measure(self) -> dict:
        o = tt_obs()
        _check(self.ctx.h, load_library().tt_measure(self.h, self.mpo.h, C.byref(o)))
        return o.as_dict()

    def set_profiling(self, on: bool):
        _check(self.ctx.h, load_library().tt_rho_set_profiling(self.h, int(on)))

    def stats(self) -> dict:
        s = tt_stats()
        _check(self.ctx.h, load_library().tt_stats_get(self.h, C.byref(s)))
        return s.as_dict()

    def bond_dims(self):
        n = self.mpo.N + 1
        arr = (C.c_int * n)()
        _check(self.ctx.h, load_library().tt_rho_bond_dims(self.h, arr, n))
        return list(arr)

    def bond_sectors(self, k):
        """[(n, s, dim)] of bond k: particle number and n_up - n_dn charges."""
        lib = load_library()
        ns = C.c_int(0)
        lib.tt_rho_bond_sectors(self.h, k, None, None, None, 0, C.byref(ns))
        n = ns.value
        qn, qs, dd = (C.c_int * max(n, 1))(), (C.c_int * max(n, 1))(), (C.c_int * max(n, 1))()
        _check(self.ctx.h, lib.tt_rho_bond_sectors(self.h, k, qn, qs, dd, n, C.byref(ns)))
        return [(qn[i], qs[i], dd[i]) for i in range(n)]

    def save(self, path):
        _check(self.ctx.h, load_library().tt_rho_save(self.h, path.encode()))

    def close(self):
        if getattr(self, "h", None):
            load_library().tt_rho_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _int_array(v):
    return (C.c_int * len(v))(*v)


def layout_sizes(mpo: Mpo, site, sectors_l, sectors_r):
    """sectors_*: list of (n, 2Sz, dim) sorted by (n, 2Sz).  Returns (x, L, R) element counts."""
    secs = list(sectors_l) + list(sectors_r)
    nsec = _int_array([len(sectors_l), len(sectors_r)])
    qn = _int_array([s[0] for s in secs])
    qs = _int_array([s[1] for s in secs])
    qd = _int_array([s[2] for s in secs])
    a, b, c = C.c_int64(), C.c_int64(), C.c_int64()
    _check(mpo.ctx.h, load_library().tt_layout_sizes(mpo.h, site, nsec, qn, qs, qd, C.byref(a), C.byref(b), C.byref(c)))
    return a.value, b.value, c.value


def heff_apply_host(ctx: Context, mpo: Mpo, site, precision, sectors_l, sectors_r, L, R, x):
    """One H^(1) apply on host FP64 numpy arrays in the documented block layouts."""
    import numpy as np
    secs = list(sectors_l) + list(sectors_r)
    nsec = _int_array([len(sectors_l), len(sectors_r)])
    qn = _int_array([s[0] for s in secs])
    qs = _int_array([s[1] for s in secs])
    qd = _int_array([s[2] for s in secs])
    L = np.ascontiguousarray(L, dtype=np.float64)
    R = np.ascontiguousarray(R, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty_like(x)
    pd = lambda a: a.ctypes.data_as(_PD)  # noqa: E731
    _check(ctx.h, load_library().tt_heff_apply_host(ctx.h, mpo.h, site, precision, nsec, qn, qs, qd,
                                                     pd(L), pd(R), pd(x), pd(y)))
    return y


def _terms_args(chl, chr_, terms):
    import numpy as np
    t = list(terms)
    return (len(chl), _int_array([c[0] for c in chl]), _int_array([c[1] for c in chl]),
            len(chr_), _int_array([c[0] for c in chr_]), _int_array([c[1] for c in chr_]),
            len(t), _int_array([x[0] for x in t]), _int_array([x[1] for x in t]), _int_array([x[2] for x in t]),
            _int_array([x[3] for x in t]), np.ascontiguousarray([x[4] for x in t], dtype=np.float64))


def layout_sizes_terms(chl, chr_, sectors_l, sectors_r):
    """Element counts (x, L, R) for MPO channels chl / chr_ (lists of (n, 2Sz))."""
    secs = list(sectors_l) + list(sectors_r)
    nsec = _int_array([len(sectors_l), len(sectors_r)])
    qn = _int_array([s[0] for s in secs])
    qs = _int_array([s[1] for s in secs])
    qd = _int_array([s[2] for s in secs])
    a, b, c = C.c_int64(), C.c_int64(), C.c_int64()
    nl, cln, cls, nr, crn, crs = _terms_args(chl, chr_, [])[:6]
    st = load_library().tt_layout_sizes_terms(nl, cln, cls, nr, crn, crs, nsec, qn, qs, qd,
                                              C.byref(a), C.byref(b), C.byref(c))
    _check(None, st)
    return a.value, b.value, c.value


def heff_apply_terms_host(ctx: Context, chl, chr_, terms, precision, sectors_l, sectors_r, L, R, x):
    """One H^(1) apply with a caller-supplied MPO tensor: terms are
    (wl, wr, sig, tau, value) with <sig|op|tau>; chl / chr_ the channel charges."""
    import numpy as np
    secs = list(sectors_l) + list(sectors_r)
    nsec = _int_array([len(sectors_l), len(sectors_r)])
    qn = _int_array([s[0] for s in secs])
    qs = _int_array([s[1] for s in secs])
    qd = _int_array([s[2] for s in secs])
    nl, cln, cls, nr, crn, crs, nt, twl, twr, tsg, tta, tv = _terms_args(chl, chr_, terms)
    L = np.ascontiguousarray(L, dtype=np.float64)
    R = np.ascontiguousarray(R, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty_like(x)
    pd = lambda a: a.ctypes.data_as(_PD)  # noqa: E731
    _check(ctx.h, load_library().tt_heff_apply_terms_host(ctx.h, nl, cln, cls, nr, crn, crs, nt, twl, twr, tsg, tta,
                                                           pd(tv), precision, nsec, qn, qs, qd,
                                                           pd(L), pd(R), pd(x), pd(y)))
    return y


def qr_device(ctx: Context, A):
    """A = Q R on the device (FP64 Householder, diag(R) >= 0).  A: torch CUDA
    float64 tensor (m, n), m >= n.  Returns (Q, R) as torch tensors."""
    import torch
    m, n = A.shape
    At = A.t().contiguous()  # column-major m x n
    Q = torch.empty((n, m), dtype=torch.float64, device=A.device)
    R = torch.empty((n, n), dtype=torch.float64, device=A.device)
    _check(ctx.h, load_library().tt_qr_device(ctx.h, C.c_void_p(At.data_ptr()), m, n, C.c_void_p(Q.data_ptr()),
                                              C.c_void_p(R.data_ptr())))
    return Q.t(), R.t()


def qr_device_noalloc(A, Q, R, stream=None):
    """tt_qr_device_noalloc on caller-provided torch CUDA float64 buffers:
    A (n, m) holds the column-major m x n input, Q (n, m) and R (n, n) receive
    the column-major factors.  Allocates nothing; queued on `stream`."""
    import torch
    n, m = A.shape
    st = (stream or torch.cuda.current_stream()).cuda_stream
    status = load_library().tt_qr_device_noalloc(C.c_void_p(A.data_ptr()), m, n, C.c_void_p(Q.data_ptr()),
                                                 C.c_void_p(R.data_ptr()), C.c_void_p(st))
    if status != TT_OK:
        raise TTError(status, "tt_qr_device_noalloc failed (sizes beyond the fixed scratch, or a CUDA error)")


class Batch:
    """Independent instances stepped together (tt_batch_*): workloads is a list
    of objects with Lx, Wy, periodic, t, U, mu, form, D; opts gives the rest."""

    def __init__(self, ctx: Context, workloads, beta0: float, opts: tt_run_opts):
        lib = load_library()
        self.ctx = ctx
        n = len(workloads)
        self.n = n
        models = (tt_model * n)(*[tt_model(w.Lx, w.Wy, int(w.periodic), w.t, 0.0, w.U, w.mu, w.form)
                                  for w in workloads])
        dmax = (C.c_int * n)(*[w.D for w in workloads])
        h = C.c_void_p()
        _check(ctx.h, lib.tt_batch_create(ctx.h, n, models, dmax, beta0, C.byref(opts), C.byref(h)))
        self.h = h

    def grow(self, dtau, beta_max):
        _check(self.ctx.h, load_library().tt_batch_grow(self.h, dtau, beta_max))

    def pad(self):
        _check(self.ctx.h, load_library().tt_batch_pad(self.h))

    def step(self, dtau, n_steps=1):
        _check(self.ctx.h, load_library().tt_batch_step(self.h, dtau, n_steps))

    def measure(self):
        obs = (tt_obs * self.n)()
        _check(self.ctx.h, load_library().tt_batch_measure(self.h, obs))
        return [o.as_dict() for o in obs]

    def set_profiling(self, on: bool):
        _check(self.ctx.h, load_library().tt_batch_set_profiling(self.h, int(on)))

    def stats(self, i) -> dict:
        s = tt_stats()
        _check(self.ctx.h, load_library().tt_batch_stats(self.h, i, C.byref(s)))
        return s.as_dict()

    def close(self):
        if getattr(self, "h", None):
            load_library().tt_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

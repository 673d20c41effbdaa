"""Python binding of the C ABI in include/tddft.h (ctypes; argument marshalling only).

Every computation happens in the CUDA library.  Importing this module loads the
in-tree shared library and raises ImportError if it has not been built; there
is no fallback implementation.

Arrays may be numpy arrays (host) or torch CUDA tensors (device); a call uses
the device form of the C ABI when its inputs are CUDA tensors.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .build import LIBPATH

if not os.path.exists(LIBPATH):
    raise ImportError("CUDA library not built: %s (run paper_2404_17133_gb300.build.build())" % LIBPATH)

_lib = C.CDLL(LIBPATH)

OK, PENDING = 0, 1
ERR_ARG, ERR_OOM, ERR_CUDA, ERR_NOCONV, ERR_INDEFINITE, ERR_TIMEOUT, ERR_BUSY = -1, -2, -3, -4, -5, -6, -7
F64, F32 = 0, 1
DIAG, RID = 0, 1
PLAIN, MIXED = 0, 1
STATUS_NAMES = {0: "OK", 1: "PENDING", -1: "ERR_ARG", -2: "ERR_OOM", -3: "ERR_CUDA", -4: "ERR_NOCONV",
                -5: "ERR_INDEFINITE", -6: "ERR_TIMEOUT", -7: "ERR_BUSY"}


class Desc(C.Structure):
    _fields_ = [("n_occ", C.c_int), ("n_vir", C.c_int), ("n_aux", C.c_int),
                ("n_aux_ris_J", C.c_int), ("n_aux_ris_K", C.c_int),
                ("a_x", C.c_double), ("coulomb_factor", C.c_double), ("t_cut_ha", C.c_double),
                ("precisions", C.c_int), ("hbm_budget_gb", C.c_double)]


class Opts(C.Structure):
    _fields_ = [("precond", C.c_int), ("n_states", C.c_int), ("n_extra_guess", C.c_int),
                ("tol", C.c_double), ("inner_tol", C.c_double), ("guess_tol", C.c_double),
                ("max_iter", C.c_int), ("inner_max_iter", C.c_int), ("max_subspace", C.c_int),
                ("precision", C.c_int), ("tensor_cores", C.c_int), ("outputs_on_device", C.c_int),
                ("ris_fp8", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("n_iter", C.c_int), ("n_matvec", C.c_int), ("n_ris_matvec", C.c_int),
                ("converged", C.c_int), ("n_restart", C.c_int), ("gpu_launches", C.c_int),
                ("max_resid", C.c_double), ("max_resid_certified", C.c_double),
                ("t_total_s", C.c_double), ("t_matvec_s", C.c_double), ("t_precond_s", C.c_double),
                ("t_guess_s", C.c_double), ("t_certify_s", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Request(C.Structure):
    _fields_ = [("opts", Opts),
                ("omega", C.c_void_p), ("X", C.c_void_p), ("Y", C.c_void_p), ("resid", C.c_void_p),
                ("mu", C.c_void_p), ("n_dip", C.c_int), ("freqs", C.c_void_p), ("n_freq", C.c_int),
                ("alpha", C.c_void_p), ("stats", Stats)]


class ServeRequest(C.Structure):
    _fields_ = [("ctx", C.c_void_p), ("desc", Desc),
                ("eps_occ", C.c_void_p), ("eps_vir", C.c_void_p),
                ("L_oo", C.c_void_p), ("L_ov", C.c_void_p), ("L_vv", C.c_void_p),
                ("Lr_oo", C.c_void_p), ("Lr_ov", C.c_void_p), ("Lr_vv", C.c_void_p),
                ("ris_K_index", C.c_void_p), ("dtype", C.c_int), ("inputs_on_device", C.c_int),
                ("kind", C.c_int), ("req", Request), ("charged_bytes", C.c_ulonglong),
                ("t_submit_s", C.c_double), ("t_start_s", C.c_double), ("t_end_s", C.c_double),
                ("error", C.c_char * 256)]


class ServerState(C.Structure):
    _fields_ = [("budget_bytes", C.c_ulonglong), ("in_use_bytes", C.c_ulonglong),
                ("peak_in_use_bytes", C.c_ulonglong), ("active", C.c_int), ("max_active", C.c_int),
                ("queued", C.c_int), ("completed", C.c_ulonglong),
                ("pool_used_at_create_bytes", C.c_ulonglong), ("pool_high_bytes", C.c_ulonglong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class BatchInfo(C.Structure):
    _fields_ = [("n_variants", C.c_int), ("variant", C.c_int), ("autotune_ms", C.c_double * 8),
                ("outer_iterations", C.c_int), ("graph_nodes", C.c_int), ("launches", C.c_longlong),
                ("graph_launches", C.c_longlong), ("t_total_s", C.c_double)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "autotune_ms"}
        d["autotune_ms"] = [self.autotune_ms[i] for i in range(self.n_variants)]
        return d


_vp, _ip, _dp = C.c_void_p, C.c_int, C.c_void_p
_lib.tddft_default_opts.argtypes = [C.POINTER(Opts)]
_lib.tddft_default_opts.restype = None
_lib.tddft_default_desc.argtypes = [C.POINTER(Desc)]
_lib.tddft_default_desc.restype = None
_lib.tddft_create.argtypes = [C.POINTER(Desc), _dp, _dp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _ip, _ip,
                              _vp, C.POINTER(_vp)]
_lib.tddft_create.restype = C.c_int
_lib.tddft_solve_tda.argtypes = [_vp, C.POINTER(Opts), _dp, _dp, _dp, C.POINTER(Stats)]
_lib.tddft_solve_tda.restype = C.c_int
_lib.tddft_solve_rpa.argtypes = [_vp, C.POINTER(Opts), _dp, _dp, _dp, _dp, C.POINTER(Stats)]
_lib.tddft_solve_rpa.restype = C.c_int
_lib.tddft_solve_polar.argtypes = [_vp, C.POINTER(Opts), _dp, _ip, _dp, _ip, _dp, C.POINTER(Stats)]
_lib.tddft_solve_polar.restype = C.c_int
_lib.tddft_apply.argtypes = [_vp, _ip, _ip, _ip, _dp, _ip, _dp, _dp, _ip]
_lib.tddft_apply.restype = C.c_int
_lib.tddft_submit.argtypes = [_vp, _ip, C.POINTER(Request), C.POINTER(C.c_ulonglong)]
_lib.tddft_submit.restype = C.c_int
_lib.tddft_poll.argtypes = [_vp, C.c_ulonglong, _ip]
_lib.tddft_poll.restype = C.c_int
_lib.tddft_destroy.argtypes = [_vp]
_lib.tddft_destroy.restype = None
_lib.tddft_last_error.argtypes = [_vp]
_lib.tddft_last_error.restype = C.c_char_p
_lib.tddft_device_bytes.argtypes = [_vp]
_lib.tddft_device_bytes.restype = C.c_ulonglong
_lib.tddft_apply_noalloc.argtypes = [_vp, _ip, _ip, _dp, _ip, _dp, _dp]
_lib.tddft_apply_noalloc.restype = C.c_int
_lib.tddft_profile.argtypes = [_vp, _ip]
_lib.tddft_profile.restype = C.c_int
_lib.tddft_profile_read.argtypes = [_vp, _ip, C.POINTER(C.c_longlong), C.POINTER(C.c_double),
                                    C.POINTER(C.c_double)]
_lib.tddft_profile_read.restype = C.c_int
_lib.tddft_estimate_bytes.argtypes = [C.POINTER(Desc), _ip, C.POINTER(Opts), _ip, _ip,
                                      C.POINTER(C.c_ulonglong), C.POINTER(C.c_ulonglong)]
_lib.tddft_estimate_bytes.restype = C.c_int
_lib.tddft_server_create.argtypes = [C.c_double, _ip, C.POINTER(_vp)]
_lib.tddft_server_create.restype = C.c_int
_lib.tddft_server_submit.argtypes = [_vp, C.POINTER(ServeRequest), C.POINTER(C.c_ulonglong)]
_lib.tddft_server_submit.restype = C.c_int
_lib.tddft_server_poll.argtypes = [_vp, C.c_ulonglong, _ip]
_lib.tddft_server_poll.restype = C.c_int
_lib.tddft_server_info.argtypes = [_vp, C.POINTER(ServerState)]
_lib.tddft_server_info.restype = C.c_int
_lib.tddft_server_destroy.argtypes = [_vp]
_lib.tddft_server_destroy.restype = None
_lib.tddft_ctx_desc.argtypes = [_vp, C.POINTER(Desc)]
_lib.tddft_ctx_desc.restype = C.c_int
_lib.tddft_profile_records.argtypes = [_vp, _ip, _ip, _dp, _dp, _dp, C.POINTER(C.c_int)]
_lib.tddft_profile_records.restype = C.c_int
_lib.tddft_add_exchange.argtypes = [_vp, C.c_double, _ip, _vp, _vp, _vp, _ip, _ip]
_lib.tddft_add_exchange.restype = C.c_int
_lib.tddft_add_kernel.argtypes = [_vp, _ip, _dp, _vp, _ip, _ip]
_lib.tddft_add_kernel.restype = C.c_int
_lib.tddft_solve_tda_batch.argtypes = [C.POINTER(_vp), _ip, C.POINTER(Opts), _dp, _dp, C.POINTER(Stats),
                                       C.POINTER(BatchInfo)]
_lib.tddft_solve_tda_batch.restype = C.c_int
_lib.tddft_pool_usage.argtypes = [_ip, C.POINTER(C.c_ulonglong), C.POINTER(C.c_ulonglong), _ip]
_lib.tddft_pool_usage.restype = C.c_int

EXPORTED = ["tddft_default_opts", "tddft_default_desc", "tddft_create", "tddft_solve_tda",
            "tddft_solve_rpa", "tddft_solve_polar", "tddft_apply", "tddft_submit", "tddft_poll",
            "tddft_destroy", "tddft_last_error", "tddft_device_bytes", "tddft_profile",
            "tddft_profile_read", "tddft_apply_noalloc", "tddft_estimate_bytes", "tddft_server_create",
            "tddft_server_submit", "tddft_server_poll", "tddft_server_info", "tddft_server_destroy",
            "tddft_ctx_desc", "tddft_add_exchange", "tddft_add_kernel",
            "tddft_profile_records", "tddft_pool_usage", "tddft_solve_tda_batch"]


class TddftError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


def lib():
    return _lib


def _is_cuda(x):
    return hasattr(x, "is_cuda") and x.is_cuda


def _ptr(x, dtype=np.float64):
    """(pointer, keepalive) for a numpy array or torch tensor (None -> NULL)."""
    if x is None:
        return None, None
    if _is_cuda(x) or hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return C.c_void_p(x.data_ptr()), x
    a = np.ascontiguousarray(x, dtype=dtype)
    return a.ctypes.data_as(C.c_void_p), a


def pool_usage(device=0, reset_high=False):
    """(used_current, used_high) bytes of the device's default stream-ordered pool."""
    cur, high = C.c_ulonglong(), C.c_ulonglong()
    st = _lib.tddft_pool_usage(int(device), C.byref(cur), C.byref(high), int(bool(reset_high)))
    if st != OK:
        raise TddftError(st, "tddft_pool_usage failed")
    return cur.value, high.value


def default_opts(**kw) -> Opts:
    o = Opts()
    _lib.tddft_default_opts(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise AttributeError(k)
        setattr(o, k, v)
    return o


def _problem_args(n_occ, n_vir, eps_occ, eps_vir, L_oo, L_ov, L_vv, Lr_oo, Lr_ov, Lr_vv, ris_K_index,
                  a_x=0.25, coulomb_factor=2.0, t_cut_ha=None, precisions=3, hbm_budget_gb=0.0, dtype=F64):
    """(Desc, the nine array pointers of tddft_create, keepalives, inputs_on_device)."""
    d = Desc()
    _lib.tddft_default_desc(C.byref(d))
    d.n_occ, d.n_vir = int(n_occ), int(n_vir)
    d.n_aux = int(L_ov.shape[0])
    d.n_aux_ris_J = int(Lr_ov.shape[0]) if Lr_ov is not None else 0
    d.n_aux_ris_K = int(len(ris_K_index)) if ris_K_index is not None else 0
    d.a_x, d.coulomb_factor = float(a_x), float(coulomb_factor)
    if t_cut_ha is not None:
        d.t_cut_ha = float(t_cut_ha)
    d.precisions, d.hbm_budget_gb = int(precisions), float(hbm_budget_gb)
    fdt = np.float64 if dtype == F64 else np.float32
    keep, ptrs = [], []
    for arr, dt in ((eps_occ, np.float64), (eps_vir, np.float64), (L_oo, fdt), (L_ov, fdt),
                    (L_vv, fdt), (Lr_oo, fdt), (Lr_ov, fdt), (Lr_vv, fdt), (ris_K_index, np.int32)):
        p, k = _ptr(arr, dt)
        ptrs.append(p)
        keep.append(k)
    return d, ptrs, keep, _is_cuda(L_ov)


def _problem_kw(prob):
    """tddft_create arguments of a synthetic problem (ris exchange rows = its s rows)."""
    return dict(n_occ=prob.n_occ, n_vir=prob.n_vir, eps_occ=prob.eps_occ, eps_vir=prob.eps_vir,
                L_oo=prob.L_oo, L_ov=prob.L_ov, L_vv=prob.L_vv, Lr_oo=prob.Lr_oo[prob.ris_K_index],
                Lr_ov=prob.Lr_ov, Lr_vv=prob.Lr_vv[prob.ris_K_index], ris_K_index=prob.ris_K_index,
                a_x=prob.a_x, coulomb_factor=prob.coulomb_factor, t_cut_ha=prob.t_cut_ha)


def _fill_request(r: Request, kind, opts: Opts, mu=None, omegas=None):
    """Point a Request at fresh output arrays; returns them (to keep alive)."""
    r.opts = opts
    bufs = {}
    if kind in (0, 1):
        k = opts.n_states
        bufs["omega"], bufs["resid"] = np.zeros(k), np.zeros(k)
        r.omega = bufs["omega"].ctypes.data
        r.resid = bufs["resid"].ctypes.data
    else:
        mu = np.ascontiguousarray(np.atleast_2d(mu), dtype=np.float64)
        om = np.ascontiguousarray(omegas, dtype=np.float64)
        bufs["mu"], bufs["freqs"] = mu, om
        bufs["alpha"] = np.zeros((om.size, mu.shape[0], mu.shape[0]))
        r.mu, r.n_dip, r.freqs, r.n_freq = mu.ctypes.data, mu.shape[0], om.ctypes.data, om.size
        r.alpha = bufs["alpha"].ctypes.data
    return bufs


def estimate_bytes(desc: Desc, kind, opts: Opts, n_dip=0, n_freq=0):
    """(factor bytes, work bytes) that a server charges for one request."""
    f, w = C.c_ulonglong(), C.c_ulonglong()
    st = _lib.tddft_estimate_bytes(C.byref(desc), int(kind), C.byref(opts), int(n_dip), int(n_freq),
                                   C.byref(f), C.byref(w))
    if st != OK:
        raise TddftError(st, "bad desc or kind")
    return f.value, w.value


class Solver:
    """One context: resident factors + the request queue (include/tddft.h)."""

    def __init__(self, n_occ, n_vir, eps_occ, eps_vir, L_oo, L_ov, L_vv, Lr_oo, Lr_ov, Lr_vv,
                 ris_K_index, a_x=0.25, coulomb_factor=2.0, t_cut_ha=None, precisions=3,
                 hbm_budget_gb=0.0, dtype=F64, stream=None):
        d, ptrs, keep, on_dev = _problem_args(n_occ, n_vir, eps_occ, eps_vir, L_oo, L_ov, L_vv, Lr_oo, Lr_ov,
                                              Lr_vv, ris_K_index, a_x, coulomb_factor, t_cut_ha, precisions,
                                              hbm_budget_gb, dtype)
        self.desc = d
        self.n_ov = d.n_occ * d.n_vir
        h = C.c_void_p()
        st = _lib.tddft_create(C.byref(d), *ptrs, int(dtype), 1 if on_dev else 0,
                               C.c_void_p(stream) if stream else None, C.byref(h))
        if st != OK:
            raise TddftError(st, _lib.tddft_last_error(None).decode())
        self.h = h
        self._pending = {}

    @classmethod
    def from_problem(cls, prob, **kw):
        """A context for a synthetic problem, with its variant terms if it has any."""
        s = cls(**_problem_kw(prob), **kw)
        ex = prob.extra or {}
        dt = kw.get("dtype", F64)
        if ex.get("exchange_lr"):
            lr = ex["exchange_lr"]
            s.add_exchange(lr["b_x"], lr["M_oo"], lr["M_ov"], lr["M_vv"], dtype=dt)
        if ex.get("kernel"):
            s.add_kernel(ex["kernel"]["w"], ex["kernel"]["F_ov"], dtype=dt)
        return s

    def add_exchange(self, b_x, M_oo, M_ov, M_vv, dtype=F64):
        """Second exchange factor set with weight b_x (tddft_add_exchange)."""
        fdt = np.float64 if dtype == F64 else np.float32
        ptrs = [_ptr(a, fdt) for a in (M_oo, M_ov, M_vv)]
        st = _lib.tddft_add_exchange(self.h, float(b_x), int(M_ov.shape[0]), *(p for p, _ in ptrs), int(dtype),
                                     1 if _is_cuda(M_ov) else 0)
        self._check(st, allow_noconv=False)

    def add_kernel(self, w, F_ov, dtype=F64):
        """Low-rank kernel sum_g w_g F^g_ia F^g_jb (tddft_add_kernel)."""
        fdt = np.float64 if dtype == F64 else np.float32
        on_dev = _is_cuda(F_ov)
        if on_dev and not _is_cuda(w):   # the weights go where the rows are
            import torch
            w = torch.as_tensor(np.asarray(w, dtype=np.float64), device=F_ov.device)
        pw, kw_ = _ptr(w, np.float64)
        pf, kf = _ptr(F_ov, fdt)
        st = _lib.tddft_add_kernel(self.h, int(F_ov.shape[0]), pw, pf, int(dtype), 1 if on_dev else 0)
        self._check(st, allow_noconv=False)

    def _check(self, st, allow_noconv=True):
        if st == OK or (allow_noconv and st == ERR_NOCONV):
            return st
        raise TddftError(st, _lib.tddft_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            _lib.tddft_destroy(self.h)
            self.h = None

    __del__ = close

    def device_bytes(self):
        return _lib.tddft_device_bytes(self.h)

    def profile(self, enable=True):
        self._check(_lib.tddft_profile(self.h, int(bool(enable))), allow_noconv=False)

    def profile_read(self, which=0):
        """which 0: the tcgen05 K1 contraction; 1: the SIMT one."""
        n, ms, fl = C.c_longlong(), C.c_double(), C.c_double()
        self._check(_lib.tddft_profile_read(self.h, which, C.byref(n), C.byref(ms), C.byref(fl)),
                    allow_noconv=False)
        return dict(launches=n.value, ms=ms.value, flops=fl.value)

    def profile_records(self, which=0):
        """Per-launch (ms, algorithmic flops, algorithmic bytes) arrays of the profiled kernel."""
        n = C.c_int()
        self._check(_lib.tddft_profile_records(self.h, which, 0, None, None, None, C.byref(n)), allow_noconv=False)
        ms, fl, by = np.zeros(n.value), np.zeros(n.value), np.zeros(n.value)
        vp = lambda a: a.ctypes.data_as(C.c_void_p)
        self._check(_lib.tddft_profile_records(self.h, which, n.value, vp(ms), vp(fl), vp(by), C.byref(n)),
                    allow_noconv=False)
        return ms, fl, by

    def solve_tda(self, opts: Opts, want_vectors=True):
        k = opts.n_states
        om, rs = np.zeros(k), np.zeros(k)
        X = np.zeros((k, self.n_ov)) if want_vectors else None
        st = Stats()
        s = _lib.tddft_solve_tda(self.h, C.byref(opts), om.ctypes.data_as(C.c_void_p),
                                 X.ctypes.data_as(C.c_void_p) if X is not None else None,
                                 rs.ctypes.data_as(C.c_void_p), C.byref(st))
        self._check(s)
        return dict(status=s, omega=om, X=X, resid=rs, stats=st.as_dict())

    def solve_rpa(self, opts: Opts, want_vectors=True):
        k = opts.n_states
        om, rs = np.zeros(k), np.zeros(k)
        X = np.zeros((k, self.n_ov)) if want_vectors else None
        Y = np.zeros((k, self.n_ov)) if want_vectors else None
        st = Stats()
        vp = lambda a: a.ctypes.data_as(C.c_void_p) if a is not None else None
        s = _lib.tddft_solve_rpa(self.h, C.byref(opts), vp(om), vp(X), vp(Y), vp(rs), C.byref(st))
        self._check(s)
        return dict(status=s, omega=om, X=X, Y=Y, resid=rs, stats=st.as_dict())

    def solve_polar(self, opts: Opts, mu, omegas):
        mu = np.ascontiguousarray(np.atleast_2d(mu), dtype=np.float64)
        om = np.ascontiguousarray(omegas, dtype=np.float64)
        nd, nf = mu.shape[0], om.size
        alpha = np.zeros((nf, nd, nd))
        st = Stats()
        s = _lib.tddft_solve_polar(self.h, C.byref(opts), mu.ctypes.data_as(C.c_void_p), nd,
                                   om.ctypes.data_as(C.c_void_p), nf, alpha.ctypes.data_as(C.c_void_p),
                                   C.byref(st))
        self._check(s)
        return dict(status=s, alpha=alpha, stats=st.as_dict())

    def apply(self, kind, X, precision=PLAIN, tensor_cores=False):
        """kind 0: A X, 1: ((A+B)X, (A-B)X), 2: T X (ris), 3: ris pair.
        tensor_cores: 0/False SIMT, 1/True tcgen05, 2 tcgen05 with the FP8 ris rows."""
        if _is_cuda(X):
            import torch
            out0 = torch.empty_like(X)
            out1 = torch.empty_like(X) if kind in (1, 3) else None
            s = _lib.tddft_apply(self.h, kind, precision, int(tensor_cores), C.c_void_p(X.data_ptr()),
                                 X.shape[0], C.c_void_p(out0.data_ptr()),
                                 C.c_void_p(out1.data_ptr()) if out1 is not None else None, 1)
        else:
            X = np.ascontiguousarray(np.atleast_2d(X), dtype=np.float64)
            out0 = np.zeros_like(X)
            out1 = np.zeros_like(X) if kind in (1, 3) else None
            s = _lib.tddft_apply(self.h, kind, precision, int(tensor_cores),
                                 X.ctypes.data_as(C.c_void_p), X.shape[0], out0.ctypes.data_as(C.c_void_p),
                                 out1.ctypes.data_as(C.c_void_p) if out1 is not None else None, 0)
        self._check(s, allow_noconv=False)
        return (out0, out1) if out1 is not None else out0

    # -- asynchronous requests ------------------------------------------------
    def submit(self, kind, opts: Opts, mu=None, omegas=None):
        """kind 0 TDA, 1 RPA, 2 polar.  Returns a ticket; buffers are kept alive here."""
        r = Request()
        bufs = _fill_request(r, kind, opts, mu, omegas)
        t = C.c_ulonglong()
        s = _lib.tddft_submit(self.h, kind, C.byref(r), C.byref(t))
        self._check(s, allow_noconv=False)
        self._pending[t.value] = (r, bufs, kind)
        return t.value

    def poll(self, ticket, timeout_ms=0):
        """Returns None while pending; else the result dict (status included)."""
        s = _lib.tddft_poll(self.h, ticket, int(timeout_ms))
        if s in (PENDING, ERR_TIMEOUT):
            return None
        r, bufs, kind = self._pending.pop(ticket)
        out = dict(status=s, stats=r.stats.as_dict())
        if s not in (OK, ERR_NOCONV):
            out["error"] = _lib.tddft_last_error(self.h).decode()
        out.update({k: v for k, v in bufs.items() if k in ("omega", "resid", "alpha")})
        return out


def solve_tda_batch(solvers, opts):
    """Batched TDA solves (tddft_solve_tda_batch): solvers[i] with opts[i],
    advanced together.  Returns (status, list of {omega, resid, stats}, info)."""
    n = len(solvers)
    if n == 0 or len(opts) != n:
        raise ValueError("need one opts per solver")
    hs = (C.c_void_p * n)(*[s.h for s in solvers])
    oa = (Opts * n)(*opts)
    ks = [min(o.n_states, s.n_ov) for s, o in zip(solvers, opts)]
    om, rs = np.zeros(sum(ks)), np.zeros(sum(ks))
    st = (Stats * n)()
    info = BatchInfo()
    status = _lib.tddft_solve_tda_batch(hs, n, oa, om.ctypes.data_as(C.c_void_p), rs.ctypes.data_as(C.c_void_p),
                                        st, C.byref(info))
    if status not in (OK, ERR_NOCONV):
        raise TddftError(status, _lib.tddft_last_error(solvers[0].h).decode())
    out, off = [], 0
    for i, k in enumerate(ks):
        out.append(dict(omega=om[off:off + k].copy(), resid=rs[off:off + k].copy(), stats=st[i].as_dict()))
        off += k
    return status, out, info.as_dict()


class Server:
    """Continuous admission of independent solves under a device-memory budget
    (tddft_server_* in include/tddft.h).  A request brings its own problem
    (``problem``: a synthetic problem, or ``create_kw``: tddft_create arguments
    as for Solver) or runs on an existing ``solver``'s resident factors."""

    def __init__(self, hbm_budget_gb=0.0, max_active=4):
        h = C.c_void_p()
        st = _lib.tddft_server_create(float(hbm_budget_gb), int(max_active), C.byref(h))
        if st != OK:
            raise TddftError(st, "tddft_server_create failed")
        self.h = h
        self._pending = {}

    def submit(self, kind, opts: Opts, problem=None, create_kw=None, solver=None, mu=None, omegas=None,
               dtype=F64, precisions=3):
        """kind 0 TDA, 1 Casida, 2 polarizability.  Returns a ticket."""
        q = ServeRequest()
        keep = []
        if solver is not None:
            q.ctx = solver.h
            keep.append(solver)
        else:
            kw = dict(create_kw) if create_kw is not None else _problem_kw(problem)
            kw.setdefault("precisions", precisions)
            kw.setdefault("dtype", dtype)
            d, ptrs, k, on_dev = _problem_args(**kw)
            keep.append(k)
            q.desc = d
            (q.eps_occ, q.eps_vir, q.L_oo, q.L_ov, q.L_vv, q.Lr_oo, q.Lr_ov, q.Lr_vv,
             q.ris_K_index) = [p.value if p is not None else None for p in ptrs]
            q.dtype, q.inputs_on_device = int(kw["dtype"]), 1 if on_dev else 0
        q.kind = int(kind)
        bufs = _fill_request(q.req, kind, opts, mu, omegas)
        t = C.c_ulonglong()
        st = _lib.tddft_server_submit(self.h, C.byref(q), C.byref(t))
        if st != OK:
            raise TddftError(st, q.error.decode())
        self._pending[t.value] = (q, bufs, keep)
        return t.value

    def poll(self, ticket, timeout_ms=0):
        """None while queued or running; else the result dict with its timings."""
        st = _lib.tddft_server_poll(self.h, ticket, int(timeout_ms))
        if st in (PENDING, ERR_TIMEOUT):
            return None
        q, bufs, _ = self._pending.pop(ticket)
        out = dict(status=st, stats=q.req.stats.as_dict(), charged_bytes=q.charged_bytes,
                   t_submit_s=q.t_submit_s, t_start_s=q.t_start_s, t_end_s=q.t_end_s,
                   latency_s=q.t_end_s - q.t_submit_s)
        if st not in (OK, ERR_NOCONV):
            out["error"] = q.error.decode()
        out.update({k: v for k, v in bufs.items() if k in ("omega", "resid", "alpha")})
        return out

    def info(self):
        s = ServerState()
        st = _lib.tddft_server_info(self.h, C.byref(s))
        if st != OK:
            raise TddftError(st, "tddft_server_info failed")
        return s.as_dict()

    def close(self):
        """Runs every queued request to its end first."""
        if getattr(self, "h", None):
            _lib.tddft_server_destroy(self.h)
            self.h = None

    __del__ = close

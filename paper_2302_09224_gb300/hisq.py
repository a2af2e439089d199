"""ctypes binding of ``libhisq.so`` (the C ABI declared in ``include/hisq.h``).

Argument marshalling only: every step of the stencil, the codecs and the
solvers runs in the library's CUDA kernels.  Functions keep the C names;
arrays may be torch tensors (host or device: ``data_ptr()`` is passed) or
numpy arrays (host).  The library is opened on first use; if it has not been
built this raises -- there is no other implementation to fall back to.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhisq.so")

# ---------------------------------------------------------------------------
# enums (mirror include/hisq.h)
# ---------------------------------------------------------------------------
HISQ_OK, HISQ_EINVAL, HISQ_ENOMEM, HISQ_ENOTCONV, HISQ_EBREAKDOWN = 0, 1, 2, 3, 4
HISQ_ECUDA, HISQ_EBUSY, HISQ_ETIMEOUT, HISQ_ENOTFOUND, HISQ_ERANGE = 5, 6, 7, 8, 9
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ENOTCONV", 4: "EBREAKDOWN", 5: "ECUDA", 6: "EBUSY",
                7: "ETIMEOUT", 8: "ENOTFOUND", 9: "ERANGE"}

HISQ_GAUGE_F64, HISQ_GAUGE_F32, HISQ_GAUGE_FIX16, HISQ_GAUGE_FIX32, HISQ_GAUGE_SE15 = 0, 1, 2, 3, 4
HISQ_SPINOR_F64, HISQ_SPINOR_F32, HISQ_SPINOR_HALF16, HISQ_SPINOR_INT20, HISQ_SPINOR_INT30, HISQ_SPINOR_INT14 = \
    0, 1, 2, 3, 4, 5
HISQ_COMPUTE_F32, HISQ_COMPUTE_F64 = 0, 1
HISQ_GAUGE_ANTIPERIODIC_T = 0x1
HISQ_GAUGE_ON_DEVICE = 0x2
HISQ_PROF_STENCIL, HISQ_PROF_STENCIL_HI, HISQ_PROF_BLAS, HISQ_PROF_CONVERT = 0, 1, 2, 3
HISQ_MAX_SHIFTS = 32

SPINOR_FMT = {"f64": 0, "f32": 1, "half": 2, "int20": 3, "int30": 4, "int14": 5}


class hisq_prec(ctypes.Structure):
    _fields_ = [("gauge", ctypes.c_int32), ("spinor", ctypes.c_int32), ("compute", ctypes.c_int32),
                ("fat_recon", ctypes.c_int32), ("long_recon", ctypes.c_int32)]

    def __repr__(self):
        return (f"hisq_prec(gauge={self.gauge}, spinor={self.spinor}, compute={self.compute}, "
                f"fat_recon={self.fat_recon}, long_recon={self.long_recon})")


def prec(name: str, long_recon: int = 12) -> hisq_prec:
    """Named triplets of Sec. 4 (gauge / fermion / compute)."""
    table = {
        "f64": (HISQ_GAUGE_F64, HISQ_SPINOR_F64, HISQ_COMPUTE_F64),
        "f32": (HISQ_GAUGE_F32, HISQ_SPINOR_F32, HISQ_COMPUTE_F32),
        "half": (HISQ_GAUGE_FIX16, HISQ_SPINOR_HALF16, HISQ_COMPUTE_F32),
        "int20": (HISQ_GAUGE_FIX16, HISQ_SPINOR_INT20, HISQ_COMPUTE_F32),
        "int14": (HISQ_GAUGE_FIX16, HISQ_SPINOR_INT14, HISQ_COMPUTE_F32),
        "int20se": (HISQ_GAUGE_SE15, HISQ_SPINOR_INT20, HISQ_COMPUTE_F32),
        "int30": (HISQ_GAUGE_FIX32, HISQ_SPINOR_INT30, HISQ_COMPUTE_F64),
        "int30f32": (HISQ_GAUGE_FIX32, HISQ_SPINOR_INT30, HISQ_COMPUTE_F32),
    }
    g, s, c = table[name]
    return hisq_prec(g, s, c, 18, long_recon)


class hisq_solver_params(ctypes.Structure):
    _fields_ = [("mass", ctypes.c_double), ("tol", ctypes.c_double), ("maxiter", ctypes.c_int32),
                ("delta", ctypes.c_double), ("sloppy", hisq_prec), ("refine", hisq_prec),
                ("nbuf", ctypes.c_int32), ("use_init_guess", ctypes.c_int32), ("on_device", ctypes.c_int32),
                ("pr_beta", ctypes.c_int32), ("reproject", ctypes.c_int32), ("l", ctypes.c_int32),
                ("use_graph", ctypes.c_int32), ("nrhs", ctypes.c_int32), ("rhs_tile", ctypes.c_int32),
                ("rhs_kernel", ctypes.c_int32), ("stream", ctypes.c_void_p), ("history", ctypes.c_void_p),
                ("history_len", ctypes.c_int32), ("ru_trigger", ctypes.c_int32)]


class hisq_solve_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("matvecs", ctypes.c_int32), ("matvecs_hi", ctypes.c_int32),
                ("reliable_updates", ctypes.c_int32), ("true_residual", ctypes.c_double),
                ("seconds", ctypes.c_double), ("nshift", ctypes.c_int32),
                ("shift_iters", ctypes.c_int32 * HISQ_MAX_SHIFTS),
                ("shift_resid_ms", ctypes.c_double * HISQ_MAX_SHIFTS),
                ("shift_resid", ctypes.c_double * HISQ_MAX_SHIFTS),
                ("refine_iters", ctypes.c_int32 * HISQ_MAX_SHIFTS)]


HISQ_REQ_CG, HISQ_REQ_MULTISHIFT = 0, 1


class hisq_request(ctypes.Structure):
    _fields_ = [("gauge", ctypes.c_void_p), ("kind", ctypes.c_int32), ("mass", ctypes.c_double),
                ("tol", ctypes.c_double), ("nshift", ctypes.c_int32), ("sigma", ctypes.c_void_p),
                ("shift_tol", ctypes.c_void_p), ("b", ctypes.c_void_p), ("x", ctypes.c_void_p),
                ("on_device", ctypes.c_int32), ("sloppy", hisq_prec), ("refine", hisq_prec),
                ("maxiter", ctypes.c_int32)]


class hisq_serve_stats_t(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_int64), ("pending", ctypes.c_int64), ("latency_p50_s", ctypes.c_double),
                ("latency_p99_s", ctypes.c_double), ("solves_per_s", ctypes.c_double)]


class hisq_kernel_stats(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double), ("launches", ctypes.c_int64), ("bytes", ctypes.c_double)]


class HisqError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None

_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_I64 = ctypes.c_int64
_SZ = ctypes.c_size_t

_SIGS = {
    "hisq_create": (_I, [_I, _SZ, ctypes.POINTER(_P)]),
    "hisq_destroy": (None, [_P]),
    "hisq_last_error": (ctypes.c_char_p, [_P]),
    "hisq_mem_used": (_SZ, [_P]),
    "hisq_load_gauge": (_I, [_P, _P, _P, _P, ctypes.c_uint, ctypes.POINTER(_P)]),
    "hisq_free_gauge": (None, [_P, _P]),
    "hisq_gauge_scale": (_D, [_P, _I]),
    "hisq_dslash": (_I, [_P, _P, hisq_prec, _I, _D, _P, _P, _P, _I, _P]),
    "hisq_dslash_noalloc": (_I, [_P, _P, hisq_prec, _I, _D, _P, _P, _P, _P]),
    "hisq_spinor_bytes": (_SZ, [_I, _I64]),
    "hisq_spinor_pack": (_I, [_P, _I, _I64, _P, _P, ctypes.POINTER(_I64), _P]),
    "hisq_spinor_pack32": (_I, [_P, _I, _I64, _P, _P, ctypes.POINTER(_I64), _P]),
    "hisq_spinor_pack_pair_int30": (_I, [_P, _I64, _P, _P, ctypes.POINTER(_I64), _P]),
    "hisq_spinor_unpack": (_I, [_P, _I, _I, _I64, _P, _P, _P]),
    "hisq_profile_enable": (None, [_P, _I]),
    "hisq_profile_reset": (None, [_P]),
    "hisq_profile_select": (None, [_P, ctypes.c_uint]),
    "hisq_profile_sample": (_I, [_P, _I]),
    "hisq_profile_read": (_I, [_P, _I, ctypes.POINTER(hisq_kernel_stats)]),
    "hisq_launch_count": (_I64, [_P]),
    "hisq_stencil_config": (_I, [_I]),
    "hisq_stencil_config_reduce": (_I, [_I]),
    "hisq_programmatic_launch": (_I, [_I]),
    "hisq_cg_split_scalars": (_I, [_I]),
    "hisq_mee_fused": (_I, [_I]),
    "hisq_mee_fused_shape": (None, [_I, _I]),
    "hisq_mee_fused_wait_test": (None, [ctypes.c_uint, _I]),
    "hisq_stencil_config_in_use": (_I, [_P, hisq_prec, _I]),
    "hisq_default_params": (None, [ctypes.POINTER(hisq_solver_params)]),
    "hisq_cg": (_I, [_P, _P, ctypes.POINTER(hisq_solver_params), _P, _P, ctypes.POINTER(hisq_solve_info)]),
    "hisq_multishift_cg": (_I, [_P, _P, ctypes.POINTER(hisq_solver_params), _I, _P, _P, _P, _P,
                                ctypes.POINTER(hisq_solve_info)]),
    "hisq_bicgstabl": (_I, [_P, _P, ctypes.POINTER(hisq_solver_params), _P, _P,
                            ctypes.POINTER(hisq_solve_info)]),
    "hisq_solve_full": (_I, [_P, _P, ctypes.POINTER(hisq_solver_params), _P, _P,
                             ctypes.POINTER(hisq_solve_info)]),
    "hisq_submit": (_I, [_P, ctypes.POINTER(hisq_request), ctypes.POINTER(ctypes.c_uint64)]),
    "hisq_poll": (_I, [_P, ctypes.c_uint64, ctypes.POINTER(_I), ctypes.POINTER(hisq_solve_info)]),
    "hisq_wait": (_I, [_P, ctypes.c_uint64, _D, ctypes.POINTER(hisq_solve_info)]),
    "hisq_serve_stats": (_I, [_P, ctypes.POINTER(hisq_serve_stats_t)]),
}


def lib():
    """The loaded library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built; run __graft_entry__.build() (nvcc, sm_103a)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name, None)
            if f is None:
                continue
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    """Names from _SIGS that the library exports."""
    L = lib()
    return [n for n in _SIGS if hasattr(L, n)]


# ---------------------------------------------------------------------------
# marshalling helpers
# ---------------------------------------------------------------------------
def _ptr(a):
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    import numpy as np

    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    raise TypeError(f"cannot pass {type(a)} as a pointer")


def _check(ctx, status: int):
    if status != HISQ_OK:
        msg = lib().hisq_last_error(ctx).decode() if ctx else ""
        raise HisqError(status, msg)
    return status


def _stream(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


# ---------------------------------------------------------------------------
# the ABI, one function each
# ---------------------------------------------------------------------------
def hisq_create(device: int = 0, hbm_budget: int = 0):
    h = _P()
    st = lib().hisq_create(int(device), int(hbm_budget), ctypes.byref(h))
    if st != HISQ_OK:
        raise HisqError(st, "hisq_create failed")
    return h.value


def hisq_destroy(ctx):
    lib().hisq_destroy(ctx)


def hisq_last_error(ctx) -> str:
    return lib().hisq_last_error(ctx).decode()


def hisq_mem_used(ctx) -> int:
    return int(lib().hisq_mem_used(ctx))


def hisq_load_gauge(ctx, dims, fat, lng, flags: int = 0):
    import numpy as np

    d = np.ascontiguousarray([int(x) for x in dims], dtype=np.int32)
    on_dev = hasattr(fat, "is_cuda") and fat.is_cuda
    if on_dev:
        flags |= HISQ_GAUGE_ON_DEVICE
    g = _P()
    _check(ctx, lib().hisq_load_gauge(ctx, d.ctypes.data, _ptr(fat), _ptr(lng), int(flags), ctypes.byref(g)))
    return g.value


def hisq_free_gauge(ctx, g):
    lib().hisq_free_gauge(ctx, g)


def hisq_gauge_scale(g, which: int) -> float:
    return float(lib().hisq_gauge_scale(g, int(which)))


def hisq_dslash(ctx, g, p: hisq_prec, out_parity: int, a: float, xpay_in, x, out, on_device: bool, stream=None):
    _check(ctx, lib().hisq_dslash(ctx, g, p, int(out_parity), float(a), _ptr(xpay_in), _ptr(x), _ptr(out),
                                  int(bool(on_device)), _stream(stream)))


HISQ_NOALLOC_MAX_SITES = 32768


def hisq_dslash_noalloc(ctx, g, p: hisq_prec, out_parity: int, a: float, xpay_in, x, out, stream=None):
    """hisq_dslash on device pointers without any device allocation (fixed scratch)."""
    _check(ctx, lib().hisq_dslash_noalloc(ctx, g, p, int(out_parity), float(a), _ptr(xpay_in), _ptr(x),
                                          _ptr(out), _stream(stream)))


def hisq_spinor_bytes(sfmt: int, n: int) -> int:
    return int(lib().hisq_spinor_bytes(int(sfmt), int(n)))


def hisq_spinor_pack(ctx, sfmt: int, n: int, x, packed, stream=None) -> int:
    bad = _I64(0)
    _check(ctx, lib().hisq_spinor_pack(ctx, int(sfmt), int(n), _ptr(x), _ptr(packed), ctypes.byref(bad),
                                       _stream(stream)))
    return int(bad.value)


def hisq_spinor_pack32(ctx, sfmt: int, n: int, x, packed, stream=None) -> int:
    bad = _I64(0)
    _check(ctx, lib().hisq_spinor_pack32(ctx, int(sfmt), int(n), _ptr(x), _ptr(packed), ctypes.byref(bad),
                                         _stream(stream)))
    return int(bad.value)


def hisq_spinor_pack_pair_int30(ctx, n: int, x, packed, stream=None) -> int:
    bad = _I64(0)
    _check(ctx, lib().hisq_spinor_pack_pair_int30(ctx, int(n), _ptr(x), _ptr(packed), ctypes.byref(bad),
                                                  _stream(stream)))
    return int(bad.value)


def hisq_spinor_unpack(ctx, sfmt: int, compute: int, n: int, packed, out, stream=None):
    _check(ctx, lib().hisq_spinor_unpack(ctx, int(sfmt), int(compute), int(n), _ptr(packed), _ptr(out),
                                         _stream(stream)))


def hisq_profile_enable(ctx, on: bool):
    lib().hisq_profile_enable(ctx, int(bool(on)))


def hisq_profile_reset(ctx):
    lib().hisq_profile_reset(ctx)


def hisq_profile_select(ctx, mask: int):
    lib().hisq_profile_select(ctx, int(mask) & 0xFFFFFFFF)


def hisq_profile_sample(ctx, every: int):
    _check(ctx, lib().hisq_profile_sample(ctx, int(every)))


def hisq_profile_read(ctx, kind: int) -> hisq_kernel_stats:
    s = hisq_kernel_stats()
    _check(ctx, lib().hisq_profile_read(ctx, int(kind), ctypes.byref(s)))
    return s


def hisq_stencil_config(cfg: int) -> int:
    return int(lib().hisq_stencil_config(int(cfg)))


def hisq_mee_fused(mode: int) -> int:
    return int(lib().hisq_mee_fused(int(mode)))


def hisq_mee_fused_shape(lag: int, blocks_per_sm: int):
    lib().hisq_mee_fused_shape(int(lag), int(blocks_per_sm))


def hisq_mee_fused_wait_test(polls: int, unreachable: bool):
    lib().hisq_mee_fused_wait_test(int(polls) & 0xFFFFFFFF, int(bool(unreachable)))


def hisq_programmatic_launch(mode: int) -> int:
    return int(lib().hisq_programmatic_launch(int(mode)))


def hisq_cg_split_scalars(mode: int) -> int:
    return int(lib().hisq_cg_split_scalars(int(mode)))


def hisq_stencil_config_reduce(cfg: int) -> int:
    return int(lib().hisq_stencil_config_reduce(int(cfg)))


def hisq_stencil_config_in_use(g, p: hisq_prec, reduce: bool) -> int:
    return int(lib().hisq_stencil_config_in_use(g, p, int(bool(reduce))))


def hisq_launch_count(ctx) -> int:
    return int(lib().hisq_launch_count(ctx))


def hisq_default_params() -> hisq_solver_params:
    p = hisq_solver_params()
    lib().hisq_default_params(ctypes.byref(p))
    return p


def hisq_cg(ctx, g, params: hisq_solver_params, b, x) -> tuple[int, hisq_solve_info]:
    """Returns (status, info); ENOTCONV is returned, other failures raise."""
    info = hisq_solve_info()
    st = lib().hisq_cg(ctx, g, ctypes.byref(params), _ptr(b), _ptr(x), ctypes.byref(info))
    if st not in (HISQ_OK, HISQ_ENOTCONV):
        _check(ctx, st)
    return st, info


def hisq_solve_full(ctx, g, params: hisq_solver_params, b, x) -> tuple[int, hisq_solve_info]:
    """Full-lattice (2m + D) x = b by even/odd reduction; returns (status, info) like hisq_cg."""
    info = hisq_solve_info()
    st = lib().hisq_solve_full(ctx, g, ctypes.byref(params), _ptr(b), _ptr(x), ctypes.byref(info))
    if st not in (HISQ_OK, HISQ_ENOTCONV):
        _check(ctx, st)
    return st, info


def set_history(params: hisq_solver_params, buf):
    """Point params.history at a float64 numpy array (kept alive by the caller)."""
    params.history = buf.ctypes.data
    params.history_len = int(buf.size)


def hisq_multishift_cg(ctx, g, params: hisq_solver_params, sigma, tol, b, xs) -> tuple[int, hisq_solve_info]:
    n = len(sigma)
    sig = (ctypes.c_double * n)(*[float(s) for s in sigma])
    tl = (ctypes.c_double * n)(*[float(t) for t in tol])
    xp = (ctypes.c_void_p * n)(*[_ptr(x) for x in xs])
    info = hisq_solve_info()
    st = lib().hisq_multishift_cg(ctx, g, ctypes.byref(params), n, sig, tl, _ptr(b), xp, ctypes.byref(info))
    if st not in (HISQ_OK, HISQ_ENOTCONV):
        _check(ctx, st)
    return st, info


def hisq_bicgstabl(ctx, g, params: hisq_solver_params, b, x) -> tuple[int, hisq_solve_info]:
    info = hisq_solve_info()
    st = lib().hisq_bicgstabl(ctx, g, ctypes.byref(params), _ptr(b), _ptr(x), ctypes.byref(info))
    if st not in (HISQ_OK, HISQ_ENOTCONV):
        _check(ctx, st)
    return st, info


def hisq_submit(ctx, gauge, kind: int, mass: float, b, x, on_device: bool, tol: float = 1e-10, sigma=None,
                shift_tol=None, sloppy: hisq_prec | None = None, refine: hisq_prec | None = None,
                maxiter: int = 100000) -> int:
    """Queue a solve; returns its ticket.  b and x must stay alive until it is done."""
    r = hisq_request()
    r.gauge = gauge
    r.kind = int(kind)
    r.mass = float(mass)
    r.tol = float(tol)
    keep = []
    if kind == HISQ_REQ_MULTISHIFT:
        n = len(sigma)
        sa = (ctypes.c_double * n)(*[float(v) for v in sigma])
        ta = (ctypes.c_double * n)(*[float(v) for v in shift_tol])
        keep += [sa, ta]
        r.nshift = n
        r.sigma = ctypes.cast(sa, ctypes.c_void_p)
        r.shift_tol = ctypes.cast(ta, ctypes.c_void_p)
    r.b = _ptr(b)
    r.x = _ptr(x)
    r.on_device = int(bool(on_device))
    r.sloppy = sloppy if sloppy is not None else prec("int20")
    r.refine = refine if refine is not None else prec("int20")
    r.maxiter = int(maxiter)
    t = ctypes.c_uint64(0)
    _check(ctx, lib().hisq_submit(ctx, ctypes.byref(r), ctypes.byref(t)))
    return int(t.value)


def hisq_poll(ctx, ticket: int):
    """(done, status, info); status is the solve's once done."""
    done = ctypes.c_int(0)
    info = hisq_solve_info()
    st = lib().hisq_poll(ctx, ctypes.c_uint64(ticket), ctypes.byref(done), ctypes.byref(info))
    if st in (HISQ_EINVAL, HISQ_ENOTFOUND):
        _check(ctx, st)
    return bool(done.value), st, info


def hisq_wait(ctx, ticket: int, timeout_s: float = 60.0):
    """(status, info) once done; raises HisqError on ETIMEOUT or an unknown ticket."""
    info = hisq_solve_info()
    st = lib().hisq_wait(ctx, ctypes.c_uint64(ticket), float(timeout_s), ctypes.byref(info))
    if st in (HISQ_ETIMEOUT, HISQ_ENOTFOUND, HISQ_EINVAL):
        _check(ctx, st)
    return st, info


def hisq_serve_stats(ctx) -> hisq_serve_stats_t:
    s = hisq_serve_stats_t()
    _check(ctx, lib().hisq_serve_stats(ctx, ctypes.byref(s)))
    return s

"""FP64 CPU oracle for the HISQ stencil, its storage formats and solvers.

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package.  It is a ctypes front
end to ``hisq_oracle.c`` (plain C, FP64, OpenMP over sites), which shares no
code with the CUDA path.  Every function cites the passage of Clark et al.,
"Maximizing the Bang Per Bit" (Lattice 2022) that it follows in the C source.

Arrays are numpy (or CPU torch) float64 in the C ABI's host layouts:
gauge ``[mu][t][z][y][x][3][3][2]``, half-lattice spinor ``[Vh][3][2]``,
full-lattice spinor ``[2][Vh][3][2]`` (even parity first).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hisq_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

# IEEE arithmetic without contraction, so the FP32 codec steps round exactly
# as written; -fcx-limited-range only drops the Annex G inf/nan recovery of
# complex multiplication, which finite operands never reach.
CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
          "-fcx-limited-range", "-fno-fast-math"]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (seconds); returns the library path."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None

_d = ctypes.c_double
_i = ctypes.c_int
_i64 = ctypes.c_int64
_p = ctypes.c_void_p


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    sig = {
        "or_set_threads": (None, [_i]),
        "or_get_threads": (_i, []),
        "or_dslash": (None, [_p, _p, _p, _i, _p, _p]),
        "or_dslash_sites": (None, [_p, _p, _p, _i, _p, _i64, _p, _p]),
        "or_mee": (None, [_p, _p, _p, _d, _d, _p, _p]),
        "or_mfull": (None, [_p, _p, _p, _d, _p, _p]),
        "or_half_pack": (_i64, [_i64, _p, _p]),
        "or_half_unpack": (None, [_i64, _p, _p]),
        "or_int20_pack": (_i64, [_i64, _p, _p]),
        "or_int20_unpack": (None, [_i64, _p, _p]),
        "or_int30_pack": (_i64, [_i64, _p, _p]),
        "or_int30_unpack": (None, [_i64, _p, _p]),
        "or_ru_trigger_first": (_i, [_i, _p, _p, _d]),
        "or_se15_pack": (_i64, [_i64, _i, _p, _p]),
        "or_se15_unpack": (None, [_i64, _i, _p, _p]),
        "or_int14_pack": (_i64, [_i64, _p, _p]),
        "or_int14_unpack": (None, [_i64, _p, _p]),
        "or_absmax": (_d, [_i64, _p]),
        "or_fix_pack": (None, [_i64, _p, _d, _i, _p]),
        "or_fix_unpack": (None, [_i64, _p, _d, _i, _i, _p]),
        "or_gauge_emulate": (None, [_p, _p, _i, _i, _i, _i, _i, _d, _p]),
        "or_spinor_emulate": (None, [_i64, _i, _p, _p]),
        "or_cg": (_i, [_p, _p, _p, _d, _d, _p, _p, _d, _i, _i, _p, _p]),
        "or_mixed_cg": (_i, [_p, _p, _p, _p, _p, _d, _i, _p, _p, _d, _d, _d, _i, _i, _i, _p, _p, _p, _p]),
        "or_mixed_bicgstabl": (_i, [_p, _p, _p, _p, _p, _d, _i, _i, _p, _p, _d, _d, _i, _p, _p, _p]),
        "or_mixed_multishift": (_i, [_p, _p, _p, _p, _p, _d, _i, _p, _p, _i, _d, _p, _p, _d, _i, _p, _p, _p, _p]),
        "or_multishift_cg": (_i, [_p, _p, _p, _d, _i, _p, _p, _p, _p, _i, _p, _p, _p]),
        "or_bicgstabl": (_i, [_p, _p, _p, _d, _i, _p, _p, _d, _i, _p, _p]),
        "or_dense": (None, [_p, _p, _p, _d, _d, _i, _p]),
        "or_schur_source": (None, [_p, _p, _p, _d, _p, _p]),
        "or_link_r8_pack": (None, [_i64, _p, _p, _p]),
        "or_link_r8_unpack": (None, [_i64, _p, _p, _p]),
        "or_reconstruct_odd": (None, [_p, _p, _p, _d, _p, _p, _p]),
        "or_solve_full": (_i, [_p, _p, _p, _d, _p, _p, _d, _i, _p, _p]),
        "or_lu_solve": (_i, [_i64, _p, _p]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


# ---------------------------------------------------------------------------
# marshalling
# ---------------------------------------------------------------------------
def _np(a, dtype=np.float64):
    if hasattr(a, "detach"):  # torch tensor
        a = a.detach().cpu().numpy()
    return np.ascontiguousarray(a, dtype=dtype)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _dims(dims):
    return np.ascontiguousarray([int(d) for d in dims], dtype=np.int32)


def vh_of(dims) -> int:
    return int(dims[0]) * int(dims[1]) * int(dims[2]) * int(dims[3]) // 2


def set_threads(n: int):
    _load().or_set_threads(int(n))


def get_threads() -> int:
    return int(_load().or_get_threads())


# ---------------------------------------------------------------------------
# stencil and operators
# ---------------------------------------------------------------------------
def dslash(dims, fat, lng, out_parity: int, x):
    """(D x) on the sites of ``out_parity``; ``x`` lives on the other parity."""
    L = _dims(dims)
    f, g, xin = _np(fat), _np(lng), _np(x)
    out = np.empty((vh_of(dims), 3, 2))
    _load().or_dslash(_ptr(L), _ptr(f), _ptr(g), int(out_parity), _ptr(xin), _ptr(out))
    return out


def dslash_sites(dims, fat, lng, out_parity: int, x, cbs):
    """The stencil at the output sites with checkerboard indices ``cbs`` only."""
    L = _dims(dims)
    f, g, xin = _np(fat), _np(lng), _np(x)
    c = np.ascontiguousarray(cbs, dtype=np.int64)
    out = np.empty((len(c), 3, 2))
    _load().or_dslash_sites(_ptr(L), _ptr(f), _ptr(g), int(out_parity), _ptr(xin), len(c), _ptr(c),
                            _ptr(out))
    return out


def mee(dims, fat, lng, m: float, x, sigma: float = 0.0):
    """(4m^2 + sigma) x - D_eo D_oe x on even sites."""
    L = _dims(dims)
    f, g, xin = _np(fat), _np(lng), _np(x)
    out = np.empty((vh_of(dims), 3, 2))
    _load().or_mee(_ptr(L), _ptr(f), _ptr(g), float(m), float(sigma), _ptr(xin), _ptr(out))
    return out


def mfull(dims, fat, lng, m: float, x):
    """(2m + D) x on the full lattice ``[2][Vh][3][2]``."""
    L = _dims(dims)
    f, g, xin = _np(fat), _np(lng), _np(x)
    out = np.empty((2, vh_of(dims), 3, 2))
    _load().or_mfull(_ptr(L), _ptr(f), _ptr(g), float(m), _ptr(xin), _ptr(out))
    return out


# ---------------------------------------------------------------------------
# storage formats
# ---------------------------------------------------------------------------
SFMT = {"f64": 0, "f32": 1, "half": 2, "int20": 3, "int30": 4, "int14": 5}
GFMT = {"f64": 0, "f32": 1, "fix16": 2, "fix32": 3, "se15": 4}


def half_pack(v):
    """FP32 [n][6] -> (records uint8 [n][16], number of non-finite sites)."""
    a = _np(v, np.float32).reshape(-1, 6)
    rec = np.zeros((a.shape[0], 16), dtype=np.uint8)
    bad = _load().or_half_pack(a.shape[0], _ptr(a), _ptr(rec))
    return rec, int(bad)


def half_unpack(rec):
    r = np.ascontiguousarray(rec, dtype=np.uint8).reshape(-1, 16)
    out = np.empty((r.shape[0], 6), dtype=np.float32)
    _load().or_half_unpack(r.shape[0], _ptr(r), _ptr(out))
    return out


def int20_pack(v):
    """FP32 [n][6] -> (words uint32 [n][4], number of non-finite sites)."""
    a = _np(v, np.float32).reshape(-1, 6)
    w = np.zeros((a.shape[0], 4), dtype=np.uint32)
    bad = _load().or_int20_pack(a.shape[0], _ptr(a), _ptr(w))
    return w, int(bad)


def int20_unpack(w):
    ww = np.ascontiguousarray(w, dtype=np.uint32).reshape(-1, 4)
    out = np.empty((ww.shape[0], 6), dtype=np.float32)
    _load().or_int20_unpack(ww.shape[0], _ptr(ww), _ptr(out))
    return out


def ru_trigger_first(r, alpha_ap, eps: float) -> int:
    """First step k at which the error-estimate trigger fires on |r_0..r_n| and |alpha_k| |A p_k|."""
    rr = _np(r).reshape(-1)
    aa = _np(alpha_ap).reshape(-1)
    assert len(aa) == len(rr) - 1
    return int(_load().or_ru_trigger_first(len(aa), _ptr(rr), _ptr(aa), float(eps)))


def se15_pack(links, nr: int = 18):
    """Links [n][nr] reals (FP64) -> (halves uint16 [n][nr], number of non-finite links)."""
    a = _np(links).reshape(-1, nr)
    h = np.zeros((a.shape[0], nr), dtype=np.uint16)
    bad = _load().or_se15_pack(a.shape[0], int(nr), _ptr(a), _ptr(h))
    return h, int(bad)


def se15_unpack(h, nr: int = 18):
    hh = np.ascontiguousarray(h, dtype=np.uint16).reshape(-1, nr)
    out = np.empty((hh.shape[0], nr), dtype=np.float64)
    _load().or_se15_unpack(hh.shape[0], int(nr), _ptr(hh), _ptr(out))
    return out


def int14_pack(v):
    """FP32 [n][6] -> (words uint32 [n][3], number of non-finite sites)."""
    a = _np(v, np.float32).reshape(-1, 6)
    w = np.zeros((a.shape[0], 3), dtype=np.uint32)
    bad = _load().or_int14_pack(a.shape[0], _ptr(a), _ptr(w))
    return w, int(bad)


def int14_unpack(w):
    ww = np.ascontiguousarray(w, dtype=np.uint32).reshape(-1, 3)
    out = np.empty((ww.shape[0], 6), dtype=np.float32)
    _load().or_int14_unpack(ww.shape[0], _ptr(ww), _ptr(out))
    return out


def int30_pack(v):
    """FP64 [n][6] -> (words uint32 [n][6], number of sites not encodable)."""
    a = _np(v).reshape(-1, 6)
    w = np.zeros((a.shape[0], 6), dtype=np.uint32)
    bad = _load().or_int30_pack(a.shape[0], _ptr(a), _ptr(w))
    return w, int(bad)


def int30_unpack(w):
    ww = np.ascontiguousarray(w, dtype=np.uint32).reshape(-1, 6)
    out = np.empty((ww.shape[0], 6), dtype=np.float64)
    _load().or_int30_unpack(ww.shape[0], _ptr(ww), _ptr(out))
    return out


def absmax(g) -> float:
    a = _np(g).reshape(-1)
    return float(_load().or_absmax(a.size, _ptr(a)))


def fix_pack(g, gmax: float, bits: int):
    a = _np(g).reshape(-1)
    q = np.empty(a.size, dtype=np.int32)
    _load().or_fix_pack(a.size, _ptr(a), float(gmax), int(bits), _ptr(q))
    return q


def fix_unpack(q, gmax: float, bits: int, compute_f32: bool):
    qq = np.ascontiguousarray(q, dtype=np.int32).reshape(-1)
    out = np.empty(qq.size)
    _load().or_fix_unpack(qq.size, _ptr(qq), float(gmax), int(bits), int(compute_f32), _ptr(out))
    return out


def gauge_emulate(dims, g, gfmt: str, recon: int, long_link: bool, antiperiodic_t: bool = False,
                  compute_f32: bool = True, gmax: float | None = None):
    """The link field as the computation sees it after storage in ``gfmt``/``recon``."""
    L = _dims(dims)
    a = _np(g)
    if gmax is None:
        gmax = absmax(a)
    out = np.empty_like(a)
    _load().or_gauge_emulate(_ptr(L), _ptr(a), GFMT[gfmt], int(recon), 3 if long_link else 1,
                             int(antiperiodic_t), int(compute_f32), float(gmax), _ptr(out))
    return out


def link_r8_pack(links, signs):
    """Links [n][3][3][2] (sign times SU(3)) and their signs -> the 8 reals of each ``V = sign * U``:
    (arg V00/pi, arg V20/pi, V01, V02, V10)."""
    a = _np(links).reshape(-1, 18)
    sg = _np(signs).reshape(-1)
    p = np.empty((a.shape[0], 8))
    _load().or_link_r8_pack(a.shape[0], _ptr(a), _ptr(sg), _ptr(p))
    return p


def link_r8_unpack(p, signs):
    """The 8 reals of each link (see link_r8_pack) -> links [n][3][3][2], rebuilt in FP64."""
    pp = _np(p).reshape(-1, 8)
    sg = _np(signs).reshape(-1)
    out = np.empty((pp.shape[0], 3, 3, 2))
    _load().or_link_r8_unpack(pp.shape[0], _ptr(pp), _ptr(sg), _ptr(out))
    return out


def spinor_emulate(x, sfmt: str):
    """Round-trip a spinor field through storage format ``sfmt``."""
    a = _np(x)
    out = np.empty_like(a)
    _load().or_spinor_emulate(a.size // 6, SFMT[sfmt], _ptr(a), _ptr(out))
    return out


# ---------------------------------------------------------------------------
# solvers
# ---------------------------------------------------------------------------
def cg(dims, fat, lng, m: float, b, tol: float, maxiter: int = 100000, sigma: float = 0.0, x0=None):
    """Textbook FP64 CG on (M_ee + sigma) x = b.  Returns (x, status, iters, true_res)."""
    L = _dims(dims)
    f, g, bb = _np(fat), _np(lng), _np(b)
    x = np.zeros_like(bb) if x0 is None else _np(x0).copy()
    it = ctypes.c_int(0)
    tr = ctypes.c_double(0.0)
    st = _load().or_cg(_ptr(L), _ptr(f), _ptr(g), float(m), float(sigma), _ptr(bb), _ptr(x), float(tol),
                       int(maxiter), int(x0 is not None), ctypes.byref(it), ctypes.byref(tr))
    return x, int(st), it.value, tr.value


def mixed_cg(dims, fat, lng, m: float, b, sfmt: str, tol: float, fat_s=None, lng_s=None, delta: float = 0.1,
             nbuf: int = 8, pr: bool = True, reproject: bool = True, maxiter: int = 100000, dyn_eps: float = 0.0):
    """Stabilised mixed-precision CG on M_ee x = b (Sec. 3.1) in FP64 with every sloppy vector write
    rounded through ``sfmt`` and the sloppy operator applied with (fat_s, lng_s) (default: the exact
    links); ``dyn_eps > 0`` replaces the delta trigger by the error-estimate trigger with that
    precision.  Returns (x, status, iters, reliable_updates, true_res, history of |r_k|/|b|, with the
    recomputed true residual at reliable updates)."""
    L = _dims(dims)
    f, g, bb = _np(fat), _np(lng), _np(b)
    fs = f if fat_s is None else _np(fat_s)
    gs = g if lng_s is None else _np(lng_s)
    x = np.zeros_like(bb)
    hist = np.zeros(int(maxiter) + 1)
    it, ru = ctypes.c_int(0), ctypes.c_int(0)
    tr = ctypes.c_double(0.0)
    opts = (1 if pr else 0) | (2 if reproject else 0)
    st = _load().or_mixed_cg(_ptr(L), _ptr(f), _ptr(g), _ptr(fs), _ptr(gs), float(m), SFMT[sfmt], _ptr(bb),
                             _ptr(x), float(tol), float(delta), float(dyn_eps), int(nbuf), opts, int(maxiter),
                             ctypes.byref(it),
                             ctypes.byref(ru), ctypes.byref(tr), _ptr(hist))
    return x, int(st), it.value, ru.value, tr.value, hist[: it.value + 1]


def schur_source(dims, fat, lng, m: float, b):
    """2m b_e - D_eo b_o: the even right-hand side of the reduced full system (b full-lattice)."""
    L = _dims(dims)
    f, g, bb = _np(fat), _np(lng), _np(b)
    out = np.empty((vh_of(dims), 3, 2))
    _load().or_schur_source(_ptr(L), _ptr(f), _ptr(g), float(m), _ptr(bb), _ptr(out))
    return out


def reconstruct_odd(dims, fat, lng, m: float, b_o, x_e):
    """x_o = (b_o - D_oe x_e) / (2m)."""
    L = _dims(dims)
    f, g, bo, xe = _np(fat), _np(lng), _np(b_o), _np(x_e)
    out = np.empty((vh_of(dims), 3, 2))
    _load().or_reconstruct_odd(_ptr(L), _ptr(f), _ptr(g), float(m), _ptr(bo), _ptr(xe), _ptr(out))
    return out


def solve_full(dims, fat, lng, m: float, b, tol: float, maxiter: int = 100000):
    """(2m + D) x = b on the full lattice by even/odd reduction, textbook CG and odd reconstruction.
    Returns (x [2][Vh][3][2], status, iters, true_res)."""
    L = _dims(dims)
    f, g, bb = _np(fat), _np(lng), _np(b)
    x = np.zeros_like(bb)
    it = ctypes.c_int(0)
    tr = ctypes.c_double(0.0)
    st = _load().or_solve_full(_ptr(L), _ptr(f), _ptr(g), float(m), _ptr(bb), _ptr(x), float(tol), int(maxiter),
                               ctypes.byref(it), ctypes.byref(tr))
    return x, int(st), it.value, tr.value


def multishift_cg(dims, fat, lng, m: float, sigmas, tols, b, maxiter: int = 100000):
    """FP64 multi-shift CG.  Returns (x [nshift][Vh][3][2], status, iters, zeta, r_base)."""
    L = _dims(dims)
    f, g, bb = _np(fat), _np(lng), _np(b)
    ns = len(sigmas)
    s = np.ascontiguousarray(sigmas, dtype=np.float64)
    t = np.ascontiguousarray(tols, dtype=np.float64)
    x = np.zeros((ns,) + bb.shape)
    its = np.zeros(ns, dtype=np.int32)
    z = np.zeros(ns)
    r = np.zeros_like(bb)
    st = _load().or_multishift_cg(_ptr(L), _ptr(f), _ptr(g), float(m), ns, _ptr(s), _ptr(t), _ptr(bb),
                                  _ptr(x), int(maxiter), _ptr(its), _ptr(z), _ptr(r))
    return x, int(st), its, z, r


# relative precision of each storage format (a shifted system's freezing floor is 10 times it)
EPS_FMT = {"f64": 0.0, "f32": 2.0 ** -24, "half": 2.0 ** -15, "int20": 2.0 ** -19, "int30": 2.0 ** -29,
           "int14": 2.0 ** -13}


def mixed_multishift(dims, fat, lng, m: float, sigmas, tols, b, sfmt: str, fat_s=None, lng_s=None,
                     delta: float = 0.1, maxiter: int = 100000):
    """The multi-shift stage with sloppy storage ``sfmt`` emulated (Sec. 3.2).  ``sigmas`` ascending.
    Returns (x [nshift][Vh][3][2], status, iters, reliable_updates, shift_iters, residuals after the stage)."""
    L = _dims(dims)
    f, g, bb = _np(fat), _np(lng), _np(b)
    fs = f if fat_s is None else _np(fat_s)
    gs = g if lng_s is None else _np(lng_s)
    ns = len(sigmas)
    s = np.ascontiguousarray(sigmas, dtype=np.float64)
    t = np.ascontiguousarray(tols, dtype=np.float64)
    x = np.zeros((ns,) + bb.shape)
    its = np.zeros(ns, dtype=np.int32)
    res = np.zeros(ns)
    it, ru = ctypes.c_int(0), ctypes.c_int(0)
    st = _load().or_mixed_multishift(_ptr(L), _ptr(f), _ptr(g), _ptr(fs), _ptr(gs), float(m), ns, _ptr(s),
                                     _ptr(t), SFMT[sfmt], EPS_FMT[sfmt], _ptr(bb), _ptr(x), float(delta),
                                     int(maxiter), ctypes.byref(it), ctypes.byref(ru), _ptr(its), _ptr(res))
    return x, int(st), it.value, ru.value, its, res


def bicgstabl(dims, fat, lng, m: float, b, l: int, tol: float, max_matvecs: int = 200000):
    """FP64 BiCGStab(l) on (2m + D) x = b.  Returns (x, status, matvecs, true_res)."""
    L = _dims(dims)
    f, g, bb = _np(fat), _np(lng), _np(b)
    x = np.zeros_like(bb)
    mv = ctypes.c_int(0)
    tr = ctypes.c_double(0.0)
    st = _load().or_bicgstabl(_ptr(L), _ptr(f), _ptr(g), float(m), int(l), _ptr(bb), _ptr(x), float(tol),
                              int(max_matvecs), ctypes.byref(mv), ctypes.byref(tr))
    return x, int(st), mv.value, tr.value


def mixed_bicgstabl(dims, fat, lng, m: float, b, l: int, sfmt: str, tol: float, fat_s=None, lng_s=None,
                    delta: float = 0.1, max_matvecs: int = 200000):
    """BiCGStab(l) on (2m + D) x = b with sloppy storage ``sfmt`` emulated and reliable updates at the end
    of a cycle (Sec. 6.1).  Returns (x, status, matvecs, reliable_updates, true_res)."""
    L = _dims(dims)
    f, g, bb = _np(fat), _np(lng), _np(b)
    fs = f if fat_s is None else _np(fat_s)
    gs = g if lng_s is None else _np(lng_s)
    x = np.zeros_like(bb)
    mv, ru = ctypes.c_int(0), ctypes.c_int(0)
    tr = ctypes.c_double(0.0)
    st = _load().or_mixed_bicgstabl(_ptr(L), _ptr(f), _ptr(g), _ptr(fs), _ptr(gs), float(m), int(l), SFMT[sfmt],
                                    _ptr(bb), _ptr(x), float(tol), float(delta), int(max_matvecs),
                                    ctypes.byref(mv), ctypes.byref(ru), ctypes.byref(tr))
    return x, int(st), mv.value, ru.value, tr.value


def dense(dims, fat, lng, which: str, m: float = 0.0, sigma: float = 0.0):
    """Dense complex matrix of 'mee', 'mfull', 'deo' or 'doe' (numpy complex128)."""
    code = {"mee": 0, "mfull": 1, "deo": 2, "doe": 3}[which]
    n = vh_of(dims) * 3 * (2 if which == "mfull" else 1)
    L = _dims(dims)
    f, g = _np(fat), _np(lng)
    a = np.zeros((n, n), dtype=np.complex128)  # row k = column k of the operator
    _load().or_dense(_ptr(L), _ptr(f), _ptr(g), float(m), float(sigma), code, _ptr(a))
    return np.ascontiguousarray(a.T)


def lu_solve(a, rhs):
    """Solve a y = rhs by the oracle's own partial-pivot LU (complex)."""
    n = a.shape[0]
    colmajor = np.ascontiguousarray(np.asarray(a, dtype=np.complex128).T)
    y = np.ascontiguousarray(np.asarray(rhs, dtype=np.complex128).reshape(-1)).copy()
    st = _load().or_lu_solve(n, _ptr(colmajor), _ptr(y))
    if st:
        raise ZeroDivisionError("singular matrix")
    return y

"""ctypes front-end of the C oracle (test infrastructure only).

Only the test-suite, the smoke check and the benchmark's CPU-baseline leg use
this module.  It builds `smolyak_oracle.c` with gcc on first use (or via
`build()`), and exposes:

  gauss_hermite(n)              Golub-Welsch Gauss-Hermite rule (Sec. 2, Eq. (6) weights)
  mode_tables(nb, nq, q0, s)    b_k(Q_u), b_k''(Q_u), w_u, Q_u for one mode/level
  enumerate_terms(D, L)         terms of R(l) in Table 2 order, with D_l (Eq. (8))
  enumerate_compact(...)        compact basis, lexicographic, first mode slowest (Table 2)
  counts(...)                   n_terms, N_s, N_cs (Table 1)
  term_map(...)                 mapping table M^B (Table 2)
  apply_H(problem, x, ...)      y = H_S x, Eq. (16), every term through its grid (Eqs. (14)-(15))
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "smolyak_oracle.c")
_LIBDIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIBDIR, "liborc.so")
_lock = threading.Lock()
_lib = None

_i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liborc.so (OpenMP if available)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:-3] + ["-fopenmp"] + base[-3:], check=True,
                       capture_output=True, text=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True, text=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        lib.orc_gauss_hermite.argtypes = [ctypes.c_int, _f64p, _f64p]
        lib.orc_mode_tables.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                        _f64p, _f64p, _f64p, _f64p]
        lib.orc_combination_coefficient.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
        lib.orc_combination_coefficient.restype = ctypes.c_int64
        lib.orc_enumerate_terms.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
        lib.orc_enumerate_terms.restype = ctypes.c_int64
        lib.orc_enumerate_compact.argtypes = [ctypes.c_int, ctypes.c_int, _i32p, _i32p, ctypes.c_void_p]
        lib.orc_enumerate_compact.restype = ctypes.c_int64
        lib.orc_counts.argtypes = [ctypes.c_int, ctypes.c_int, _i32p, _i32p,
                                   ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                                   ctypes.POINTER(ctypes.c_int64)]
        lib.orc_term_map.argtypes = [ctypes.c_int, ctypes.c_int, _i32p, _i32p, _i64p, _i64p]
        lib.orc_apply.argtypes = [ctypes.c_int, ctypes.c_int, _i32p, _i32p, _i32p, _i32p,
                                  _f64p, _f64p, _f64p,
                                  ctypes.c_int, _f64p, _i32p, _i32p, _i32p,
                                  _f64p, _f64p, ctypes.c_int,
                                  ctypes.c_void_p, ctypes.c_int64, ctypes.c_int]
        lib.orc_max_threads.restype = ctypes.c_int
        _lib = lib
        return lib


def _check(rc):
    if rc != 0:
        raise RuntimeError(f"oracle returned status {rc}")


def gauss_hermite(n: int):
    lib = _load()
    x = np.zeros(n); w = np.zeros(n)
    _check(lib.orc_gauss_hermite(n, x, w))
    return x, w


def mode_tables(nb: int, nq: int, q0: float = 0.0, scale: float = 1.0):
    """Returns (B[nq,nb], D2[nq,nb], W[nq], Q[nq])."""
    lib = _load()
    B = np.zeros(nq * nb); D2 = np.zeros(nq * nb); W = np.zeros(nq); Q = np.zeros(nq)
    _check(lib.orc_mode_tables(nb, nq, q0, scale, B, D2, W, Q))
    return B.reshape(nq, nb), D2.reshape(nq, nb), W, Q


def combination_coefficient(D: int, L: int, sum_l: int) -> int:
    return int(_load().orc_combination_coefficient(D, L, sum_l))


def enumerate_terms(D: int, L: int):
    """(levels[n_terms, D] int32, coef[n_terms] int64), Table 2 order."""
    lib = _load()
    n = lib.orc_enumerate_terms(D, L, None, None)
    lv = np.zeros((n, D), np.int32); c = np.zeros(n, np.int64)
    lib.orc_enumerate_terms(D, L, lv.ctypes.data, c.ctypes.data)
    return lv, c


def _rule(v, D):
    return np.ascontiguousarray(np.broadcast_to(np.asarray(v, np.int32), (D,)))


def enumerate_compact(D: int, L: int, nb_A=1, nb_B=1):
    lib = _load()
    a, b = _rule(nb_A, D), _rule(nb_B, D)
    n = lib.orc_enumerate_compact(D, L, a, b, None)
    k = np.zeros((n, D), np.int32)
    lib.orc_enumerate_compact(D, L, a, b, k.ctypes.data)
    return k


def counts(D: int, L: int, nb_A=1, nb_B=1):
    """(n_terms, N_s, N_cs) by generating functions (valid for any D)."""
    lib = _load()
    nt, ns, nc = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(lib.orc_counts(D, L, _rule(nb_A, D), _rule(nb_B, D),
                          ctypes.byref(nt), ctypes.byref(ns), ctypes.byref(nc)))
    return nt.value, ns.value, nc.value


def term_map(D: int, L: int, nb_A=1, nb_B=1):
    """(term_offsets[n_terms+1], cs_index[N_s]) -- M^B of Table 2, 0-based."""
    lib = _load()
    nt, ns, _ = counts(D, L, nb_A, nb_B)
    off = np.zeros(nt + 1, np.int64); cs = np.zeros(ns, np.int64)
    _check(lib.orc_term_map(D, L, _rule(nb_A, D), _rule(nb_B, D), off, cs))
    return off, cs


def n_compact(p) -> int:
    return counts(p.D, p.L, p.nb_A, p.nb_B)[2]


def apply_H(p, x: np.ndarray, term_subset=None, threads: int = 0) -> np.ndarray:
    """y = H_S x by Eq. (16) over all terms (or a subset of term
    indices in Table 2 order).  x: (nvec, N_cs) or (N_cs,) float64."""
    lib = _load()
    x = np.ascontiguousarray(np.asarray(x, np.float64))
    squeeze = x.ndim == 1
    X = x.reshape(1, -1) if squeeze else x
    nvec, ncs = X.shape
    y = np.zeros_like(X)
    sub = None
    nsub = 0
    if term_subset is not None:
        sub = np.ascontiguousarray(np.asarray(term_subset, np.int64))
        nsub = sub.shape[0]
    i32 = lambda a: np.ascontiguousarray(np.asarray(a, np.int32))
    f64 = lambda a: np.ascontiguousarray(np.asarray(a, np.float64))
    coef = f64(p.coef) if p.nmono else np.zeros(1)
    nfac = i32(p.nfac) if p.nmono else np.zeros(1, np.int32)
    fmode = i32(p.fmode) if len(p.fmode) else np.zeros(1, np.int32)
    fpow = i32(p.fpow) if len(p.fpow) else np.zeros(1, np.int32)
    rc = lib.orc_apply(p.D, p.L, i32(p.nb_A), i32(p.nb_B), i32(p.nq_A), i32(p.nq_B),
                       f64(p.q0), f64(p.scale), f64(p.omega),
                       p.nmono, coef, nfac, fmode, fpow,
                       X, y, nvec,
                       None if sub is None else sub.ctypes.data, nsub, int(threads))
    _check(rc)
    return y.reshape(-1) if squeeze else y


def max_threads() -> int:
    return int(_load().orc_max_threads())

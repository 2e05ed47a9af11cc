"""GB300 Smolyak operator action (arXiv 2111.13655) -- Python binding.

A thin ctypes layer over libsmolyak.so (include/smolyak.h): every function has
the C name and only marshals arguments; all arithmetic of the operator action
runs in the library's CUDA kernels.  Device buffers are torch CUDA tensors
(float64, contiguous); streams are torch.cuda.Stream objects or None (the
current torch stream).

If the library has not been built, every call raises: there is no CPU path.
Build it with `python -m paper_2111_13655_gb300.build`.

Typical use (problems come from paper_2111_13655_gb300.synth or any Problem
with the same fields):

    import torch, paper_2111_13655_gb300 as sg
    from paper_2111_13655_gb300 import synth
    p = synth.workload_C3()                      # D=12 L=10 chained Henon-Heiles
    with sg.sg_create(p, "mixed") as ctx:        # or "fp64"
        x = torch.randn(8 * ctx.n_cs, dtype=torch.float64, device="cuda")
        y = torch.empty_like(x)
        sg.sg_apply_H(ctx, x, y, 8)              # y = H_S x for 8 vectors
        ev, res, vec, ok = sg.sg_eigs(ctx, 20, "davidson", block=8, tol=1e-3, vectors=True)
    with sg.sg_create(p, "fp64") as c64:         # FP64 refinement of the mixed eigenpairs
        ev, res, ok = sg.sg_eigs_refine(c64, vec.view(-1), tol=1e-9)

Many problems per apply: sg_batch_create / sg_apply_H_batch.  Propagation:
sg_propagate on one context, or Server (continuous batching of requests).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libsmolyak.so")

SG_OK, SG_EINVAL, SG_ENOMEM, SG_ECUDA, SG_ENOCONV, SG_ETIMEOUT, SG_EBUDGET, SG_EUNSUPPORTED = range(8)
SG_FP64, SG_MIXED, SG_DF64 = 0, 1, 2
SG_LANCZOS, SG_DAVIDSON = 0, 1
_STATUS = {0: "SG_OK", 1: "SG_EINVAL", 2: "SG_ENOMEM", 3: "SG_ECUDA", 4: "SG_ENOCONV",
           5: "SG_ETIMEOUT", 6: "SG_EBUDGET", 7: "SG_EUNSUPPORTED"}


class SgError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class _Basis(ctypes.Structure):
    _fields_ = [("nb_A", ctypes.c_int), ("nb_B", ctypes.c_int),
                ("q0", ctypes.c_double), ("scale", ctypes.c_double)]


class _Grid(ctypes.Structure):
    _fields_ = [("nq_A", ctypes.c_int), ("nq_B", ctypes.c_int)]


class _Poly(ctypes.Structure):
    _fields_ = [("nterms", ctypes.c_int), ("coef", ctypes.c_void_p), ("nfac", ctypes.c_void_p),
                ("mode", ctypes.c_void_p), ("power", ctypes.c_void_p)]


class _Ham(ctypes.Structure):
    _fields_ = [("omega", ctypes.c_void_p), ("V", _Poly)]


class _PropRequest(ctypes.Structure):
    _fields_ = [("D", ctypes.c_int), ("L", ctypes.c_int), ("basis", ctypes.c_void_p), ("grids", ctypes.c_void_p),
                ("H", ctypes.c_void_p), ("psi0", ctypes.c_void_p), ("factors", ctypes.c_void_p),
                ("ld", ctypes.c_int), ("dt", ctypes.c_double), ("nsteps", ctypes.c_int), ("order", ctypes.c_int)]


class _EigRequest(ctypes.Structure):
    _fields_ = [("D", ctypes.c_int), ("L", ctypes.c_int), ("basis", ctypes.c_void_p), ("grids", ctypes.c_void_p),
                ("H", ctypes.c_void_p), ("nev", ctypes.c_int), ("block", ctypes.c_int), ("tol", ctypes.c_double),
                ("max_it", ctypes.c_int), ("want_vectors", ctypes.c_int)]


_lib = None
_lock = threading.Lock()
_vp, _i64, _i32, _dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
_P64 = ctypes.POINTER(ctypes.c_int64)

# name -> (restype, argtypes): every entry point declared in include/smolyak.h
SIGNATURES = {
    "sg_create": (_i32, [_i32, _i32, _vp, _vp, _vp, _i32, ctypes.POINTER(_vp)]),
    "sg_plan": (_i32, [_i32, _i32, _vp, _vp, _vp, _i32, ctypes.POINTER(_vp)]),
    "sg_size": (_i32, [_vp, _P64, _P64, _P64, _P64, _P64]),
    "sg_apply_H": (_i32, [_vp, _vp, _vp, _i32, _vp]),
    "sg_apply_H_host": (_i32, [_vp, _vp, _vp, _i32, _vp]),
    "sg_apply_H_noalloc": (_i32, [_vp, _vp, _vp, _i32, _vp]),
    "sg_apply_H_part": (_i32, [_vp, _vp, _i32, _i32, _i32, _vp, _vp]),
    "sg_apply_H_finish": (_i32, [_vp, _vp, _vp, _vp, _i32, _vp]),
    "sg_part_size": (_i32, [_vp, _i32, _i32, _P64, _P64]),
    "sg_term_levels": (_i32, [_vp, _i64, _i64, _vp, _vp]),
    "sg_index_map": (_i32, [_vp, _i64, _i64, _vp, _vp, _vp]),
    "sg_compact_rank": (_i32, [_vp, _vp, _i64, _vp]),
    "sg_mode_tables": (_i32, [_vp, _i32, _i32, ctypes.POINTER(_i32), ctypes.POINTER(_i32),
                              _vp, _vp, _vp, _vp]),
    "sg_device_error": (_i32, [_vp, ctypes.POINTER(_i32)]),
    "sg_eigs": (_i32, [_vp, _i32, _i32, _i32, _dbl, _i32, _vp, _vp, _vp, _vp]),
    "sg_eigs_refine": (_i32, [_vp, _i32, _vp, _vp, _vp, _dbl, _i32, _vp]),
    "sg_propagate": (_i32, [_vp, _vp, _dbl, _i32, _i32, _vp, _vp, _vp]),
    "sg_product_state": (_i32, [_vp, _vp, _i32, _vp]),
    "sg_last_error": (ctypes.c_char_p, [_vp]),
    "sg_batch_create": (_i32, [_vp, _i32, ctypes.POINTER(_vp)]),
    "sg_batch_size": (_i32, [_vp, _P64, _P64, ctypes.POINTER(_i32)]),
    "sg_apply_H_batch": (_i32, [_vp, _vp, _vp, _i32, _vp]),
    "sg_batch_last_error": (ctypes.c_char_p, [_vp]),
    "sg_batch_destroy": (None, [_vp]),
    "sg_tune": (_i32, [_vp, _i32, ctypes.POINTER(_i32), ctypes.POINTER(_dbl), _vp]),
    "sg_tune_plan": (_i32, [_vp, ctypes.POINTER(_i32), ctypes.POINTER(_i32), ctypes.POINTER(_i32)]),
    "sg_server_create": (_i32, [_i32, _i64, ctypes.POINTER(_vp)]),
    "sg_server_submit": (_i32, [_vp, _vp, _P64]),
    "sg_server_submit_eigs": (_i32, [_vp, _vp, _P64]),
    "sg_server_progress": (_i32, [_vp, _i32, ctypes.POINTER(_i32), ctypes.POINTER(_i32)]),
    "sg_server_query": (_i32, [_vp, _i64, ctypes.POINTER(_i32), _P64, ctypes.POINTER(_i32)]),
    "sg_server_result": (_i32, [_vp, _i64, _vp, _vp, _vp, _vp]),
    "sg_server_eig_result": (_i32, [_vp, _i64, _vp, _vp, _vp, _vp, ctypes.POINTER(_i32)]),
    "sg_server_stats": (_i32, [_vp, _P64, _P64, _P64]),
    "sg_server_last_error": (ctypes.c_char_p, [_vp]),
    "sg_server_destroy": (None, [_vp]),
    "sg_measure_peak": (_i32, [_i32, _dbl, ctypes.POINTER(_dbl), ctypes.POINTER(_i32), _vp]),
    "sg_destroy": (None, [_vp]),
}


def lib():
    """Load libsmolyak.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                                   "`python -m paper_2111_13655_gb300.build` (there is no CPU fallback)")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
        return _lib


def _check(st: int, ctx=None):
    if st != SG_OK:
        msg = lib().sg_last_error(ctx.ptr if ctx is not None else None)
        raise SgError(st, (msg or b"").decode(errors="replace"))


def _stream_ptr(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Ctx:
    """Owner of one sg_ctx* (release with sg_destroy or a `with` block)."""

    def __init__(self, ptr: int, problem, precision: int, device: bool):
        self.ptr = ptr
        self.problem = problem
        self.precision = precision
        self.device = device
        n = sg_size(self)
        self.n_cs, self.n_terms, self.n_s, self.n_grid = n["n_cs"], n["n_terms"], n["n_s"], n["n_grid"]

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        sg_destroy(self)

    def __del__(self):
        try:
            sg_destroy(self)
        except Exception:
            pass


def _marshal(p):
    D = p.D
    basis = (_Basis * D)(*[_Basis(int(p.nb_A[i]), int(p.nb_B[i]), float(p.q0[i]), float(p.scale[i]))
                           for i in range(D)])
    grids = (_Grid * D)(*[_Grid(int(p.nq_A[i]), int(p.nq_B[i])) for i in range(D)])
    keep = [np.ascontiguousarray(p.omega, np.float64), np.ascontiguousarray(p.coef, np.float64),
            np.ascontiguousarray(p.nfac, np.int32), np.ascontiguousarray(p.fmode, np.int32),
            np.ascontiguousarray(p.fpow, np.int32)]
    poly = _Poly(int(p.nmono), keep[1].ctypes.data, keep[2].ctypes.data,
                 keep[3].ctypes.data if keep[3].size else None,
                 keep[4].ctypes.data if keep[4].size else None)
    ham = _Ham(keep[0].ctypes.data, poly)
    return basis, grids, ham, keep


def _precision(precision) -> int:
    if precision in (SG_FP64, "fp64", "FP64"):
        return SG_FP64
    if precision in (SG_MIXED, "mixed", "MIXED", "fp32"):
        return SG_MIXED
    if precision in (SG_DF64, "df64", "DF64"):
        return SG_DF64
    raise ValueError(f"unknown precision {precision!r}")


def sg_create(problem, precision="fp64") -> Ctx:
    """Context on the current CUDA device for a synth.Problem."""
    prec = _precision(precision)
    basis, grids, ham, keep = _marshal(problem)
    out = _vp()
    _check(lib().sg_create(problem.D, problem.L, ctypes.addressof(basis), ctypes.addressof(grids),
                           ctypes.addressof(ham), prec, ctypes.byref(out)))
    return Ctx(out.value, problem, prec, True)


def sg_plan(problem, precision="fp64") -> Ctx:
    """Host-only context (no GPU needed): sizes, terms, ranking, 1D tables."""
    prec = _precision(precision)
    basis, grids, ham, keep = _marshal(problem)
    out = _vp()
    _check(lib().sg_plan(problem.D, problem.L, ctypes.addressof(basis), ctypes.addressof(grids),
                         ctypes.addressof(ham), prec, ctypes.byref(out)))
    return Ctx(out.value, problem, prec, False)


def sg_size(ctx: Ctx) -> dict:
    v = [ctypes.c_int64() for _ in range(5)]
    _check(lib().sg_size(ctx.ptr, *[ctypes.byref(a) for a in v]), ctx)
    return dict(zip(["n_cs", "n_terms", "n_s", "n_grid", "bytes_device"], [a.value for a in v]))


def _dev_ptr(t, n_expected: int, name: str):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous float64 CUDA tensor")
    if t.numel() != n_expected:
        raise ValueError(f"{name} has {t.numel()} elements, expected {n_expected}")
    # the library requires the context's device to be current: a tensor on
    # another GPU would hand its kernels a foreign pointer
    cur = torch.cuda.current_device()
    if t.device.index != cur:
        raise ValueError(f"{name} is on cuda:{t.device.index}, the current device is cuda:{cur}")
    return t.data_ptr()


def sg_apply_H(ctx: Ctx, x, y, nvec: int = None, stream=None) -> None:
    """y = H_S x on the device (x, y: float64 CUDA tensors with nvec*N_cs elements)."""
    if nvec is None:
        nvec = x.numel() // ctx.n_cs
    xp = _dev_ptr(x, nvec * ctx.n_cs, "x")
    yp = _dev_ptr(y, nvec * ctx.n_cs, "y")
    _check(lib().sg_apply_H(ctx.ptr, xp, yp, int(nvec), _stream_ptr(stream)), ctx)


def sg_apply_H_noalloc(ctx: Ctx, x, y, nvec: int = None, stream=None) -> None:
    """y = H_S x like sg_apply_H, for callers that may not allocate device
    memory at this point: the apply's scratch comes from a fixed 16 MiB array
    in the library (nvec <= 64, nvec * N_cs <= 524272).  Calls that overlap on
    the GPU share that array and race."""
    if nvec is None:
        nvec = x.numel() // ctx.n_cs
    xp = _dev_ptr(x, nvec * ctx.n_cs, "x")
    yp = _dev_ptr(y, nvec * ctx.n_cs, "y")
    _check(lib().sg_apply_H_noalloc(ctx.ptr, xp, yp, int(nvec), _stream_ptr(stream)), ctx)


def acc_words(ctx: Ctx, nvec: int) -> int:
    """int64 words of the fixed-point accumulators of nvec vectors (sg_apply_H_part)."""
    return ctx.n_cs * nvec * (1 if ctx.precision == SG_MIXED else 4)


def _acc_ptr(acc, n_expected: int):
    import torch
    if not isinstance(acc, torch.Tensor) or not acc.is_cuda or acc.dtype != torch.int64 or not acc.is_contiguous():
        raise TypeError("acc must be a contiguous int64 CUDA tensor")
    if acc.numel() != n_expected:
        raise ValueError(f"acc has {acc.numel()} elements, expected {n_expected}")
    return acc.data_ptr()


def sg_apply_H_part(ctx: Ctx, x, acc, nvec: int, part: int, nparts: int, stream=None) -> None:
    """Adds the contributions of the terms at processing positions p = part
    (mod nparts) into the int64 accumulators acc (device, acc_words(ctx, nvec))."""
    xp = _dev_ptr(x, nvec * ctx.n_cs, "x")
    _check(lib().sg_apply_H_part(ctx.ptr, xp, int(nvec), int(part), int(nparts),
                                 _acc_ptr(acc, acc_words(ctx, nvec)), _stream_ptr(stream)), ctx)


def sg_apply_H_finish(ctx: Ctx, x, acc, y, nvec: int, stream=None) -> None:
    """y = H_S x from the accumulators summed over all parts; clears acc."""
    xp = _dev_ptr(x, nvec * ctx.n_cs, "x")
    yp = _dev_ptr(y, nvec * ctx.n_cs, "y")
    _check(lib().sg_apply_H_finish(ctx.ptr, xp, _acc_ptr(acc, acc_words(ctx, nvec)), yp, int(nvec),
                                   _stream_ptr(stream)), ctx)


def sg_part_size(ctx: Ctx, part: int, nparts: int):
    """(terms, summed cost estimate) of one part of a term-sharded apply (host)."""
    a, b = ctypes.c_int64(), ctypes.c_int64()
    _check(lib().sg_part_size(ctx.ptr, int(part), int(nparts), ctypes.byref(a), ctypes.byref(b)), ctx)
    return a.value, b.value


def sg_apply_H_host(ctx: Ctx, x_host, y_host, nvec: int = None, stream=None) -> None:
    """Host-buffer form: copies in, applies, copies out; returns when y_host is written.
    x_host, y_host: contiguous float64 numpy arrays or pinned CPU torch tensors."""
    def ptr(a):
        if isinstance(a, np.ndarray):
            if a.dtype != np.float64 or not a.flags.c_contiguous:
                raise TypeError("host buffers must be contiguous float64")
            return a.ctypes.data, a.size
        if a.dtype.is_floating_point and a.dtype.itemsize == 8 and not a.is_cuda and a.is_contiguous():
            return a.data_ptr(), a.numel()
        raise TypeError("host buffers must be contiguous float64")
    xp, nx = ptr(x_host)
    yp, ny = ptr(y_host)
    if nvec is None:
        nvec = nx // ctx.n_cs
    if nx != nvec * ctx.n_cs or ny != nx:
        raise ValueError("host buffer sizes do not match nvec * N_cs")
    _check(lib().sg_apply_H_host(ctx.ptr, xp, yp, int(nvec), _stream_ptr(stream)), ctx)


def sg_term_levels(ctx: Ctx, t0: int = 0, nt: int = None):
    """(levels[nt, D] int32, coef[nt] int32) of terms [t0, t0+nt) in Table-2 order."""
    if nt is None:
        nt = ctx.n_terms - t0
    lv = np.zeros((nt, ctx.problem.D), np.int32)
    c = np.zeros(nt, np.int32)
    _check(lib().sg_term_levels(ctx.ptr, t0, nt, lv.ctypes.data, c.ctypes.data), ctx)
    return lv, c


def sg_index_map(ctx: Ctx, t0: int = 0, nt: int = None, stream=None):
    """(offsets[nt+1] int64 numpy, cs_index int64 CUDA tensor): M^B of Table 2."""
    import torch
    if nt is None:
        nt = ctx.n_terms - t0
    off = np.zeros(nt + 1, np.int64)
    _check(lib().sg_index_map(ctx.ptr, t0, nt, off.ctypes.data, None, None), ctx)
    out = torch.empty(int(off[-1]), dtype=torch.int64, device="cuda")
    _check(lib().sg_index_map(ctx.ptr, t0, nt, off.ctypes.data,
                              out.data_ptr() if out.numel() else None, _stream_ptr(stream)), ctx)
    return off, out


def sg_compact_rank(ctx: Ctx, k) -> np.ndarray:
    k = np.ascontiguousarray(np.asarray(k, np.int32).reshape(-1, ctx.problem.D))
    r = np.zeros(k.shape[0], np.int64)
    _check(lib().sg_compact_rank(ctx.ptr, k.ctypes.data, k.shape[0], r.ctypes.data), ctx)
    return r


def sg_mode_tables(ctx: Ctx, mode: int, level: int) -> dict:
    nb, nq = ctypes.c_int(), ctypes.c_int()
    _check(lib().sg_mode_tables(ctx.ptr, mode, level, ctypes.byref(nb), ctypes.byref(nq),
                                None, None, None, None), ctx)
    nb, nq = nb.value, nq.value
    B = np.zeros((nq, nb)); BW = np.zeros((nb, nq)); K = np.zeros((nb, nb)); Q = np.zeros(nq)
    _check(lib().sg_mode_tables(ctx.ptr, mode, level, None, None, B.ctypes.data, BW.ctypes.data,
                                K.ctypes.data, Q.ctypes.data), ctx)
    return {"nb": nb, "nq": nq, "B": B, "BW": BW, "K": K, "Q": Q}


def sg_device_error(ctx: Ctx) -> int:
    c = ctypes.c_int()
    _check(lib().sg_device_error(ctx.ptr, ctypes.byref(c)), ctx)
    return c.value


def sg_eigs(ctx: Ctx, nev: int, method="davidson", block: int = 0, tol: float = 1e-8, max_it: int = 200,
            vectors: bool = False, stream=None):
    """Lowest nev eigenpairs.  Returns (evals, resid, evecs or None, converged)."""
    import torch
    m = {"lanczos": SG_LANCZOS, "davidson": SG_DAVIDSON}.get(method, method)
    ev = np.zeros(nev); rs = np.zeros(nev)
    vec = torch.empty(nev * ctx.n_cs, dtype=torch.float64, device="cuda") if vectors else None
    st = lib().sg_eigs(ctx.ptr, nev, int(m), block, tol, max_it, ev.ctypes.data,
                       vec.data_ptr() if vec is not None else None, rs.ctypes.data, _stream_ptr(stream))
    if st not in (SG_OK, SG_ENOCONV):
        _check(st, ctx)
    return ev, rs, (vec.view(nev, ctx.n_cs) if vec is not None else None), st == SG_OK


def sg_eigs_refine(ctx: Ctx, evecs, tol: float = 1e-10, max_it: int = 100, stream=None):
    """Refine nev eigenpairs from the given device vectors (nev x N_cs, in/out).
    Returns (evals, resid, converged)."""
    nev = evecs.numel() // ctx.n_cs
    _dev_ptr(evecs, nev * ctx.n_cs, "evecs")
    ev = np.zeros(nev); rs = np.zeros(nev)
    st = lib().sg_eigs_refine(ctx.ptr, nev, evecs.data_ptr(), ev.ctypes.data, rs.ctypes.data, tol, max_it,
                              _stream_ptr(stream))
    if st not in (SG_OK, SG_ENOCONV):
        _check(st, ctx)
    return ev, rs, st == SG_OK


def sg_propagate(ctx: Ctx, psi, dt: float, nsteps: int, order: int = 64, stream=None):
    """Chebyshev propagation of psi (device, 2*N_cs: real part then imaginary
    part, in place).  Returns (norm_log, energy_log) at the start of each step."""
    _dev_ptr(psi, 2 * ctx.n_cs, "psi")
    nl = np.zeros(max(nsteps, 1)); el = np.zeros(max(nsteps, 1))
    _check(lib().sg_propagate(ctx.ptr, psi.data_ptr(), dt, nsteps, order, nl.ctypes.data, el.ctypes.data,
                              _stream_ptr(stream)), ctx)
    return nl[:nsteps], el[:nsteps]


def sg_tune(ctx: Ctx, nvec: int = 8, stream=None):
    """Measured choice of the fast path's plan (slicing target, block/warp
    split, shared-memory budget per block) for nvec-vector applies; returns
    (slicing target kept, ms per apply).  sg_tune_plan reports the whole plan."""
    vt, ms = ctypes.c_int(), ctypes.c_double()
    _check(lib().sg_tune(ctx.ptr, int(nvec), ctypes.byref(vt), ctypes.byref(ms), _stream_ptr(stream)), ctx)
    return vt.value, ms.value


def sg_tune_plan(ctx: Ctx) -> dict:
    """The plan the context uses now: slicing target, block/warp split, KB per block."""
    a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib().sg_tune_plan(ctx.ptr, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), ctx)
    return {"slice_vt": a.value, "warp_vt": b.value, "smem_kb": c.value}


def sg_product_state(ctx: Ctx, factors) -> np.ndarray:
    """psi_k = prod_i factors[i][k_i] over the compact basis (host array)."""
    f = np.ascontiguousarray(np.asarray(factors, np.float64))
    out = np.zeros(ctx.n_cs)
    _check(lib().sg_product_state(ctx.ptr, f.ctypes.data, f.shape[1], out.ctypes.data), ctx)
    return out


class Batch:
    """Owner of one sg_batch* over several contexts (kept alive by this object).
    Vectors of problem j start at nvec * offsets[j] in the batched buffers."""

    def __init__(self, ptr: int, ctxs):
        self.ptr = ptr
        self.ctxs = list(ctxs)
        a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int()
        _check(lib().sg_batch_size(ptr, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        self.n_cs_total, self.n_terms_total, self.launches_per_apply = a.value, b.value, c.value
        self.offsets = np.concatenate([[0], np.cumsum([c.n_cs for c in self.ctxs])]).astype(np.int64)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        sg_batch_destroy(self)

    def __del__(self):
        try:
            sg_batch_destroy(self)
        except Exception:
            pass


def sg_batch_create(ctxs) -> Batch:
    """One batched operator over contexts of one device and precision."""
    arr = (_vp * len(ctxs))(*[c.ptr for c in ctxs])
    out = _vp()
    st = lib().sg_batch_create(arr, len(ctxs), ctypes.byref(out))
    if st != SG_OK:
        raise SgError(st, "sg_batch_create: contexts must be device contexts of the current device and one "
                          "precision, 1..65535 of them")
    return Batch(out.value, ctxs)


def sg_apply_H_batch(b: Batch, x, y, nvec: int, stream=None) -> None:
    """y_j = H_j x_j for every problem j (device float64 tensors of nvec * sum N_cs
    elements, problem after problem)."""
    xp = _dev_ptr(x, nvec * b.n_cs_total, "x")
    yp = _dev_ptr(y, nvec * b.n_cs_total, "y")
    st = lib().sg_apply_H_batch(b.ptr, xp, yp, int(nvec), _stream_ptr(stream))
    if st != SG_OK:
        raise SgError(st, (lib().sg_batch_last_error(b.ptr) or b"").decode(errors="replace"))


def sg_batch_destroy(b: Batch) -> None:
    if b is not None and getattr(b, "ptr", None):
        lib().sg_batch_destroy(b.ptr)
        b.ptr = None


SG_REQ_QUEUED, SG_REQ_ACTIVE, SG_REQ_DONE, SG_REQ_FAILED = range(4)


class Server:
    """Request server on the current CUDA device (continuous batching of
    Chebyshev propagation requests and block-Davidson eigen requests; see
    sg_server_* in include/smolyak.h)."""

    def __init__(self, precision="fp64", hbm_budget_bytes: int = 150 * 10**9):
        out = _vp()
        st = lib().sg_server_create(_precision(precision), int(hbm_budget_bytes), ctypes.byref(out))
        if st != SG_OK:
            raise SgError(st, "sg_server_create failed")
        self.ptr = out.value
        self.nsteps = {}
        self.n_cs = {}
        self.nev = {}

    def _err(self, st):
        if st != SG_OK:
            raise SgError(st, (lib().sg_server_last_error(self.ptr) or b"").decode(errors="replace"))

    def submit(self, problem, dt: float, nsteps: int, order: int = 64, psi0=None, factors=None) -> int:
        """Queue a propagation of psi0 (complex, N_cs, or a (2, N_cs) real/imaginary
        array) or of the real product state of `factors` (D x ld)."""
        basis, grids, ham, keep = _marshal(problem)
        req = _PropRequest(problem.D, problem.L, ctypes.addressof(basis), ctypes.addressof(grids),
                           ctypes.addressof(ham), None, None, 0, float(dt), int(nsteps), int(order))
        if psi0 is not None:
            a = np.asarray(psi0)
            a = np.concatenate([a.real, a.imag]) if np.iscomplexobj(a) else a.reshape(-1)
            a = np.ascontiguousarray(a, np.float64)
            keep.append(a)
            req.psi0 = a.ctypes.data
        else:
            f = np.ascontiguousarray(np.asarray(factors, np.float64))
            keep.append(f)
            req.factors, req.ld = f.ctypes.data, f.shape[1]
        rid = ctypes.c_int64()
        self._err(lib().sg_server_submit(self.ptr, ctypes.byref(req), ctypes.byref(rid)))
        st, n, _ = self.query(rid.value)
        self.nsteps[rid.value], self.n_cs[rid.value] = int(nsteps), n
        return rid.value

    def submit_eigs(self, problem, nev: int, block: int = 0, tol: float = 1e-8, max_it: int = 200,
                    vectors: bool = False) -> int:
        """Queue the nev lowest eigenpairs of the problem's H_S (block Davidson)."""
        basis, grids, ham, keep = _marshal(problem)
        req = _EigRequest(problem.D, problem.L, ctypes.addressof(basis), ctypes.addressof(grids),
                          ctypes.addressof(ham), int(nev), int(block), float(tol), int(max_it), int(bool(vectors)))
        rid = ctypes.c_int64()
        self._err(lib().sg_server_submit_eigs(self.ptr, ctypes.byref(req), ctypes.byref(rid)))
        st, n, _ = self.query(rid.value)
        self.n_cs[rid.value], self.nev[rid.value] = n, int(nev)
        self.nsteps[rid.value] = 0
        return rid.value

    def eig_result(self, rid: int, vectors: bool = False):
        """(evals, resid, evecs (nev x N_cs) or None, (queue_s, latency_s), converged pairs)."""
        n, nev = self.n_cs[rid], self.nev[rid]
        ev, rs, tm = np.zeros(nev), np.zeros(nev), np.zeros(2)
        vec = np.zeros((nev, n)) if vectors else None
        conv = ctypes.c_int()
        st = lib().sg_server_eig_result(self.ptr, int(rid), ev.ctypes.data, rs.ctypes.data,
                                        vec.ctypes.data if vec is not None else None, tm.ctypes.data,
                                        ctypes.byref(conv))
        if st not in (SG_OK, SG_ENOCONV):
            self._err(st)
        return ev, rs, vec, (float(tm[0]), float(tm[1])), conv.value

    def progress(self, max_iters: int = 1):
        """Runs up to max_iters engine iterations; returns (active, queued)."""
        a, q = ctypes.c_int(), ctypes.c_int()
        self._err(lib().sg_server_progress(self.ptr, int(max_iters), ctypes.byref(a), ctypes.byref(q)))
        return a.value, q.value

    def query(self, rid: int):
        """(state, N_cs, steps done) of a request."""
        st, n, k = ctypes.c_int(), ctypes.c_int64(), ctypes.c_int()
        self._err(lib().sg_server_query(self.ptr, int(rid), ctypes.byref(st), ctypes.byref(n), ctypes.byref(k)))
        return st.value, n.value, k.value

    def result(self, rid: int):
        """(psi complex N_cs, norm_log, energy_log, (queue_s, latency_s)) of a finished request."""
        n, ns = self.n_cs[rid], self.nsteps[rid]
        psi = np.zeros(2 * n)
        nl, el, tm = np.zeros(max(ns, 1)), np.zeros(max(ns, 1)), np.zeros(2)
        self._err(lib().sg_server_result(self.ptr, int(rid), psi.ctypes.data, nl.ctypes.data, el.ctypes.data,
                                         tm.ctypes.data))
        return psi[:n] + 1j * psi[n:], nl[:ns], el[:ns], (float(tm[0]), float(tm[1]))

    def stats(self):
        a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        self._err(lib().sg_server_stats(self.ptr, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return {"iterations": a.value, "applications": b.value, "bytes_in_use": c.value}

    def run(self, chunk: int = 64):
        """Drives the engine until no request is active or queued."""
        while True:
            a, q = self.progress(chunk)
            if a == 0 and q == 0:
                return

    def close(self):
        if getattr(self, "ptr", None):
            lib().sg_server_destroy(self.ptr)
            self.ptr = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


SG_PEAK_FP32, SG_PEAK_FP32X2, SG_PEAK_FP64 = range(3)


def sg_measure_peak(kind="fp32", seconds: float = 1.0, stream=None):
    """Measured multiply-add throughput of the current device: (flop/s, SM count).
    kind: "fp32" (scalar fma), "fp32x2" (packed two-lane fma) or "fp64"."""
    k = {"fp32": SG_PEAK_FP32, "fp32x2": SG_PEAK_FP32X2, "fp64": SG_PEAK_FP64}.get(kind, kind)
    f, n = ctypes.c_double(), ctypes.c_int()
    st = lib().sg_measure_peak(int(k), float(seconds), ctypes.byref(f), ctypes.byref(n), _stream_ptr(stream))
    if st != SG_OK:
        raise SgError(st, "sg_measure_peak failed")
    return f.value, n.value


def sg_last_error(ctx: Ctx = None) -> str:
    return (lib().sg_last_error(ctx.ptr if ctx is not None else None) or b"").decode(errors="replace")


def sg_destroy(ctx: Ctx) -> None:
    if ctx is not None and getattr(ctx, "ptr", None):
        lib().sg_destroy(ctx.ptr)
        ctx.ptr = None

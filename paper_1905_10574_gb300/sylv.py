"""Thin Python binding of the CUDA library (C ABI of include/sylv.h).

Functions named like the C entry points (``sylv_tri_solve``, ``sylv_tri_solve_ex``,
``sylv_tri_solve_batched``, ``sylv_batch_*``, ``sylv_tri_solve_backward``,
``sylv_workspace_size``, ``sylv_error_string``) only marshal arguments: device
pointers, sizes, options.  Every step of the solve runs in the library's CUDA
kernels.  ``solve``/``batch_solve``/``SylvesterSolve`` are conveniences on torch
CUDA tensors (float64); they lay matrices out column-major, allocate the
workspace through torch (so calls can be captured in CUDA graphs) and call the
same entry points.  There is no CPU path: if the library is missing, loading
raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libsylv.so")

SYLV_OK = 0
SYLV_NEAR_SINGULAR = 1
SYLV_SCALE_UNDERFLOW = 2
SYLV_NOT_CONVERGED = 3
SYLV_OVERFLOWED = 4
SYLV_ERR_STRUCTURE_A = 101
SYLV_ERR_STRUCTURE_B = 102
SYLV_ERR_NONFINITE = 103
SYLV_ERR_RANGE = 104
SYLV_ERR_TIMEOUT = 105
SYLV_ERR_CUDA = 106
SYLV_ERR_WORKSPACE = 107
SYLV_ERR_UNSUPPORTED = 108

SYLV_FP64 = 0
SYLV_FP64_NONROBUST = 1
SYLV_FP32_REFINE = 2
PRECISIONS = {"fp64": SYLV_FP64, "fp64_nonrobust": SYLV_FP64_NONROBUST, "fp32_refine": SYLV_FP32_REFINE}


class sylv_opts(ctypes.Structure):
    _fields_ = [("transa", ctypes.c_int32), ("transb", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("tile", ctypes.c_int32), ("omega", ctypes.c_double), ("tol", ctypes.c_double),
                ("maxit", ctypes.c_int32), ("sync", ctypes.c_int32), ("timeout_ms", ctypes.c_int64),
                ("stream", ctypes.c_void_p), ("workspace", ctypes.c_void_p),
                ("workspace_bytes", ctypes.c_size_t), ("isgn", ctypes.c_int32), ("max_sms", ctypes.c_int32)]


class sylv_result(ctypes.Structure):
    _fields_ = [("log2scale", ctypes.c_int64), ("scale", ctypes.c_double), ("info", ctypes.c_int32),
                ("iters", ctypes.c_int32), ("last_update", ctypes.c_double),
                ("scale_events", ctypes.c_int32), ("min_tile_exp", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


# Every symbol include/sylv.h declares, with its ctypes signature.
_i64, _i32, _pd, _vp = ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p
_P64 = ctypes.POINTER(ctypes.c_int64)
_PP = ctypes.POINTER(ctypes.c_void_p)
SIGNATURES = {
    "sylv_default_opts": (None, [ctypes.POINTER(sylv_opts)]),
    "sylv_tri_solve": (ctypes.c_int, [_i64, _i64, _pd, _i64, _pd, _i64, _pd, _i64, _i64,
                                      ctypes.POINTER(ctypes.c_double)]),
    "sylv_tri_solve_ex": (ctypes.c_int, [_i64, _i64, _pd, _i64, _pd, _i64, _pd, _i64,
                                         ctypes.POINTER(sylv_opts), _vp]),
    "sylv_workspace_size": (ctypes.c_size_t, [_i64, _i64, ctypes.POINTER(sylv_opts)]),
    "sylv_schur_workspace_size": (ctypes.c_size_t, [_i64, _i64, ctypes.POINTER(sylv_opts)]),
    "sylv_batch_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), _i32, _P64, _P64, _PP, _P64, _PP,
                                         _P64, _PP, _P64, ctypes.POINTER(sylv_opts)]),
    "sylv_batch_create_tiles": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), _i32, _P64, _P64, _PP, _P64, _PP,
                                               _P64, _PP, _P64, ctypes.POINTER(ctypes.c_int32),
                                               ctypes.POINTER(sylv_opts)]),
    "sylv_batch_execute": (ctypes.c_int, [_vp, _vp]),
    "sylv_batch_results": (ctypes.c_int, [_vp, ctypes.POINTER(sylv_result)]),
    "sylv_batch_destroy": (None, [_vp]),
    "sylv_tri_solve_batched": (ctypes.c_int, [_i32, _P64, _P64, _PP, _P64, _PP, _P64, _PP, _P64,
                                              ctypes.POINTER(sylv_opts), ctypes.POINTER(sylv_result)]),
    "sylv_tri_solve_backward": (ctypes.c_int, [_i64, _i64, _pd, _i64, _pd, _i64, _pd, _i64, _i64, _pd, _i64,
                                               _pd, _i64, _pd, _i64, ctypes.POINTER(sylv_opts), _vp]),
    "sylv_error_string": (ctypes.c_char_p, [ctypes.c_int]),
    "sylv_version": (ctypes.c_char_p, []),
    "sylv_diag_wait_timeout": (ctypes.c_int, [_i64, _vp]),
    "sylv_diag_guards": (ctypes.c_int, [_i64, _pd, _pd, _pd, _pd, _pd, _pd, _pd, ctypes.c_double, _vp]),
    "sylv_diag_fma_rate": (ctypes.c_int, [_i32, _i64, ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_double), _vp]),
    "sylv_residual": (ctypes.c_int, [_i64, _i64, _pd, _i64, _pd, _i64, _pd, _i64, _pd, _i64, _pd, _i64, _vp]),
    "sylv_tri_solve_triangular": (ctypes.c_int, [_i64, _i64, _pd, _i64, _pd, _i64, ctypes.POINTER(sylv_opts),
                                                 _vp]),
    "sylv_solve_schur": (ctypes.c_int, [_i64, _i64, _pd, _i64, _pd, _i64, _pd, _i64, _pd, _i64, _pd, _i64,
                                        ctypes.POINTER(sylv_opts), _vp]),
    "sylv_tri_solve_noalloc": (ctypes.c_int, [_i64, _i64, _pd, _i64, _pd, _i64, _pd, _i64, _i64, _vp,
                                              ctypes.POINTER(sylv_result)]),
    "sylv_tri_solve_backward_batched": (ctypes.c_int, [_i32, _P64, _P64, _PP, _P64, _PP, _P64, _PP, _P64, _P64, _PP,
                                                       _P64, _PP, _P64, _PP, _P64, ctypes.POINTER(sylv_opts),
                                                       ctypes.POINTER(sylv_result)]),
    "sylv_profile": (ctypes.c_int, [ctypes.c_int]),
    "sylv_profile_read": (ctypes.c_int, [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)]),
}

_lib = None


def load(path: str | None = None):
    """Load libsylv.so (raises OSError if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise OSError(f"CUDA library not built: {p} (run paper_1905_10574_gb300.build)")
    L = ctypes.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


class SylvError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {code} ({sylv_error_string(code)})")


# ------------------------------------------------------------------ C-ABI mirrors
def sylv_default_opts() -> sylv_opts:
    o = sylv_opts()
    load().sylv_default_opts(ctypes.byref(o))
    return o


def sylv_error_string(code: int) -> str:
    return load().sylv_error_string(int(code)).decode()


def sylv_version() -> str:
    return load().sylv_version().decode()


def sylv_diag_wait_timeout(timeout_ms: int, stream=None) -> int:
    return load().sylv_diag_wait_timeout(int(timeout_ms), stream)


def sylv_diag_guards(count, c, t, x, z_update, b, d, z_division, omega, stream=None) -> int:
    """Device pointers (ints): the solver's ProtectUpdate/ProtectDivision evaluated
    element by element; returns the status code."""
    return load().sylv_diag_guards(int(count), c, t, x, z_update, b, d, z_division, float(omega), stream)


def sylv_diag_fma_rate(kind: int, iters: int, stream=None):
    """(status, GFLOP/s, ms) of the FMA peak probe: kind 0 binary64, 1 binary32."""
    g, t = ctypes.c_double(0.0), ctypes.c_double(0.0)
    rc = load().sylv_diag_fma_rate(int(kind), int(iters), ctypes.byref(g), ctypes.byref(t), stream)
    return rc, g.value, t.value


def sylv_profile(enable: bool) -> int:
    return load().sylv_profile(int(bool(enable)))


def sylv_profile_read():
    """(summed DAG-kernel milliseconds, launches) since the last read."""
    ms = ctypes.c_double(0.0)
    n = ctypes.c_int64(0)
    rc = load().sylv_profile_read(ctypes.byref(ms), ctypes.byref(n))
    if rc != 0:
        raise SylvError(rc, "sylv_profile_read")
    return ms.value, n.value


def sylv_tri_solve(m, n, A, lda, B, ldb, C, ldc, tile=0):
    """Device pointers (ints); returns (status, scale)."""
    sc = ctypes.c_double(0.0)
    rc = load().sylv_tri_solve(m, n, A, lda, B, ldb, C, ldc, tile, ctypes.byref(sc))
    return rc, sc.value


def sylv_tri_solve_noalloc(m, n, A, lda, B, ldb, C, ldc, tile=0, stream=None):
    """Device pointers (ints).  Solves with the library's fixed device scratch (no
    allocation); returns (status, sylv_result)."""
    res = sylv_result()
    rc = load().sylv_tri_solve_noalloc(m, n, A, lda, B, ldb, C, ldc, tile, stream, ctypes.byref(res))
    return rc, res


def sylv_tri_solve_triangular(m, n, A, lda, C, ldc, opts: sylv_opts | None = None, result=None) -> int:
    """Device pointers (ints).  Robust op(A) X = alpha C; ``result``: a sylv_result (host,
    sync mode) or a device address (async mode).  Returns the status code."""
    o = opts if opts is not None else sylv_default_opts()
    if isinstance(result, sylv_result):
        res = ctypes.cast(ctypes.pointer(result), ctypes.c_void_p)
    else:
        res = result
    return load().sylv_tri_solve_triangular(m, n, A, lda, C, ldc, ctypes.byref(o), res)


def sylv_solve_schur(m, n, U, ldu, TA, ldta, V, ldv, TB, ldtb, C, ldc, opts: sylv_opts | None = None,
                     result=None) -> int:
    """Device pointers (ints).  A X + isgn X B = alpha C from real Schur forms
    A = U TA U^T, B = V TB V^T; ``result`` as for sylv_tri_solve_ex."""
    o = opts if opts is not None else sylv_default_opts()
    if isinstance(result, sylv_result):
        res = ctypes.cast(ctypes.pointer(result), ctypes.c_void_p)
    else:
        res = result
    return load().sylv_solve_schur(m, n, U, ldu, TA, ldta, V, ldv, TB, ldtb, C, ldc, ctypes.byref(o), res)


def schur_solve(U, TA, V, TB, C, *, precision="fp64", tile=0, isgn=1, check=True):
    """A X + isgn X B = alpha C for CUDA float64 tensors given A = U TA U^T and
    B = V TB V^T (real Schur forms); returns (X, Result) with X column-major."""
    torch = _torch()
    U, TA, V, TB = (fortran(t) for t in (U, TA, V, TB))
    X = fortran(C).clone()
    m, n = X.shape
    o = make_opts(precision=precision, tile=tile, isgn=isgn,
                  stream=torch.cuda.current_stream(X.device).cuda_stream, sync=True)
    res = sylv_result()
    rc = sylv_solve_schur(m, n, U.data_ptr(), _ld(U), TA.data_ptr(), _ld(TA), V.data_ptr(), _ld(V), TB.data_ptr(),
                          _ld(TB), X.data_ptr(), _ld(X), o, res)
    if check and (rc >= 100 or rc < 0):
        raise SylvError(rc, "sylv_solve_schur")
    return X, Result(**res.as_dict())


def triangular_solve(A, C, *, transa=False, precision="fp64", tile=0, omega=0.0, check=True):
    """Robust op(A) X = alpha C for CUDA float64 tensors (A upper quasi-triangular);
    returns (X, Result) with X column-major."""
    torch = _torch()
    A = fortran(A)
    X = fortran(C).clone()
    m, n = X.shape
    o = make_opts(transa=transa, precision=precision, tile=tile, omega=omega,
                  stream=torch.cuda.current_stream(X.device).cuda_stream, sync=True)
    res = sylv_result()
    rc = sylv_tri_solve_triangular(m, n, A.data_ptr(), _ld(A), X.data_ptr(), _ld(X), o, res)
    if check and (rc >= 100 or rc < 0):
        raise SylvError(rc, "sylv_tri_solve_triangular")
    return X, Result(**res.as_dict())


def sylv_residual(m, n, A, lda, B, ldb, X, ldx, C, ldc, R, ldr, stream=None) -> int:
    """Device pointers (ints).  R <- C - (A X + X B) to binary64 accuracy (tensor cores);
    synchronizes the stream and returns the status code."""
    return load().sylv_residual(m, n, A, lda, B, ldb, X, ldx, C, ldc, R, ldr, stream)


def sylv_tri_solve_ex(m, n, A, lda, B, ldb, C, ldc, opts: sylv_opts | None = None, result=None):
    """Device pointers (ints).  ``result``: a sylv_result (host, sync mode) or a device
    address (async mode).  Returns the status code."""
    o = opts if opts is not None else sylv_default_opts()
    if isinstance(result, sylv_result):
        res = ctypes.cast(ctypes.pointer(result), ctypes.c_void_p)
    else:
        res = result
    return load().sylv_tri_solve_ex(m, n, A, lda, B, ldb, C, ldc, ctypes.byref(o), res)


def sylv_workspace_size(m, n, opts: sylv_opts | None = None) -> int:
    o = opts if opts is not None else sylv_default_opts()
    return int(load().sylv_workspace_size(m, n, ctypes.byref(o)))


def _i64arr(v):
    return (ctypes.c_int64 * len(v))(*[int(x) for x in v])


def _ptrarr(v):
    return (ctypes.c_void_p * len(v))(*[int(x) for x in v])


def sylv_batch_create(m, n, A, lda, B, ldb, C, ldc, opts: sylv_opts | None = None, tiles=None):
    """Lists of sizes and device pointers (and optionally a tile size per equation);
    returns an opaque plan handle."""
    o = opts if opts is not None else sylv_default_opts()
    h = ctypes.c_void_p()
    cnt = len(m)
    if tiles is None:
        rc = load().sylv_batch_create(ctypes.byref(h), cnt, _i64arr(m), _i64arr(n), _ptrarr(A), _i64arr(lda),
                                      _ptrarr(B), _i64arr(ldb), _ptrarr(C), _i64arr(ldc), ctypes.byref(o))
    else:
        t = (ctypes.c_int32 * max(cnt, 1))(*[int(x) for x in tiles])
        rc = load().sylv_batch_create_tiles(ctypes.byref(h), cnt, _i64arr(m), _i64arr(n), _ptrarr(A), _i64arr(lda),
                                            _ptrarr(B), _i64arr(ldb), _ptrarr(C), _i64arr(ldc), t, ctypes.byref(o))
    if rc != 0:
        raise SylvError(rc, "sylv_batch_create")
    return h


def sylv_batch_execute(plan, stream=None) -> int:
    return load().sylv_batch_execute(plan, stream)


def sylv_batch_results(plan, count: int):
    arr = (sylv_result * max(count, 1))()
    rc = load().sylv_batch_results(plan, arr)
    return rc, [arr[i] for i in range(count)]


def sylv_batch_destroy(plan) -> None:
    load().sylv_batch_destroy(plan)


def sylv_tri_solve_batched(m, n, A, lda, B, ldb, C, ldc, opts: sylv_opts | None = None):
    o = opts if opts is not None else sylv_default_opts()
    cnt = len(m)
    arr = (sylv_result * max(cnt, 1))()
    rc = load().sylv_tri_solve_batched(cnt, _i64arr(m), _i64arr(n), _ptrarr(A), _i64arr(lda), _ptrarr(B),
                                       _i64arr(ldb), _ptrarr(C), _i64arr(ldc), ctypes.byref(o), arr)
    return rc, [arr[i] for i in range(cnt)]


def sylv_tri_solve_backward_batched(m, n, A, lda, B, ldb, Y, ldy, log2scale, G, ldg, dA, ldda, dB, lddb,
                                    opts: sylv_opts | None = None):
    """Lists of sizes / device pointers (dA, dB: lists with 0 for 'skip', or None);
    returns (status, [sylv_result])."""
    o = opts if opts is not None else sylv_default_opts()
    cnt = len(m)
    arr = (sylv_result * max(cnt, 1))()
    rc = load().sylv_tri_solve_backward_batched(
        cnt, _i64arr(m), _i64arr(n), _ptrarr(A), _i64arr(lda), _ptrarr(B), _i64arr(ldb), _ptrarr(Y), _i64arr(ldy),
        _i64arr(log2scale), _ptrarr(G), _i64arr(ldg), _ptrarr(dA) if dA is not None else None,
        _i64arr(ldda) if dA is not None else None, _ptrarr(dB) if dB is not None else None,
        _i64arr(lddb) if dB is not None else None, ctypes.byref(o), arr)
    return rc, [arr[i] for i in range(cnt)]


def sylv_tri_solve_backward(m, n, A, lda, B, ldb, Y, ldy, log2scale, G, ldg, dA, ldda, dB, lddb,
                            opts: sylv_opts | None = None, result=None):
    o = opts if opts is not None else sylv_default_opts()
    if isinstance(result, sylv_result):
        res = ctypes.cast(ctypes.pointer(result), ctypes.c_void_p)
    else:
        res = result
    return load().sylv_tri_solve_backward(m, n, A, lda, B, ldb, Y, ldy, log2scale, G, ldg, dA or None, ldda,
                                          dB or None, lddb, ctypes.byref(o), res)


# ------------------------------------------------------------------ torch conveniences
def _torch():
    import torch
    return torch


def fortran(t):
    """Column-major (Fortran-ordered) float64 copy/view of a 2-D tensor."""
    torch = _torch()
    t = t.to(torch.float64)
    if t.dim() != 2:
        raise ValueError("expected a matrix")
    r, c = t.shape
    if t.stride(0) == 1 and (t.stride(1) >= max(r, 1) or c <= 1):
        return t
    return t.t().contiguous().t()


def empty_fortran(m, n, device, dtype=None):
    torch = _torch()
    return torch.empty((n, m), dtype=dtype or torch.float64, device=device).t()


def _ld(t) -> int:
    return max(int(t.stride(1)) if t.shape[1] > 1 else int(t.shape[0]), 1)


@dataclass
class Result:
    log2scale: int
    scale: float
    info: int
    iters: int
    last_update: float
    scale_events: int
    min_tile_exp: int


def make_opts(*, transa=False, transb=False, precision="fp64", tile=0, omega=0.0, tol=0.0, maxit=0,
              timeout_ms=0, stream=None, sync=True, isgn=1, max_sms=0) -> sylv_opts:
    o = sylv_default_opts()
    o.isgn = -1 if isgn < 0 else 1
    o.max_sms = int(max_sms)
    o.transa = int(bool(transa))
    o.transb = int(bool(transb))
    o.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    o.tile = int(tile)
    o.omega = float(omega)
    o.tol = float(tol)
    o.maxit = int(maxit)
    o.timeout_ms = int(timeout_ms)
    o.stream = stream
    o.sync = int(bool(sync))
    return o


def solve(A, B, C, *, transa=False, transb=False, precision="fp64", tile=0, omega=0.0, tol=0.0, maxit=0,
          timeout_ms=0, inplace=False, check=True, isgn=1, max_sms=0):
    """Solve op(A) Y + isgn Y op(B) = alpha C (isgn = +1 or -1) for CUDA float64 tensors;
    returns (Y, Result).  Y is column-major; with inplace=True and a column-major C, C
    itself is overwritten.  max_sms caps the SMs the tile kernel occupies (0 = all)."""
    torch = _torch()
    A = fortran(A)
    B = fortran(B)
    Cf = fortran(C)
    Y = Cf if (inplace or Cf.data_ptr() != C.data_ptr()) else Cf.clone()
    m, n = Y.shape
    stream = torch.cuda.current_stream(Y.device).cuda_stream
    o = make_opts(transa=transa, transb=transb, precision=precision, tile=tile, omega=omega, tol=tol,
                  maxit=maxit, timeout_ms=timeout_ms, stream=stream, sync=True, isgn=isgn, max_sms=max_sms)
    ws_bytes = sylv_workspace_size(m, n, o)
    ws = torch.empty(max(ws_bytes, 1) + 256, dtype=torch.uint8, device=Y.device)
    base = (ws.data_ptr() + 255) // 256 * 256
    o.workspace = base
    o.workspace_bytes = ws_bytes
    res = sylv_result()
    rc = sylv_tri_solve_ex(m, n, A.data_ptr(), _ld(A), B.data_ptr(), _ld(B), Y.data_ptr(), _ld(Y), o, res)
    if check and (rc >= 100 or rc < 0):
        raise SylvError(rc, "sylv_tri_solve_ex")
    return Y, Result(**res.as_dict())


def residual(A, B, X, C, *, stream=None):
    """R = C - (A X + X B) for float64 CUDA tensors (A, B read in their quasi-triangular
    parts), computed by sylv_residual; returns a new column-major tensor."""
    torch = _torch()
    A, B, X, C = (fortran(t) for t in (A, B, X, C))
    m, n = C.shape
    R = empty_fortran(m, n, C.device, torch.float64)
    s = stream if stream is not None else torch.cuda.current_stream(C.device).cuda_stream
    rc = sylv_residual(m, n, A.data_ptr(), _ld(A), B.data_ptr(), _ld(B), X.data_ptr(), _ld(X), C.data_ptr(), _ld(C),
                       R.data_ptr(), _ld(R), s)
    if rc != 0:
        raise SylvError(rc, "sylv_residual")
    return R


def batch_solve(As, Bs, Cs, *, transa=False, transb=False, tile=0, precision="fp64", timeout_ms=0, isgn=1,
                tol=0.0, maxit=0):
    """Solve a list of equations op(A_i) Y_i + Y_i op(B_i) = alpha_i C_i in one batched
    launch; Cs are overwritten when they are column-major float64 CUDA tensors, else
    copies are solved.  precision "fp32_refine" refines every equation to tol (0: the
    library default).  Returns (Ys, [Result])."""
    torch = _torch()
    As = [fortran(a) for a in As]
    Bs = [fortran(b) for b in Bs]
    Ys = [fortran(c) for c in Cs]
    o = make_opts(transa=transa, transb=transb, tile=tile, precision=precision, timeout_ms=timeout_ms,
                  stream=torch.cuda.current_stream().cuda_stream, isgn=isgn, tol=tol, maxit=maxit)
    plan = sylv_batch_create([y.shape[0] for y in Ys], [y.shape[1] for y in Ys], [a.data_ptr() for a in As],
                             [_ld(a) for a in As], [b.data_ptr() for b in Bs], [_ld(b) for b in Bs],
                             [y.data_ptr() for y in Ys], [_ld(y) for y in Ys], o)
    try:
        rc = sylv_batch_execute(plan, o.stream)
        if rc != 0:
            raise SylvError(rc, "sylv_batch_execute")
        rc, res = sylv_batch_results(plan, len(Ys))
        if rc >= 100:
            raise SylvError(rc, "sylv_batch_results")
    finally:
        sylv_batch_destroy(plan)
    return Ys, [Result(**r.as_dict()) for r in res]


class SylvesterSolve:
    """torch.autograd.Function: Y = solve(A, B, C) (robust FP64, alpha held fixed), with the
    hand-written adjoint of sylv_tri_solve_backward.  Use ``SylvesterSolve.apply(A, B, C,
    transa, transb, tile)``; passing one tensor as both A and B (with transb=True) gives the
    Lyapunov form A Y + Y A^T = C and autograd adds both gradient contributions."""

    _fn = None

    @classmethod
    def apply(cls, A, B, C, transa=False, transb=False, tile=0):
        if cls._fn is None:
            cls._fn = _make_autograd_fn()
        return cls._fn.apply(A, B, C, transa, transb, tile)


def _make_autograd_fn():
    torch = _torch()

    class _Fn(torch.autograd.Function):
        @staticmethod
        def forward(ctx, A, B, C, transa, transb, tile):
            Y, res = solve(A.detach(), B.detach(), C.detach(), transa=transa, transb=transb, tile=tile)
            ctx.save_for_backward(A, B, Y)
            ctx.cfg = (transa, transb, tile, res.log2scale)
            return Y

        @staticmethod
        def backward(ctx, gY):
            A, B, Y = ctx.saved_tensors
            transa, transb, tile, e = ctx.cfg
            Af, Bf = fortran(A.detach()), fortran(B.detach())
            G = fortran(gY.detach()).clone()
            m, n = G.shape
            dA = empty_fortran(m, m, G.device)
            dB = empty_fortran(n, n, G.device)
            o = make_opts(transa=transa, transb=transb, tile=tile,
                          stream=torch.cuda.current_stream(G.device).cuda_stream)
            res = sylv_result()
            rc = sylv_tri_solve_backward(m, n, Af.data_ptr(), _ld(Af), Bf.data_ptr(), _ld(Bf), Y.data_ptr(),
                                         _ld(Y), int(e), G.data_ptr(), _ld(G), dA.data_ptr(), _ld(dA),
                                         dB.data_ptr(), _ld(dB), o, res)
            if rc >= 100 or rc < 0:
                raise SylvError(rc, "sylv_tri_solve_backward")
            return dA, dB, G, None, None, None

    return _Fn


class BatchSylvesterSolve:
    """torch.autograd.Function over a batch of equations of one shape: A (b, m, m),
    B (b, n, n), C (b, m, n) CUDA float64 tensors -> Y (b, m, n), each
    op(A_i) Y_i + Y_i op(B_i) = alpha_i C_i solved robustly in one batched launch;
    backward runs the batched adjoint (sylv_tri_solve_backward_batched).  Passing
    one tensor as both A and B with transb=True gives Lyapunov equations."""

    _fn = None

    @classmethod
    def apply(cls, A, B, C, transa=False, transb=False, tile=0):
        if cls._fn is None:
            cls._fn = _make_batch_autograd_fn()
        return cls._fn.apply(A, B, C, transa, transb, tile)


def batch_fortran(t):
    """(b, r, c) float64 tensor whose every [i] is column-major (strides (r*c, 1, r))."""
    torch = _torch()
    t = t.to(torch.float64)
    b, r, c = t.shape
    if t.stride(1) == 1 and t.stride(2) == max(r, 1) and t.stride(0) == r * c:
        return t
    return t.transpose(1, 2).contiguous().transpose(1, 2)


def _make_batch_autograd_fn():
    torch = _torch()

    class _Fn(torch.autograd.Function):
        @staticmethod
        def forward(ctx, A, B, C, transa, transb, tile):
            Af, Bf = batch_fortran(A.detach()), batch_fortran(B.detach())
            Y = batch_fortran(C.detach()).clone()
            cnt, m, n = Y.shape
            o = make_opts(transa=transa, transb=transb, tile=tile, stream=torch.cuda.current_stream().cuda_stream)
            ea, eb, ey = Af.element_size(), Bf.element_size(), Y.element_size()
            plan = sylv_batch_create([m] * cnt, [n] * cnt, [Af.data_ptr() + i * Af.stride(0) * ea for i in range(cnt)],
                                     [max(m, 1)] * cnt, [Bf.data_ptr() + i * Bf.stride(0) * eb for i in range(cnt)],
                                     [max(n, 1)] * cnt, [Y.data_ptr() + i * Y.stride(0) * ey for i in range(cnt)],
                                     [max(m, 1)] * cnt, o)
            try:
                rc = sylv_batch_execute(plan, o.stream)
                if rc != 0:
                    raise SylvError(rc, "sylv_batch_execute")
                rc, res = sylv_batch_results(plan, cnt)
                if rc >= 100:
                    raise SylvError(rc, "sylv_batch_results")
            finally:
                sylv_batch_destroy(plan)
            ctx.save_for_backward(Af, Bf, Y)
            ctx.cfg = (transa, transb, tile, [r.log2scale for r in res])
            return Y

        @staticmethod
        def backward(ctx, gY):
            Af, Bf, Y = ctx.saved_tensors
            transa, transb, tile, es = ctx.cfg
            G = batch_fortran(gY.detach()).clone()
            cnt, m, n = G.shape
            dA = torch.empty((cnt, m, m), dtype=torch.float64, device=G.device).transpose(1, 2)
            dB = torch.empty((cnt, n, n), dtype=torch.float64, device=G.device).transpose(1, 2)
            o = make_opts(transa=transa, transb=transb, tile=tile, stream=torch.cuda.current_stream().cuda_stream)

            def ptrs(t):
                return [t.data_ptr() + i * t.stride(0) * t.element_size() for i in range(cnt)]

            rc, res = sylv_tri_solve_backward_batched([m] * cnt, [n] * cnt, ptrs(Af), [max(m, 1)] * cnt, ptrs(Bf),
                                                      [max(n, 1)] * cnt, ptrs(Y), [max(m, 1)] * cnt, es, ptrs(G),
                                                      [max(m, 1)] * cnt, ptrs(dA), [max(m, 1)] * cnt, ptrs(dB),
                                                      [max(n, 1)] * cnt, o)
            if rc >= 100 or rc < 0:
                raise SylvError(rc, "sylv_tri_solve_backward_batched")
            return dA, dB, G, None, None, None

    return _Fn

"""TEST INFRASTRUCTURE ONLY: Python face of the FP64 CPU oracle.

Only the test suite, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this module.  It shares no code with the GPU library and never
imports it.

Contents, each written from the paper (Schwarz & Kjelgaard Mikkelsen 2019):
  * ``trsyl``      -- Algorithm 2 (robust, global scale) / Algorithm 1 (plain) in C
                      (``sylv_oracle.c``), with op(A)/op(B) transposes reduced to
                      the untransposed problem by index reversal.
  * ``small_solve``, ``protect_update``, ``protect_division`` -- the Sec. 2.1
                      building blocks, exposed for the pins.
  * ``kron_solve`` -- the textbook Kronecker form of eq. (2),
                      (I_n (x) A + B^T (x) I_m) vec(X) = vec(C), by dense LU.
  * ``residual``   -- the relative residual of eq. (9), evaluated with a common
                      power-of-two shift so that tiny alpha or huge Y cannot
                      under/overflow it.
  * ``smin_of``    -- the pivot floor for near-singular small systems.
  * ``schur_solve``-- the Bartels-Stewart reduction of Sec. 1 (eqs. (3)-(5)) around
                      ``trsyl``: U^T C V, the triangular solve, U Y V^T (numpy GEMMs).
  * ``residual_matrix`` -- R = C - (A X + X B) from its definition (eq. (7) with
                      alpha = 1) in extended precision, and ``residual_matrix_exact``
                      in exact rational arithmetic for tiny cases.
  * ``solve_decimal`` -- the unscaled solution X of eq. (2) by plain block
                      substitution (Algorithm 1's order) in decimal arithmetic with
                      50 significant digits and an exponent range no solution here
                      can leave, so nothing over- or underflows and no scaling is
                      needed; ``decimal_scaled`` rounds alpha X to binary64.  The
                      reference where alpha < 2^-1074: there Algorithm 2's single
                      factor flushes right-hand sides it has not reached yet.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sylv_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")

OMEGA = 2.0 ** 1020  # overflow threshold: 2^1020 leaves x16 headroom below the largest double
EPS = 2.0 ** -52
SMALLNUM = 2.0 ** -1022

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle's C source into ``oracle/_build/liboracle.so`` with gcc."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        # -ffp-contract=off: no fused multiply-add contraction, so x86 and Arm
        # hosts round every product and sum the same way.
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        d, i, i64 = ctypes.c_double, ctypes.c_int, ctypes.c_int64
        pd = ctypes.POINTER(ctypes.c_double)
        L.oracle_protect_update.argtypes = [d, d, d, d]
        L.oracle_protect_update.restype = i
        L.oracle_protect_division.argtypes = [d, d, d]
        L.oracle_protect_division.restype = i
        L.oracle_small_solve.argtypes = [i, i, pd, i, pd, i, pd, i, d, d, i, ctypes.POINTER(i)]
        L.oracle_small_solve.restype = i
        L.oracle_blocks.argtypes = [i64, pd, i64, ctypes.POINTER(i64)]
        L.oracle_blocks.restype = i
        L.oracle_trsyl.argtypes = [i64, i64, pd, i64, pd, i64, pd, i64, d, d, i,
                                   ctypes.POINTER(i64), pd, ctypes.POINTER(i)]
        L.oracle_trsyl.restype = i
        _lib = L
    return _lib


def _pd(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _fortran(a) -> np.ndarray:
    return np.asfortranarray(np.asarray(a, dtype=np.float64))


def protect_update(c: float, t: float, x: float, omega: float = OMEGA) -> int:
    """log2 of ProtectUpdate's power-of-two factor (Sec. 2.1)."""
    return lib().oracle_protect_update(float(c), float(t), float(x), float(omega))


def protect_division(b: float, d: float, omega: float = OMEGA) -> int:
    """log2 of ProtectDivision's power-of-two factor (Sec. 2.1)."""
    return lib().oracle_protect_division(float(b), float(d), float(omega))


def quasi_tri(T) -> np.ndarray:
    """The part of T the solver reads: upper triangle plus first subdiagonal."""
    return np.triu(np.asarray(T, dtype=np.float64), -1)


def smin_of(A, B) -> float:
    """Pivot floor for the small solves: max(2^-52 * largest |entry| of A and B, 2^-1022)."""
    amax = float(np.max(np.abs(quasi_tri(A)))) if np.size(A) else 0.0
    bmax = float(np.max(np.abs(quasi_tri(B)))) if np.size(B) else 0.0
    return max(EPS * max(amax, bmax), SMALLNUM)


def small_solve(A11, B11, R, smin: float = SMALLNUM, omega: float = OMEGA, robust: bool = True):
    """Robust <=2x2 by <=2x2 Sylvester solve A11 Z + Z B11 = beta R (Sec. 2.1).

    Returns (Z, log2beta, info)."""
    A11 = _fortran(A11)
    B11 = _fortran(B11)
    Z = np.array(R, dtype=np.float64, order="F", copy=True)
    ma, nb = A11.shape[0], B11.shape[0]
    lb = ctypes.c_int(0)
    info = lib().oracle_small_solve(ma, nb, _pd(A11), max(ma, 1), _pd(B11), max(nb, 1), _pd(Z),
                                    max(ma, 1), float(smin), float(omega), int(robust),
                                    ctypes.byref(lb))
    return Z, lb.value, info


def blocks(T) -> list[int] | None:
    """Start indices of the 1x1/2x2 diagonal blocks (plus the end), or None if T is not
    quasi-triangular."""
    T = _fortran(T)
    n = T.shape[0]
    starts = (ctypes.c_int64 * (n + 1))()
    nb = lib().oracle_blocks(n, _pd(T), max(n, 1), starts)
    if nb < 0:
        return None
    return [int(starts[i]) for i in range(nb + 1)]


def anti_transpose(T) -> np.ndarray:
    """J T^T J with J the reversal permutation; upper quasi-triangular if T is."""
    return np.ascontiguousarray(np.flip(np.asarray(T).T, (0, 1)))


def trsyl(A, B, C, robust: bool = True, transa: bool = False, transb: bool = False,
          omega: float = OMEGA, smin: float | None = None):
    """Solve op(A) Y + Y op(B) = alpha C with Algorithm 2 (robust) or Algorithm 1.

    op(A)^T cases are reduced to the untransposed one: with J the reversal
    permutation, A^T Y + Y B = C  <=>  (J A^T J)(J Y) + (J Y) B = J C, and likewise
    on the right for B.

    Returns a dict with Y, log2scale (alpha = 2^log2scale), info, peak (largest
    magnitude Y ever held) and nan_seen.
    """
    A = quasi_tri(A)
    B = quasi_tri(B)
    C = np.asarray(C, dtype=np.float64)
    m, n = C.shape
    if smin is None:
        smin = smin_of(A, B)
    if transa:
        A = anti_transpose(A)
        C = np.flip(C, 0)
    if transb:
        B = anti_transpose(B)
        C = np.flip(C, 1)
    Af, Bf = _fortran(A), _fortran(B)
    Y = np.array(C, dtype=np.float64, order="F", copy=True)
    e = ctypes.c_int64(0)
    peak = ctypes.c_double(0.0)
    nan_seen = ctypes.c_int(0)
    info = lib().oracle_trsyl(m, n, _pd(Af), max(m, 1), _pd(Bf), max(n, 1), _pd(Y), max(m, 1),
                              float(smin), float(omega), int(robust), ctypes.byref(e),
                              ctypes.byref(peak), ctypes.byref(nan_seen))
    if transa:
        Y = np.flip(Y, 0)
    if transb:
        Y = np.flip(Y, 1)
    return {"Y": np.ascontiguousarray(Y), "log2scale": int(e.value), "info": int(info),
            "peak": float(peak.value), "nan_seen": bool(nan_seen.value)}


def kron_solve(A, B, C, transa: bool = False, transb: bool = False, isgn: int = 1) -> np.ndarray:
    """X with op(A) X + isgn X op(B) = C from the Kronecker form of eq. (2):
    (I_n (x) op(A) + isgn op(B)^T (x) I_m) vec(X) = vec(C), vec stacking columns."""
    A = quasi_tri(A)
    B = quasi_tri(B)
    if transa:
        A = A.T
    if transb:
        B = B.T
    C = np.asarray(C, dtype=np.float64)
    m, n = C.shape
    K = np.kron(np.eye(n), A) + (1.0 if isgn >= 0 else -1.0) * np.kron(B.T, np.eye(m))
    x = np.linalg.solve(K, C.reshape(-1, order="F"))
    return x.reshape((m, n), order="F")


def _shift_for(Y: np.ndarray) -> int:
    amax = float(np.max(np.abs(Y))) if Y.size else 0.0
    if amax == 0.0 or not np.isfinite(amax):
        return 0
    return -int(np.frexp(amax)[1])


def residual(A, B, Y, C, log2scale: int, transa: bool = False, transb: bool = False) -> float:
    """Eq. (9): ||alpha C - (op(A) Y + Y op(B))||_F / ((||A||_F + ||B||_F) ||Y||_F + ||alpha C||_F).

    Numerator and denominator are both homogeneous of degree one in (Y, alpha C), so
    both are multiplied by a common power of two 2^s that brings max|Y| to [1/2, 1);
    alpha C is formed as ldexp(C, log2scale + s), which may underflow harmlessly."""
    A = quasi_tri(A)
    B = quasi_tri(B)
    opA = A.T if transa else A
    opB = B.T if transb else B
    Y = np.asarray(Y, dtype=np.float64)
    s = _shift_for(Y)
    Ys = np.ldexp(Y, s)
    aC = np.ldexp(np.asarray(C, dtype=np.float64), int(log2scale) + s)
    R = aC - (opA @ Ys + Ys @ opB)
    den = (np.linalg.norm(A) + np.linalg.norm(B)) * np.linalg.norm(Ys) + np.linalg.norm(aC)
    if den == 0.0:
        return 0.0 if np.linalg.norm(R) == 0.0 else float("inf")
    return float(np.linalg.norm(R) / den)


def scaled_solution(Y, log2scale: int) -> np.ndarray:
    """Y / alpha = Y * 2^-log2scale (the solution X of the unscaled equation)."""
    return np.ldexp(np.asarray(Y, dtype=np.float64), -int(log2scale))


def quasi_mask(T) -> np.ndarray:
    """Entries the solver reads: upper triangle plus nonzero first-subdiagonal entries."""
    T = np.asarray(T, dtype=np.float64)
    n = T.shape[0]
    r, c = np.indices((n, n))
    return (r <= c) | ((r == c + 1) & (T != 0.0))


def kron_grad(A, B, C, W, transa: bool = False, transb: bool = False, isgn: int = 1):
    """Gradients of L = sum(W * X), op(A) X + isgn X op(B) = C, from the Kronecker form
    K vec(X) = vec(C), K = I_n (x) op(A) + isgn op(B)^T (x) I_m (eq. (2) vectorised).

    dL/dvec(C) = K^-T vec(W) =: lam and dL/dK = -lam vec(X)^T.  op(A)[i,k] sits in K
    at (i + m j, k + m j) for every j; op(B)[k,j] sits at (i + m j, i + m k) for every
    i; the gradient of an entry is the sum of dL/dK over its positions.  Gradients
    of A (B) are those of op(A) (op(B)), transposed back when op = T, and restricted
    to the entries the solver reads.  Returns (dA, dB, dC, X)."""
    A = quasi_tri(A)
    B = quasi_tri(B)
    opA = A.T if transa else A
    opB = B.T if transb else B
    C = np.asarray(C, dtype=np.float64)
    m, n = C.shape
    sg = 1.0 if isgn >= 0 else -1.0
    K = np.kron(np.eye(n), opA) + sg * np.kron(opB.T, np.eye(m))
    x = np.linalg.solve(K, C.reshape(-1, order="F"))
    lam = np.linalg.solve(K.T, np.asarray(W, dtype=np.float64).reshape(-1, order="F"))
    GK = -np.outer(lam, x)
    dopA = np.zeros((m, m))
    for i in range(m):
        for k in range(m):
            dopA[i, k] = sum(GK[i + m * j, k + m * j] for j in range(n))
    dopB = np.zeros((n, n))
    for k in range(n):
        for j in range(n):
            dopB[k, j] = sg * sum(GK[i + m * j, i + m * k] for i in range(m))
    dA = dopA.T if transa else dopA
    dB = dopB.T if transb else dopB
    dA = np.where(quasi_mask(A), dA, 0.0)
    dB = np.where(quasi_mask(B), dB, 0.0)
    return dA, dB, lam.reshape((m, n), order="F"), x.reshape((m, n), order="F")


def residual_matrix(A, B, X, C) -> np.ndarray:
    """R = C - (A X + X B) with A, B read in their quasi-triangular parts (upper triangle
    and first subdiagonal), evaluated in numpy's long double (x87 extended or binary128,
    64 or 113 significand bits) and rounded once to binary64 at the end."""
    ld = np.longdouble
    Aq = np.triu(np.asarray(A, dtype=np.float64), -1).astype(ld)
    Bq = np.triu(np.asarray(B, dtype=np.float64), -1).astype(ld)
    Xl = np.asarray(X, dtype=np.float64).astype(ld)
    Cl = np.asarray(C, dtype=np.float64).astype(ld)
    return (Cl - (Aq @ Xl + Xl @ Bq)).astype(np.float64)


def residual_matrix_exact(A, B, X, C) -> np.ndarray:
    """The same residual in exact rational arithmetic (Python fractions), rounded once
    to binary64: for tiny cases only."""
    from fractions import Fraction
    A, B, X, C = (np.asarray(t, dtype=np.float64) for t in (A, B, X, C))
    m, n = C.shape
    F = lambda v: Fraction(float(v))  # noqa: E731  (a double is an exact rational)
    R = np.empty((m, n))
    for i in range(m):
        for j in range(n):
            acc = F(C[i, j])
            for k in range(max(0, i - 1), m):
                acc -= F(A[i, k]) * F(X[k, j])
            for k in range(0, min(n, j + 2)):
                acc -= F(X[i, k]) * F(B[k, j])
            R[i, j] = float(acc)
    return R


def schur_solve(U, TA, V, TB, C, isgn: int = 1):
    """X and log2(alpha) with A X + isgn X B = alpha C for A = U TA U^T, B = V TB V^T
    (Sec. 1, eqs. (3)-(5)): C~ = U^T C V, TA Y + isgn Y TB = alpha C~, X = U Y V^T."""
    U, TA, V, TB, C = (np.asarray(t, dtype=np.float64) for t in (U, TA, V, TB, C))
    Ct = U.T @ C @ V
    out = trsyl(TA, TB if isgn >= 0 else -TB, Ct)
    return U @ out["Y"] @ V.T, out["log2scale"]


def _decimal_blocks(T) -> list[tuple[int, int]]:
    """(start, size) of the diagonal blocks of an upper quasi-triangular T: a nonzero
    T[i+1, i] starts a 2x2 block at i."""
    n = T.shape[0]
    out, i = [], 0
    while i < n:
        size = 2 if (i + 1 < n and T[i + 1, i] != 0.0) else 1
        out.append((i, size))
        i += size
    return out


def _decimal_gauss(M, r):
    """Gaussian elimination with partial pivoting on a small dense Decimal system."""
    n = len(r)
    M = [row[:] for row in M]
    r = list(r)
    for k in range(n):
        p = max(range(k, n), key=lambda i: abs(M[i][k]))
        M[k], M[p] = M[p], M[k]
        r[k], r[p] = r[p], r[k]
        for i in range(k + 1, n):
            f = M[i][k] / M[k][k]
            for j in range(k, n):
                M[i][j] -= f * M[k][j]
            r[i] -= f * r[k]
    x = [None] * n
    for i in range(n - 1, -1, -1):
        acc = r[i]
        for j in range(i + 1, n):
            acc -= M[i][j] * x[j]
        x[i] = acc / M[i][i]
    return x


def solve_decimal(A, B, C, transa: bool = False, transb: bool = False, digits: int = 50):
    """X with op(A) X + X op(B) = C (eq. (2), no scaling) as a list of rows of
    ``decimal.Decimal``.  Block substitution in Algorithm 1's order: for each diagonal
    block of B from the left and each diagonal block of A from the bottom, the block's
    right-hand side C_kl - sum_{i>k} A_ki X_il - sum_{j<l} X_kj B_jl (eq. (6)) and the
    small system of eq. (2) for the block pair, by Gaussian elimination.  The binary64
    inputs are exact decimals; every operation keeps `digits` significant digits and
    the exponent range is unbounded for these sizes.  Transposes as in ``trsyl``."""
    import decimal
    A = quasi_tri(A)
    B = quasi_tri(B)
    C = np.asarray(C, dtype=np.float64)
    if transa:
        A = anti_transpose(A)
        C = np.flip(C, 0)
    if transb:
        B = anti_transpose(B)
        C = np.flip(C, 1)
    m, n = C.shape
    ctx = decimal.Context(prec=digits, Emax=decimal.MAX_EMAX, Emin=decimal.MIN_EMIN)
    with decimal.localcontext(ctx):
        D = decimal.Decimal
        Ad = [[D(float(A[i, j])) for j in range(m)] for i in range(m)]
        Bd = [[D(float(B[i, j])) for j in range(n)] for i in range(n)]
        X = [[None] * n for _ in range(m)]
        ablk, bblk = _decimal_blocks(A), _decimal_blocks(B)
        for c0, nb in bblk:
            for r0, ma in reversed(ablk):
                idx = [(ii, jj) for jj in range(nb) for ii in range(ma)]  # vec order
                rhs = []
                for ii, jj in idx:
                    i, j = r0 + ii, c0 + jj
                    acc = D(float(C[i, j]))
                    for k in range(r0 + ma, m):
                        if Ad[i][k]:
                            acc -= Ad[i][k] * X[k][j]
                    for k in range(c0):
                        if Bd[k][j]:
                            acc -= X[i][k] * Bd[k][j]
                    rhs.append(acc)
                M = [[D(0)] * len(idx) for _ in idx]
                for u, (i, j) in enumerate(idx):
                    for v, (i2, j2) in enumerate(idx):
                        e = D(0)
                        if j == j2:
                            e += Ad[r0 + i][r0 + i2]
                        if i == i2:
                            e += Bd[c0 + j2][c0 + j]
                        M[u][v] = e
                z = _decimal_gauss(M, rhs)
                for u, (i, j) in enumerate(idx):
                    X[r0 + i][c0 + j] = z[u]
    if transa:
        X = X[::-1]
    if transb:
        X = [row[::-1] for row in X]
    return X


def decimal_scaled(X, log2scale: int) -> np.ndarray:
    """alpha X = X * 2^log2scale rounded to binary64 (0 where it underflows)."""
    import decimal
    ctx = decimal.Context(prec=60, Emax=decimal.MAX_EMAX, Emin=decimal.MIN_EMIN)
    with decimal.localcontext(ctx):
        two = decimal.Decimal(2) ** int(log2scale)
        rows = [[float(v * two) for v in row] for row in X]
    return np.array(rows, dtype=np.float64).reshape(len(X), len(X[0]) if X else 0)

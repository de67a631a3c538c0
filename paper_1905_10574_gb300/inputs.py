"""Seeded synthetic inputs for the triangular Sylvester equation A Y + Y B = alpha C.

This module only draws random matrices with the structure of the paper's
workloads; it holds none of the solver's arithmetic, and both the GPU path and
the CPU oracle take their inputs from it.  Every matrix is float64, column-major
(Fortran order), drawn from numpy's PCG64 generator with the given seed.

Generators
  * ``quasi_triangular(n, seed, kind=...)`` -- upper quasi-triangular (real Schur
    form, Sec. 1 eq. (4)) with 1x1 and standardized 2x2 diagonal blocks [a b; c a],
    bc < 0.  A 2x2 block starts at a free index with probability 1/3, so about half
    of the eigenvalues sit in 2x2 blocks (2p/(1+p) = 1/2 for p = 1/3).
      kind="benign":   a ~ U[1,10], |b|,|c| ~ U[0.5,2], strictly-upper U[-1,1].
      kind="wellcond": as "benign" with the strictly-upper part scaled by 1/sqrt(n)
                       (the in-block b entries unscaled); the benign kind's
                       triangular part makes back substitution grow exponentially
                       with n, this one keeps the solve well conditioned.
      kind="growth":   as "benign" with the strictly-upper part scaled by ``upper``
                       (large values make unscaled substitution overflow).
  * ``paper_matrix(n, mu, seed)`` -- the test matrices of Sec. 3: ones in the
    strictly-upper part, diagonal blocks mu*T with T = 1 or [1 1; -1 1].
  * ``rhs(m, n, seed)`` -- C with entries U[-1,1].
  * ``batch_shapes(count, lo, hi, seed)`` -- per-instance (m, n) log-uniform in [lo, hi].
"""
from __future__ import annotations

import numpy as np

__all__ = ["quasi_triangular", "paper_matrix", "rhs", "batch_shapes", "diagonal_pattern",
           "problem"]


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def diagonal_pattern(n: int, rng: np.random.Generator, p_pair: float = 1.0 / 3.0) -> list[int]:
    """Start indices of 2x2 diagonal blocks: at each free index a pair starts with
    probability p_pair (never past the last index)."""
    starts = []
    i = 0
    while i < n:
        if i + 1 < n and rng.random() < p_pair:
            starts.append(i)
            i += 2
        else:
            i += 1
    return starts


def quasi_triangular(n: int, seed: int, kind: str = "benign", upper: float = 1.0,
                     p_pair: float = 1.0 / 3.0) -> np.ndarray:
    rng = _rng(seed)
    T = np.zeros((n, n), dtype=np.float64, order="F")
    if n == 0:
        return T
    if kind == "benign":
        su = 1.0
    elif kind == "wellcond":
        su = 1.0 / np.sqrt(n)
    elif kind == "growth":
        su = float(upper)
    else:
        raise ValueError(f"unknown kind {kind!r}")
    U = rng.uniform(-1.0, 1.0, size=(n, n)) * su
    T[:, :] = np.triu(U, 1)
    diag = rng.uniform(1.0, 10.0, size=n)
    T[np.arange(n), np.arange(n)] = diag
    for i in diagonal_pattern(n, rng, p_pair):
        a = diag[i]
        b = rng.uniform(0.5, 2.0)
        c = -rng.uniform(0.5, 2.0)
        if rng.random() < 0.5:
            b, c = -b, -c
        T[i, i] = a
        T[i + 1, i + 1] = a
        T[i, i + 1] = b
        T[i + 1, i] = c
    return T


def paper_matrix(n: int, mu: float, seed: int = 0, p_pair: float = 1.0 / 3.0,
                 pairs: list[int] | None = None) -> np.ndarray:
    """Sec. 3 test matrix: strictly-upper ones; diagonal blocks mu*1 or mu*[1 1; -1 1].
    The 2x2 blocks start at the indices ``pairs`` if given, else at random."""
    rng = _rng(seed)
    T = np.triu(np.ones((n, n), dtype=np.float64), 1)
    T[np.arange(n), np.arange(n)] = mu
    starts = diagonal_pattern(n, rng, p_pair) if pairs is None else list(pairs)
    for i in starts:
        T[i, i + 1] = mu
        T[i + 1, i] = -mu
    return np.asfortranarray(T)


def rhs(m: int, n: int, seed: int) -> np.ndarray:
    rng = _rng(seed)
    return np.asfortranarray(rng.uniform(-1.0, 1.0, size=(m, n)))


def batch_shapes(count: int, lo: int, hi: int, seed: int) -> list[tuple[int, int]]:
    """Per-instance (m, n), each log-uniform over [lo, hi] and rounded to an integer."""
    rng = _rng(seed)
    u = rng.uniform(np.log(lo), np.log(hi), size=(count, 2))
    mn = np.clip(np.rint(np.exp(u)).astype(np.int64), lo, hi)
    return [(int(a), int(b)) for a, b in mn]


def problem(m: int, n: int, seed: int, kind: str = "benign", upper: float = 1.0):
    """(A, B, C) for one equation, drawn from the streams 3*seed, 3*seed+1 and
    3*seed+2 (distinct streams, so m == n does not give B == A)."""
    A = quasi_triangular(m, 3 * seed + 0, kind, upper)
    B = quasi_triangular(n, 3 * seed + 1, kind, upper)
    C = rhs(m, n, 3 * seed + 2)
    return A, B, C


# Named workloads (shapes and generator settings of the benchmark configurations).
# "overflow_4000": robust vs non-robust FP64 at m = n = 4000.  The strictly-upper
# scale 4.1 was chosen with the FP64 oracle (tests/golden/calibrate_overflow.py):
# the unscaled growth log2 max|X| is ~353 bits at m = n = 1000 and grows linearly
# with the order, ~1400 bits at 4000: past the binary64 range (1024), so the
# non-robust solve overflows, while alpha = 2^-(growth - 1020) stays representable.
WORKLOADS = {
    "benign_256": dict(m=256, n=256, seed=0, kind="benign", upper=1.0, tile=64),
    "overflow_4000": dict(m=4000, n=4000, seed=0, kind="growth", upper=4.1, tile=32),
    "overflow_1000": dict(m=1000, n=1000, seed=0, kind="growth", upper=16.0, tile=32),
    "benign_1000": dict(m=1000, n=1000, seed=0, kind="benign", upper=1.0, tile=32),
    "benign_4000": dict(m=4000, n=4000, seed=0, kind="benign", upper=1.0, tile=32),
    "benign_8000": dict(m=8000, n=8000, seed=0, kind="benign", upper=1.0, tile=32),
    "benign_10000": dict(m=10000, n=10000, seed=0, kind="benign", upper=1.0, tile=32),
    "benign_20000": dict(m=20000, n=20000, seed=0, kind="benign", upper=1.0, tile=32),
    "wellcond_8000": dict(m=8000, n=8000, seed=0, kind="wellcond", upper=1.0, tile=32),
    "wellcond_4000": dict(m=4000, n=4000, seed=0, kind="wellcond", upper=1.0, tile=32),
}


def workload(name: str):
    """(A, B, C, settings) of a named workload."""
    w = WORKLOADS[name]
    A, B, C = problem(w["m"], w["n"], w["seed"], kind=w["kind"], upper=w["upper"])
    return A, B, C, w

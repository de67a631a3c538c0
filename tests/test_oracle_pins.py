"""Pins of the FP64 CPU oracle against facts fixed by the paper and by mathematics.

Each test would fail on a plausible mistake in the oracle: a dropped update term,
a wrong sign or index, a transposed operand, a scale factor applied twice or not
at all, a wrong guard in ProtectUpdate/ProtectDivision.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from paper_1905_10574_gb300 import inputs

OMEGA = 2.0 ** 1020


# ---------------------------------------------------------------- ProtectUpdate / ProtectDivision
def _edge_values():
    vals = [0.0, 2.0 ** -1074, 2.0 ** -1022, 0.5, 1.0, 1.0 + 2 ** -52, 2.0, 3.0,
            2.0 ** 100, 2.0 ** 500, 2.0 ** 1019, OMEGA * 0.75, OMEGA]
    rng = np.random.default_rng(7)
    vals += list(np.ldexp(rng.uniform(0.5, 1.0, 40), rng.integers(-1074, 1020, 40)))
    return [float(v) for v in vals]


def test_protect_update_contract(orc):
    """Sec. 2.1: zeta in (0,1], a power of two, zeta*(c + t*x) <= Omega (checked in exact
    rational arithmetic); no scaling when c + t*x <= Omega/2; and zeta is the largest
    power of two allowed, up to rounding: 2*zeta*(c + t*x) > Omega*(1 - 2^-48)."""
    vals = _edge_values()
    rng = np.random.default_rng(1)
    triples = [(c, t, x) for c in vals[::3] for t in vals[::2] for x in vals]
    triples += [tuple(float(v) for v in np.ldexp(rng.uniform(0.5, 1, 3), rng.integers(-60, 1021, 3)))
                for _ in range(3000)]
    for c, t, x in triples:
        if max(c, t, x) > OMEGA:
            continue
        z = orc.protect_update(c, t, x)
        assert z <= 0
        zeta = Fraction(2) ** z
        tot = Fraction(c) + Fraction(t) * Fraction(x)
        assert zeta * tot <= Fraction(OMEGA), (c, t, x, z)
        if tot <= Fraction(OMEGA) / 2:
            assert z == 0, (c, t, x, z)
        if z < 0:
            assert 2 * zeta * tot > Fraction(OMEGA) * (1 - Fraction(1, 2 ** 48)), (c, t, x, z)


def test_protect_division_contract(orc):
    """Sec. 2.1: zeta*|b|/d <= Omega exactly; zeta == 1 when |b|/d <= Omega; otherwise
    zeta is the largest power of two that satisfies the bound."""
    vals = _edge_values()
    for b in vals:
        for d in vals:
            if d == 0.0 or b > OMEGA:
                continue
            for sb in (1.0, -1.0):
                z = orc.protect_division(sb * b, -d if sb < 0 else d)
                q = Fraction(b) / Fraction(d)
                zeta = Fraction(2) ** z
                assert zeta * q <= Fraction(OMEGA), (b, d, z)
                if q <= Fraction(OMEGA):
                    assert z == 0
                else:
                    assert 2 * zeta * q > Fraction(OMEGA), (b, d, z)


# ---------------------------------------------------------------- small solves (Sec. 2.1)
def _block(size, rng):
    if size == 1:
        return np.array([[rng.uniform(1, 10)]])
    a = rng.uniform(1, 10)
    b, c = rng.uniform(0.5, 2), -rng.uniform(0.5, 2)
    return np.array([[a, b], [c, a]])


@pytest.mark.parametrize("ma,nb", [(1, 1), (1, 2), (2, 1), (2, 2)])
def test_small_solve_matches_kronecker_lu(orc, ma, nb):
    """All four block shapes against a dense LU of (I (x) A11 + B11^T (x) I)."""
    rng = np.random.default_rng(100 + 10 * ma + nb)
    for _ in range(200):
        A11, B11 = _block(ma, rng), _block(nb, rng)
        if rng.random() < 0.5:  # also non-standardized blocks (any 2x2 with complex eigenvalues)
            A11 = A11 + np.triu(rng.uniform(-1, 1, A11.shape), 1)
        R = rng.uniform(-1, 1, (ma, nb))
        Z, lb, info = orc.small_solve(A11, B11, R)
        assert info == 0 and lb == 0
        K = np.kron(np.eye(nb), A11) + np.kron(B11.T, np.eye(ma))
        ref = np.linalg.solve(K, R.reshape(-1, order="F")).reshape((ma, nb), order="F")
        np.testing.assert_allclose(Z, ref, rtol=1e-13, atol=1e-15)


def test_small_solve_guards_scale_exactly(orc):
    """A divisor far below 1 with a right-hand side near Omega must scale, by a power of
    two, and Z/beta must still solve the system."""
    A11 = np.array([[2.0 ** -600]])
    B11 = np.array([[0.0]])
    R = np.array([[2.0 ** 1000]])
    Z, lb, info = orc.small_solve(A11, B11, R)
    assert lb < 0 and abs(Z[0, 0]) <= OMEGA
    # R / A11 = 2^1600 exactly; ProtectDivision picks the largest power of two that
    # keeps the quotient <= Omega = 2^1020, so beta = 2^-580 and Z = 2^1020.
    assert lb == -580
    assert Z[0, 0] == math.ldexp(1.0, 1600 + lb)


def test_small_solve_near_singular_perturbs(orc):
    """lambda(A11) + lambda(B11) = 0: the pivot is replaced by smin and info = 1."""
    Z, lb, info = orc.small_solve(np.array([[3.0]]), np.array([[-3.0]]), np.array([[1.0]]), smin=2.0 ** -40)
    assert info == 1
    assert Z[0, 0] == 2.0 ** 40


# ---------------------------------------------------------------- full solves
def test_diagonal_closed_form_bit_exact(orc):
    """Diagonal A and B: Y_ij = C_ij / (a_i + b_j), one rounding, alpha = 1."""
    rng = np.random.default_rng(3)
    m, n = 37, 23
    a = rng.uniform(1, 10, m)
    b = rng.uniform(1, 10, n)
    C = rng.uniform(-1, 1, (m, n))
    out = orc.trsyl(np.diag(a), np.diag(b), C)
    assert out["log2scale"] == 0 and out["info"] == 0
    assert np.array_equal(out["Y"], C / (a[:, None] + b[None, :]))


@pytest.mark.parametrize("m,n", [(1, 1), (2, 2), (1, 5), (5, 1), (3, 7), (16, 16), (24, 9), (19, 24)])
@pytest.mark.parametrize("transa,transb", [(False, False), (True, False), (False, True), (True, True)])
def test_matches_kronecker_brute_force(orc, m, n, transa, transb):
    """Eq. (2) in Kronecker form, dense LU, on quasi-triangular inputs with 2x2 blocks."""
    seed = 1000 * m + n + 7 * transa + 13 * transb
    A, B, C = inputs.problem(m, n, seed, kind="benign")
    out = orc.trsyl(A, B, C, transa=transa, transb=transb)
    X = orc.scaled_solution(out["Y"], out["log2scale"])
    ref = orc.kron_solve(A, B, C, transa, transb)
    assert out["log2scale"] == 0
    err = np.linalg.norm(X - ref) / np.linalg.norm(ref)
    assert err < 1e-12, err


def test_kronecker_catches_ignored_lower_part(orc):
    """Entries below the first subdiagonal are not part of the input; the oracle must
    ignore them (garbage there must not change Y)."""
    A, B, C = inputs.problem(12, 10, 5)
    A2 = A + np.tril(np.full(A.shape, 7.0), -2)
    B2 = B + np.tril(np.full(B.shape, -3.0), -2)
    assert np.array_equal(orc.trsyl(A, B, C)["Y"], orc.trsyl(A2, B2, C)["Y"])


def test_lapack_dtrsyl_cross_check(orc):
    """Same Y/alpha as LAPACK's scalar robust solver (called as a library, never read)."""
    sl = pytest.importorskip("scipy.linalg.lapack")
    for (m, n, kind) in [(64, 48, "benign"), (96, 96, "wellcond"), (33, 70, "wellcond")]:
        A, B, C = inputs.problem(m, n, m + n, kind=kind)
        for ta, tb in [(False, False), (True, False), (False, True), (True, True)]:
            out = orc.trsyl(A, B, C, transa=ta, transb=tb)
            x, scale, info = sl.dtrsyl(A, B, C, trana="T" if ta else "N", tranb="T" if tb else "N")
            assert info == 0
            X = orc.scaled_solution(out["Y"], out["log2scale"])
            ref = x / scale
            err = np.linalg.norm(X - ref) / np.linalg.norm(ref)
            assert err < 1e-11, (m, n, kind, ta, tb, err)


def test_forced_scaling_is_exact_power_of_two(orc):
    """With a tiny Omega the robust solve must scale, and Y/alpha must equal the unscaled
    solution: scaling by powers of two changes no digit (no subnormals here)."""
    A, B, C = inputs.problem(40, 30, 11, kind="growth", upper=10.0)
    ref = orc.trsyl(A, B, C)
    assert ref["log2scale"] == 0 and ref["peak"] > 2.0 ** 30
    # Omega must stay above the inputs' norms (Alg. 2's precondition, ~2^7.6 here)
    # but below the growth of the solve (~2^31).
    small = orc.trsyl(A, B, C, omega=2.0 ** 12)
    assert small["log2scale"] < -10
    assert small["peak"] <= 2.0 ** 12
    X = orc.scaled_solution(small["Y"], small["log2scale"])
    err = np.linalg.norm(X - ref["Y"]) / np.linalg.norm(ref["Y"])
    assert err < 1e-13, err


def test_omega_never_exceeded_where_plain_substitution_overflows(orc):
    """The Ensure clause of Algorithm 2: with growth beyond the double range the robust
    solve keeps every entry <= Omega at all times, while Algorithm 1 overflows."""
    A, B, C = inputs.problem(48, 48, 3, kind="growth", upper=1e120)
    plain = orc.trsyl(A, B, C, robust=False)
    assert plain["nan_seen"] or not np.isfinite(plain["peak"])
    rob = orc.trsyl(A, B, C)
    assert rob["peak"] <= OMEGA and not rob["nan_seen"]
    assert np.all(np.isfinite(rob["Y"]))
    assert rob["log2scale"] < -100
    assert orc.residual(A, B, rob["Y"], C, rob["log2scale"]) < 1e-14


def test_no_scaling_on_paper_matrices_with_mu_m(orc):
    """Sec. 4: with mu = m and nu = n the paper's test matrices need no scaling."""
    m, n = 60, 44
    A = inputs.paper_matrix(m, float(m), seed=1)
    B = inputs.paper_matrix(n, float(n), seed=2)
    C = np.ones((m, n))
    out = orc.trsyl(A, B, C)
    assert out["log2scale"] == 0
    assert orc.residual(A, B, out["Y"], C, 0) < 1e-15


def test_paper_small_mu_triggers_scaling(orc):
    """Sec. 4: small mu makes the same matrices need scaling (cost-of-robustness sweep)."""
    m = n = 300
    A = inputs.paper_matrix(m, 1e-3, seed=1)
    B = inputs.paper_matrix(n, 1e-2, seed=2)
    out = orc.trsyl(A, B, np.ones((m, n)))
    assert out["log2scale"] < 0
    assert out["peak"] <= OMEGA and not out["nan_seen"]


def test_worked_example_eigenvalues(orc):
    """Sec. 3's 5x5 example: the generator's 2x2 block encoding mu*[1 1; -1 1] gives the
    matrix printed in the paper, with eigenvalues mu, mu, mu(1+i), mu(1-i), mu."""
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_example_5x5.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    coef = np.array([[float(v) for v in r] for r in rows]).reshape(5, 5, 2)
    mu = 3.0
    printed = coef[:, :, 0] * mu + coef[:, :, 1]
    gen = inputs.paper_matrix(5, mu, pairs=[2])
    assert np.array_equal(gen, printed)
    ev = np.sort_complex(np.linalg.eigvals(gen))
    want = np.sort_complex(np.array([mu, mu, mu * (1 + 1j), mu * (1 - 1j), mu]))
    np.testing.assert_allclose(ev, want, atol=1e-6)
    assert orc.blocks(gen) == [0, 1, 2, 4, 5]


def test_block_scan_rejects_non_quasi_triangular(orc):
    T = np.triu(np.ones((6, 6)))
    T[2, 1] = 1.0
    T[3, 2] = 1.0
    assert orc.blocks(T) is None
    out = orc.trsyl(T, np.eye(3), np.ones((6, 3)))
    assert out["info"] == -2


def test_residual_eq9_exact_solution(orc):
    """Eq. (9) is zero for an exactly representable solution and sees a one-entry defect."""
    rng = np.random.default_rng(0)
    m, n = 9, 7
    A = np.triu(rng.integers(-3, 4, (m, m)).astype(float))
    B = np.triu(rng.integers(-3, 4, (n, n)).astype(float))
    X = rng.integers(-5, 6, (m, n)).astype(float)
    C = A @ X + X @ B
    assert orc.residual(A, B, X, C, 0) == 0.0
    X2 = X.copy()
    X2[4, 3] += 1.0
    R = C - (A @ X2 + X2 @ B)
    want = np.linalg.norm(R) / ((np.linalg.norm(A) + np.linalg.norm(B)) * np.linalg.norm(X2) + np.linalg.norm(C))
    assert math.isclose(orc.residual(A, B, X2, C, 0), want, rel_tol=1e-15)
    # residual is invariant under a common power-of-two scaling of (Y, alpha)
    assert math.isclose(orc.residual(A, B, X2 * 2.0 ** -900, C, -900), want, rel_tol=1e-15)


def test_lyapunov_symmetry(orc):
    """A Y + Y A^T = C with symmetric C has a symmetric solution."""
    A = inputs.quasi_triangular(30, 4, kind="wellcond")
    C = inputs.rhs(30, 30, 5)
    C = C + C.T
    out = orc.trsyl(A, A, C, transb=True)
    Y = out["Y"]
    assert np.linalg.norm(Y - Y.T) <= 1e-13 * np.linalg.norm(Y)
    ref = orc.kron_solve(A, A, C, False, True)
    assert np.linalg.norm(Y - ref) <= 1e-12 * np.linalg.norm(ref)


@pytest.mark.parametrize("transa,transb", [(False, False), (True, False), (False, True)])
def test_kron_grad_matches_finite_differences(orc, transa, transb):
    """The Kronecker-form gradients against central differences of the Kronecker solve."""
    m, n = 5, 4
    A, B, C = inputs.problem(m, n, 21, kind="wellcond")
    W = inputs.rhs(m, n, 99)
    dA, dB, dC, _ = orc.kron_grad(A, B, C, W, transa, transb)
    h = 1e-6

    def loss(A_, B_, C_):
        return float(np.sum(W * orc.kron_solve(A_, B_, C_, transa, transb)))

    maskA, maskB = orc.quasi_mask(A), orc.quasi_mask(B)
    for (i, j) in [(0, 0), (0, 3), (1, 2), (3, 4), (4, 4)]:
        E = np.zeros_like(A)
        E[i, j] = h
        fd = (loss(A + E, B, C) - loss(A - E, B, C)) / (2 * h)
        want = fd if maskA[i, j] else 0.0
        assert abs(dA[i, j] - want) <= 1e-7 * max(1.0, abs(fd)), (i, j, dA[i, j], fd)
    for (i, j) in [(0, 1), (2, 3), (1, 1)]:
        E = np.zeros_like(B)
        E[i, j] = h
        fd = (loss(A, B + E, C) - loss(A, B - E, C)) / (2 * h)
        assert abs(dB[i, j] - fd) <= 1e-7 * max(1.0, abs(fd)), (i, j, dB[i, j], fd)
        assert maskB[i, j]
    for (i, j) in [(0, 0), (4, 3), (2, 1)]:
        E = np.zeros_like(C)
        E[i, j] = h
        fd = (loss(A, B, C + E) - loss(A, B, C - E)) / (2 * h)
        assert abs(dC[i, j] - fd) <= 1e-7 * max(1.0, abs(fd))


def test_residual_matrix_against_exact_rationals(orc):
    """The extended-precision residual R = C - (A X + X B) agrees with exact rational
    arithmetic (independent evaluation: fractions, explicit quasi-triangular index
    ranges) on a tiny case with 2x2 blocks and a wide magnitude range."""
    rng = np.random.default_rng(5)
    m, n = 9, 7
    A = orc.quasi_tri(np.triu(rng.uniform(-1, 1, (m, m)), -1))
    A[3, 2] = 0.75
    B = orc.quasi_tri(np.triu(rng.uniform(-1, 1, (n, n)), -1))
    B[5, 4] = -1.25
    X = rng.uniform(-1, 1, (m, n)) * np.exp2(rng.integers(-30, 30, (m, n)))
    C = rng.uniform(-1, 1, (m, n))
    R = orc.residual_matrix(A, B, X, C)
    Rx = orc.residual_matrix_exact(A, B, X, C)
    scale = np.abs(np.triu(A, -1)) @ np.abs(X) + np.abs(X) @ np.abs(np.triu(B, -1)) + np.abs(C)
    assert np.all(np.abs(R - Rx) <= 2.0 ** -52 * np.abs(Rx) + 2.0 ** -60 * scale)


def test_residual_matrix_diagonal_closed_form(orc):
    """Diagonal A, B: R_ij = C_ij - (a_i + b_j) X_ij."""
    rng = np.random.default_rng(6)
    a, b = rng.uniform(1, 5, 6), rng.uniform(1, 5, 4)
    X, C = rng.uniform(-1, 1, (6, 4)), rng.uniform(-1, 1, (6, 4))
    R = orc.residual_matrix(np.diag(a), np.diag(b), X, C)
    ref = C - (a[:, None] + b[None, :]) * X  # three roundings in binary64
    bound = 4 * 2.0 ** -53 * (np.abs(a[:, None] + b[None, :]) * np.abs(X) + np.abs(C))
    assert np.all(np.abs(R - ref) <= bound)


def test_kron_sign_variant_against_definition(orc):
    """isgn = -1: the Kronecker solve satisfies A X - X B = C entry by entry, and equals
    the isgn = +1 solve with -B (the two forms of the same equation)."""
    rng = np.random.default_rng(12)
    m, n = 7, 5
    A = orc.quasi_tri(np.triu(rng.uniform(-1, 1, (m, m)), 0) + np.diag(rng.uniform(1, 3, m)))
    B = orc.quasi_tri(np.triu(rng.uniform(-1, 1, (n, n)), 0) - np.diag(rng.uniform(1, 3, n)))
    B[2, 1] = 0.5
    C = rng.uniform(-1, 1, (m, n))
    X = orc.kron_solve(A, B, C, isgn=-1)
    assert np.allclose(A @ X - X @ np.triu(B, -1), C, rtol=0, atol=1e-13)
    assert np.allclose(X, orc.kron_solve(A, -B, C), rtol=0, atol=1e-14)


def test_kron_grad_sign_variant_fd(orc):
    """Gradients of L = sum(W X) for A X - X B = C against central differences."""
    rng = np.random.default_rng(13)
    m, n = 4, 3
    A = np.triu(rng.uniform(-1, 1, (m, m)), 1) + np.diag(rng.uniform(1, 2, m))
    B = np.triu(rng.uniform(-1, 1, (n, n)), 1) - np.diag(rng.uniform(1, 2, n))
    C, W = rng.uniform(-1, 1, (m, n)), rng.uniform(-1, 1, (m, n))
    dA, dB, dC, _ = orc.kron_grad(A, B, C, W, isgn=-1)
    L = lambda A_, B_, C_: float(np.sum(W * orc.kron_solve(A_, B_, C_, isgn=-1)))  # noqa: E731
    h = 1e-6
    for (M, D) in ((A, dA), (B, dB), (C, dC)):
        for (i, j) in [(0, 0), (0, M.shape[1] - 1), (M.shape[0] - 1, M.shape[1] - 1)]:
            Mp, Mm = M.copy(), M.copy()
            Mp[i, j] += h
            Mm[i, j] -= h
            args_p = [Mp if M is X else X for X in (A, B, C)]
            args_m = [Mm if M is X else X for X in (A, B, C)]
            fd = (L(*args_p) - L(*args_m)) / (2 * h)
            assert abs(fd - D[i, j]) <= 1e-7 * max(1.0, abs(fd))


def test_triangular_solve_is_sylvester_with_zero_b(orc):
    """The robust triangular solve op(A) X = alpha C is Algorithm 2 with B = 0: the
    oracle's solve with a zero B agrees with dense LU on a quasi-triangular A."""
    rng = np.random.default_rng(14)
    m, n = 11, 4
    A = np.triu(rng.uniform(-1, 1, (m, m)), 1) + np.diag(rng.uniform(1, 3, m))
    A[4, 3], A[3, 4], A[4, 4] = -0.9, 1.1, A[3, 3]  # a 2x2 block at rows 3-4
    C = rng.uniform(-1, 1, (m, n))
    out = orc.trsyl(A, np.zeros((n, n)), C)
    assert out["info"] == 0 and out["log2scale"] == 0
    assert np.allclose(out["Y"], np.linalg.solve(orc.quasi_tri(A), C), rtol=0, atol=1e-13)
    outT = orc.trsyl(A, np.zeros((n, n)), C, transa=True)
    assert np.allclose(outT["Y"], np.linalg.solve(orc.quasi_tri(A).T, C), rtol=0, atol=1e-13)


def test_schur_solve_against_dense_sylvester(orc):
    """The Bartels-Stewart form around the oracle's triangular solve matches scipy's
    dense Sylvester solver on A = U TA U^T, B = V TB V^T (real Schur forms from scipy)."""
    sla = pytest.importorskip("scipy.linalg")
    rng = np.random.default_rng(15)
    m, n = 9, 6
    A = rng.standard_normal((m, m)) + 4 * np.eye(m)
    B = rng.standard_normal((n, n)) + 4 * np.eye(n)
    C = rng.standard_normal((m, n))
    TA, U = sla.schur(A, output="real")
    TB, V = sla.schur(B, output="real")
    X, e = orc.schur_solve(U, TA, V, TB, C)
    assert e == 0
    assert np.allclose(X, sla.solve_sylvester(A, B, C), rtol=0, atol=1e-12)
    Xm, _ = orc.schur_solve(U, TA, V, -TB, C, isgn=-1)
    assert np.allclose(Xm, X, rtol=0, atol=1e-14)


# ---------------------------------------------------------------- the decimal reference solution
@pytest.mark.parametrize("ta,tb", [(False, False), (False, True), (True, False), (True, True)])
def test_decimal_solution_matches_kronecker(orc, ta, tb):
    """eq. (2): the decimal block substitution against the textbook Kronecker solve
    (dense LU, a different method), with 2x2 blocks on both sides and transposes."""
    A, B, C = inputs.problem(11, 9, 4, kind="benign")
    X = orc.decimal_scaled(orc.solve_decimal(A, B, C, ta, tb), 0)
    K = orc.kron_solve(A, B, C, ta, tb)
    assert np.linalg.norm(X - K) / np.linalg.norm(K) <= 1e-13


def test_decimal_solution_beyond_binary64_satisfies_equation_exactly(orc):
    """A growth input whose solution leaves the binary64 range (max|X| ~ 1e400): the
    decimal solution, converted exactly to rationals, satisfies A X + X B = C
    entry by entry to ~1e-45 relative to |A||X| + |X||B| (exact rational residual), so
    neither an exponent limit nor a dropped term can hide in it."""
    A, B, C = inputs.problem(8, 7, 2, kind="growth", upper=1e60)
    A, B = np.triu(A, -1), np.triu(B, -1)
    X = orc.solve_decimal(A, B, C)
    F = [[Fraction(v) for v in row] for row in X]
    m, n = C.shape
    Af = [[Fraction(float(A[i, j])) for j in range(m)] for i in range(m)]
    Bf = [[Fraction(float(B[i, j])) for j in range(n)] for i in range(n)]
    big = max(abs(v) for row in F for v in row)
    assert big > Fraction(10) ** 400
    for i in range(m):
        for j in range(n):
            r = Fraction(float(C[i, j])) - sum(Af[i][k] * F[k][j] for k in range(m)) \
                - sum(F[i][k] * Bf[k][j] for k in range(n))
            s = sum(abs(Af[i][k] * F[k][j]) for k in range(m)) + sum(abs(F[i][k] * Bf[k][j]) for k in range(n))
            assert abs(r) <= s * Fraction(1, 10 ** 45)


def test_decimal_scaled_agrees_with_algorithm2_without_scaling(orc):
    """Where Algorithm 2 needs no scaling (alpha = 1), its binary64 result and the
    rounded decimal solution agree to rounding; decimal_scaled applies 2^log2scale
    exactly (a power of two moves no significand)."""
    A, B, C = inputs.problem(40, 30, 6, kind="benign")
    ref = orc.trsyl(A, B, C)
    assert ref["log2scale"] == 0
    X = orc.solve_decimal(A, B, C)
    Y = orc.decimal_scaled(X, 0)
    assert np.linalg.norm(Y - ref["Y"]) / np.linalg.norm(Y) <= 1e-13
    assert np.array_equal(orc.decimal_scaled(X, -300), np.ldexp(Y, -300))

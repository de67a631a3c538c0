"""GPU parity of sylv_residual (R = C - (A X + X B), the refinement's first residual,
on the bf16 tensor cores by error-free splitting) against the oracle's definition of
the same residual in extended precision.

Bound (balanced inputs): each element within 2^-44 (|A||X| + |X||B|)_ij + 2^-52 |R_ij|
of the oracle.  The splitting keeps 56 bits below each row/column maximum and drops
pairs of slices that weigh below 2^-56, so even rows dominated by their diagonal
(the well-conditioned generator) stay near 2^-48; the oracle itself is accurate to
~2^-60.  With rows or columns of very
different magnitudes the guarantee is relative to the row and column maxima instead
(_rowcol_bound), which is what the refinement needs (a normwise residual).
"""
import numpy as np
import pytest

from paper_1905_10574_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def sy():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_10574_gb300 import build, sylv
    build.build()
    sylv.load()
    return sylv


def _gpu_residual(sy, A, B, X, C):
    d = lambda t: torch.from_numpy(np.asfortranarray(t)).cuda()  # noqa: E731
    R = sy.residual(d(A), d(B), d(X), d(C))
    torch.cuda.synchronize()
    return R.cpu().numpy()


def _bound(A, B, X, R):
    Aq, Bq = np.abs(np.triu(A, -1)), np.abs(np.triu(B, -1))
    return 2.0 ** -44 * (Aq @ np.abs(X) + np.abs(X) @ Bq) + 2.0 ** -52 * np.abs(R)


def test_exact_dyadic_inputs(orc, sy):
    """A, B with 8-bit entries and X with binary32 entries: every slice product is
    captured, so the GPU result differs from the exact residual only by the binary64
    roundings of its ~12 final sums (< 2^-48 of the magnitudes involved)."""
    rng = np.random.default_rng(11)
    m, n = 200, 150
    A = np.triu(rng.integers(-255, 256, (m, m)) / 256.0, -1)
    A[np.tril_indices(m, -2)] = 0
    B = np.triu(rng.integers(-255, 256, (n, n)) / 256.0, -1)
    X = rng.uniform(-1, 1, (m, n)).astype(np.float32).astype(np.float64)
    C = rng.uniform(-1, 1, (m, n))
    R = _gpu_residual(sy, A, B, X, C)
    ref = orc.residual_matrix(A, B, X, C)
    scale = np.abs(A) @ np.abs(X) + np.abs(X) @ np.abs(B) + np.abs(C)
    assert np.all(np.abs(R - ref) <= 2.0 ** -48 * scale)


@pytest.mark.parametrize("m,n", [(1, 1), (5, 3), (64, 64), (130, 70), (257, 129), (64, 200), (300, 300)])
def test_random_shapes(orc, sy, m, n):
    A, B, C = inputs.problem(m, n, seed=m * 1000 + n, kind="benign")
    rng = np.random.default_rng(m + n)
    X = rng.uniform(-1, 1, (m, n))
    R = _gpu_residual(sy, A, B, X, C)
    ref = orc.residual_matrix(A, B, X, C)
    assert np.all(np.isfinite(R))
    assert np.all(np.abs(R - ref) <= _bound(A, B, X, ref))


def _rowcol_bound(A, B, X, R):
    """The splitting's own guarantee: each slice pair is exact and what is dropped lies
    below 2^-56 of (row maximum) x (column maximum) per product term, so the error is
    bounded by K * 2^-54 * max_k|left(i,k)| * max_k|right(k,j)| for each product (a
    normwise guarantee; componentwise only when rows and columns are balanced); the
    test allows 2^-44."""
    Aq, Bq = np.abs(np.triu(A, -1)), np.abs(np.triu(B, -1))
    Xa = np.abs(X)
    m, n = X.shape
    ax = m * np.max(Aq, axis=1)[:, None] * np.max(Xa, axis=0)[None, :]
    xb = n * np.max(Xa, axis=1)[:, None] * np.max(Bq, axis=0)[None, :]
    return 2.0 ** -44 * (ax + xb) + 2.0 ** -52 * np.abs(R)


def test_quasi_blocks_on_tile_edges_and_wide_ranges(orc, sy):
    """2x2 blocks straddling the 64- and 128-row tile edges (the subdiagonal entries
    must be read), and rows/columns whose magnitudes differ by 2^+-200: the error
    stays within the splitting's row/column-maximum bound."""
    m, n = 260, 200
    rng = np.random.default_rng(3)
    A = np.triu(rng.uniform(-1, 1, (m, m)))
    B = np.triu(rng.uniform(-1, 1, (n, n)))
    for i in (63, 127, 191):
        A[i + 1, i] = 0.5
    for j in (63, 127):
        B[j + 1, j] = -0.75
    A *= np.exp2(rng.integers(-200, 200, m))[:, None]
    X = rng.uniform(-1, 1, (m, n)) * np.exp2(rng.integers(-200, 200, n))[None, :]
    C = rng.uniform(-1, 1, (m, n))
    R = _gpu_residual(sy, A, B, X, C)
    ref = orc.residual_matrix(A, B, X, C)
    assert np.all(np.isfinite(R))
    assert np.all(np.abs(R - ref) <= _rowcol_bound(A, B, X, ref))


def test_argument_errors(sy):
    d = torch.zeros((4, 4), dtype=torch.float64, device="cuda")
    p = d.data_ptr()
    assert sy.sylv_residual(-1, 4, p, 4, p, 4, p, 4, p, 4, p, 4, None) == -1
    assert sy.sylv_residual(4, 4, p, 4, p, 4, 0, 4, p, 4, p, 4, None) == -7
    assert sy.sylv_residual(4, 4, p, 4, p, 4, p, 4, 0, 4, p, 4, None) == -9
    assert sy.sylv_residual(4, 4, p, 4, p, 4, p, 4, p, 4, p, 2, None) == -12
    assert sy.sylv_residual(0, 4, p, 1, p, 4, p, 1, p, 1, p, 1, None) == 0


def test_full_size_sampled(orc, sy):
    """m = n = 4000 (the mixed-precision workload's shape at half size): 256 sampled
    entries against the definition evaluated entry by entry in extended precision."""
    A, B, C, _ = inputs.workload("wellcond_4000")
    rng = np.random.default_rng(9)
    X = rng.uniform(-1, 1, C.shape).astype(np.float32).astype(np.float64)
    R = _gpu_residual(sy, A, B, X, C)
    m, n = C.shape
    ld = np.longdouble
    idx = rng.integers(0, m, 256), rng.integers(0, n, 256)
    for i, j in zip(*idx):
        a = A[i, max(0, i - 1):].astype(ld)
        b = B[: min(n, j + 2), j].astype(ld)
        ref = ld(C[i, j]) - (a @ X[max(0, i - 1):, j].astype(ld) + X[i, : min(n, j + 2)].astype(ld) @ b)
        scale = np.abs(A[i, max(0, i - 1):]) @ np.abs(X[max(0, i - 1):, j]) + \
            np.abs(X[i, : min(n, j + 2)]) @ np.abs(B[: min(n, j + 2), j])
        assert abs(R[i, j] - float(ref)) <= 2.0 ** -44 * scale + 2.0 ** -52 * abs(float(ref))


def test_subnormal_and_huge_rows(orc, sy):
    """Rows of A in the subnormal range (the splitting reads their bits without the
    hidden bit) and columns of X near 1e300: the residual stays within the row/column
    maximum bound of the oracle's definition."""
    m, n = 150, 90
    rng = np.random.default_rng(17)
    A = np.triu(rng.uniform(-1, 1, (m, m)))
    B = np.triu(rng.uniform(-1, 1, (n, n)))
    A[10:20] *= 1e-310   # subnormal rows (their diagonal entries too)
    A[30] *= 5e-324      # the smallest subnormal scale: entries 0 or +-4.9e-324
    X = rng.uniform(-1, 1, (m, n))
    X[:, 40:45] *= 1e300
    C = rng.uniform(-1, 1, (m, n))
    R = _gpu_residual(sy, A, B, X, C)
    ref = orc.residual_matrix(A, B, X, C)
    assert np.all(np.isfinite(R))
    assert np.all(np.abs(R - ref) <= _rowcol_bound(A, B, X, ref))

"""The seeded input generators shared by the GPU tests and the oracle: the structure of
the paper's matrices (upper quasi-triangular, Sec. 1 eq. (4), with standardized 2x2
diagonal blocks holding complex-conjugate eigenvalues), the stated mix of 1x1 and
2x2 blocks, the scaling of each kind, the Sec. 3 test matrices, reproducibility per
seed, and the batch shape distribution."""
import numpy as np
import pytest

from paper_1905_10574_gb300 import inputs


def pair_starts(T):
    n = T.shape[0]
    return [i for i in range(n - 1) if T[i + 1, i] != 0.0]


@pytest.mark.parametrize("kind", ["benign", "wellcond", "growth"])
def test_quasi_triangular_structure(kind):
    n = 300
    T = inputs.quasi_triangular(n, 7, kind=kind, upper=4.0)
    assert T.dtype == np.float64 and T.flags.f_contiguous
    assert np.all(np.tril(T, -2) == 0.0)
    st = pair_starts(T)
    assert st and all(b - a >= 2 for a, b in zip(st, st[1:]))  # 2x2 blocks never touch
    for i in st:
        a, b, c, d = T[i, i], T[i, i + 1], T[i + 1, i], T[i + 1, i + 1]
        assert a == d and b * c < 0 and 0.5 <= abs(b) <= 2 and 0.5 <= abs(c) <= 2
        assert np.all(np.abs(np.linalg.eigvals(T[i:i + 2, i:i + 2]).imag) > 0)
    assert np.all((np.diag(T) >= 1) & (np.diag(T) <= 10))


def test_half_the_eigenvalues_in_pairs():
    n = 20000
    frac = 2 * len(pair_starts(inputs.quasi_triangular(n, 3))) / n
    assert abs(frac - 0.5) < 0.02


def test_kind_scaling():
    """One seed, three kinds: the same draws, with the strictly upper part outside the
    2x2 blocks scaled by 1, 1/sqrt(n) and `upper`."""
    n = 400
    Tb = inputs.quasi_triangular(n, 11, "benign")
    Tw = inputs.quasi_triangular(n, 11, "wellcond")
    Tg = inputs.quasi_triangular(n, 11, "growth", upper=4.0)
    assert pair_starts(Tb) == pair_starts(Tw) == pair_starts(Tg)
    mask = np.triu(np.ones((n, n), dtype=bool), 1)
    for i in pair_starts(Tb):
        mask[i, i + 1] = False
    assert np.allclose(Tw[mask], Tb[mask] / np.sqrt(n), rtol=1e-15, atol=0)
    assert np.allclose(Tg[mask], 4.0 * Tb[mask], rtol=1e-15, atol=0)
    assert np.array_equal(np.diag(Tb), np.diag(Tw))
    with pytest.raises(ValueError):
        inputs.quasi_triangular(4, 0, "other")


def test_reproducible_and_distinct_streams():
    A1, B1, C1 = inputs.problem(50, 50, 5)
    A2, B2, C2 = inputs.problem(50, 50, 5)
    assert np.array_equal(A1, A2) and np.array_equal(B1, B2) and np.array_equal(C1, C2)
    assert not np.array_equal(A1, B1)
    assert not np.array_equal(A1, inputs.problem(50, 50, 6)[0])
    assert C1.flags.f_contiguous and np.all(np.abs(C1) <= 1)


def test_paper_matrix():
    n, mu = 40, 1e-3
    T = inputs.paper_matrix(n, mu, pairs=[0, 5, 38])
    ones = np.triu(np.ones((n, n)), 1)
    for i in (0, 5, 38):
        ones[i, i + 1] = 0.0
    assert np.array_equal(T * ones, ones)
    assert np.all(np.diag(T) == mu) and np.all(np.tril(T, -2) == 0)
    for i in (0, 5, 38):
        assert T[i, i + 1] == mu and T[i + 1, i] == -mu


def test_batch_shapes():
    sh = inputs.batch_shapes(4096, 16, 512, seed=1234)
    a = np.array(sh)
    assert a.shape == (4096, 2) and a.min() >= 16 and a.max() <= 512
    assert abs(np.median(np.log(a)) - 0.5 * np.log(16 * 512)) < 0.1  # log-uniform
    assert sh == inputs.batch_shapes(4096, 16, 512, seed=1234)


def test_named_workloads():
    for w in inputs.WORKLOADS.values():
        assert w["tile"] in (32, 64) and w["m"] > 0 and w["n"] > 0
    A, B, C, w = inputs.workload("benign_256")
    assert A.shape == B.shape == C.shape == (256, 256) and w["kind"] == "benign"

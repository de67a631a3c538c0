"""GPU parity of sylv_solve_schur, the Bartels-Stewart wrapper (Sec. 1, eqs. (3)-(5)):
dense A = U TA U^T and B = V TB V^T (real Schur forms from scipy on the host), the
library's GEMMs and robust solve on the device, against the oracle's
U (trsyl(TA, TB, U^T C V)) V^T and against the residual of the dense equation."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
sla = pytest.importorskip("scipy.linalg")


@pytest.fixture(scope="module")
def sy():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_10574_gb300 import build, sylv
    build.build()
    sylv.load()
    return sylv


def dev(a):
    return torch.from_numpy(np.asfortranarray(a)).cuda()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def dense_problem(m, n, seed, shift=4.0):
    """Dense A, B with spectra in the right half plane (so A X + X B is well posed),
    their real Schur forms, and C."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, m)) / np.sqrt(m) + shift * np.eye(m)
    B = rng.standard_normal((n, n)) / np.sqrt(n) + shift * np.eye(n)
    C = rng.standard_normal((m, n))
    TA, U = sla.schur(A, output="real")
    TB, V = sla.schur(B, output="real")
    return A, B, C, U, TA, V, TB


@pytest.mark.parametrize("m,n,precision", [(50, 37, "fp64"), (200, 130, "fp64"), (64, 300, "fp64"),
                                           (300, 260, "fp32_refine")])
def test_schur_solve(orc, sy, m, n, precision):
    A, B, C, U, TA, V, TB = dense_problem(m, n, seed=m + n)
    X, res = sy.schur_solve(dev(U), dev(TA), dev(V), dev(TB), dev(C), precision=precision)
    torch.cuda.synchronize()
    X = X.cpu().numpy()
    assert res.info == 0 and res.log2scale == 0
    ref, e = orc.schur_solve(U, TA, V, TB, C)
    assert e == 0
    assert rel(X, ref) <= 1e-12
    R = A @ X + X @ B - C
    assert np.linalg.norm(R) <= 1e-12 * (np.linalg.norm(A) + np.linalg.norm(B)) * np.linalg.norm(X) + \
        1e-12 * np.linalg.norm(C)


def test_schur_solve_sign_variant(orc, sy):
    """A X - X B = C with B = -B0 (spectrum in the left half plane)."""
    A, B0, C, U, TA, V, TB0 = dense_problem(90, 70, seed=4)
    X, res = sy.schur_solve(dev(U), dev(TA), dev(V), dev(-TB0), dev(C), isgn=-1)
    torch.cuda.synchronize()
    X = X.cpu().numpy()
    assert res.info == 0
    ref, _ = orc.schur_solve(U, TA, V, -TB0, C, isgn=-1)
    assert rel(X, ref) <= 1e-12
    assert rel(A @ X - X @ (-B0), C) <= 1e-12


def test_schur_solve_arguments(sy):
    d = torch.zeros((4, 4), dtype=torch.float64, device="cuda")
    p = d.data_ptr()
    res = sy.sylv_result()
    assert sy.sylv_solve_schur(-1, 4, p, 4, p, 4, p, 4, p, 4, p, 4, None, res) == -1
    assert sy.sylv_solve_schur(4, 4, 0, 4, p, 4, p, 4, p, 4, p, 4, None, res) == -3
    assert sy.sylv_solve_schur(4, 4, p, 4, 0, 4, p, 4, p, 4, p, 4, None, res) == -5
    assert sy.sylv_solve_schur(4, 4, p, 4, p, 4, 0, 4, p, 4, p, 4, None, res) == -7
    assert sy.sylv_solve_schur(4, 4, p, 4, p, 4, p, 4, p, 2, p, 4, None, res) == -10
    assert sy.sylv_solve_schur(4, 4, p, 4, p, 4, p, 4, p, 4, p, 2, None, res) == -12
    o = sy.make_opts(transa=True)
    assert sy.sylv_solve_schur(4, 4, p, 4, p, 4, p, 4, p, 4, p, 4, o, res) == sy.SYLV_ERR_UNSUPPORTED
    assert sy.sylv_solve_schur(0, 4, p, 1, p, 1, p, 4, p, 4, p, 1, None, res) == 0

"""GPU tests of the solver's variants beyond the paper's equation: the sign variant
op(A) Y - Y op(B) = alpha C (LAPACK's ISGN = -1) and the SM cap of the persistent
tile kernel (for SM-scaling measurements).

The sign variant is checked against the oracle's Kronecker solve of the signed
equation, and bitwise against the +1 solve with -B (negation is exact, so both run
the same arithmetic).  Test matrices take B with eigenvalues of negative real part,
so that A Y - Y B is as well conditioned as the paper's A Y + Y B.
"""
import ctypes

import numpy as np
import pytest

from paper_1905_10574_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

FWD_TOL = 1e-13  # FP64 results: Y/alpha against the oracle, relative Frobenius norm
REFINE_TOL = 1e-12  # FP32 + refinement: forward error after refinement


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


def solve(sy, A, B, C, **kw):
    Y, res = sy.solve(dev(A), dev(B), dev(C), **kw)
    torch.cuda.synchronize()
    return Y.cpu().numpy(), res


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def signed_problem(m, n, seed):
    A, Bg, C = inputs.problem(m, n, seed, kind="wellcond")
    return A, -Bg, C, Bg  # A Y - Y (-Bg) = C is A Y + Y Bg = C


@pytest.mark.parametrize("m,n,tile", [(70, 45, 32), (130, 97, 24), (64, 200, 0)])
def test_sign_variant(orc, sy, m, n, tile):
    A, B, C, Bg = signed_problem(m, n, seed=m + n)
    Y, res = solve(sy, A, B, C, isgn=-1, tile=tile)
    Yp, resp = solve(sy, A, Bg, C, tile=tile)
    assert res.info == 0 and res.log2scale == resp.log2scale
    assert np.array_equal(Y, Yp)  # the same arithmetic on -(-Bg) = Bg
    if m * n <= 4000:
        ref = orc.kron_solve(A, B, C, isgn=-1)
        assert rel(Y, ref) <= FWD_TOL
    ref = orc.trsyl(A, Bg, C)
    assert rel(np.ldexp(Y, int(ref["log2scale"]) - int(res.log2scale)), ref["Y"]) <= FWD_TOL


def test_sign_variant_transposed(orc, sy):
    A, B, C, _ = signed_problem(40, 33, seed=5)
    Y, res = solve(sy, A, B, C, isgn=-1, transa=True, transb=True)
    assert res.info == 0
    ref = orc.kron_solve(A, B, C, transa=True, transb=True, isgn=-1)
    assert rel(Y, ref) <= FWD_TOL


def test_sign_variant_mixed_precision(orc, sy):
    A, B, C, Bg = signed_problem(300, 260, seed=8)
    Y, res = solve(sy, A, B, C, isgn=-1, precision="fp32_refine")
    Y64, _ = solve(sy, A, B, C, isgn=-1)
    assert res.info == 0 and res.iters >= 1
    assert rel(Y, Y64) <= REFINE_TOL


def test_sign_variant_batched(sy):
    probs = [signed_problem(m, n, seed=i) for i, (m, n) in enumerate([(20, 30), (64, 17), (100, 100), (33, 95)])]
    As = [dev(p[0]) for p in probs]
    Bs = [dev(p[1]) for p in probs]
    Cs = [dev(p[2]) for p in probs]
    Ys, res = sy.batch_solve(As, Bs, Cs, isgn=-1)
    torch.cuda.synchronize()
    for (A, B, C, _), Yb, r in zip(probs, Ys, res):
        Y, r1 = solve(sy, A, B, C, isgn=-1)
        assert r.info == 0 and r.log2scale == r1.log2scale
        assert np.array_equal(Yb.cpu().numpy(), Y)


def test_sign_variant_adjoint(orc, sy):
    """dA, dB, dC of L = sum(W Y) for A Y - Y B = C against the oracle's Kronecker
    gradient of the signed equation."""
    rng = np.random.default_rng(3)
    m, n = 9, 7
    A, B, C, _ = signed_problem(m, n, seed=21)
    W = rng.uniform(-1, 1, (m, n))
    Ad, Bd = dev(A), dev(B)
    Y = dev(C).clone()
    o = sy.make_opts(isgn=-1)
    res = sy.sylv_result()
    rc = sy.sylv_tri_solve_ex(m, n, Ad.data_ptr(), m, Bd.data_ptr(), n, Y.data_ptr(), m, o, res)
    assert rc == 0 and res.log2scale == 0
    G = dev(W).clone()
    dA = torch.zeros((m, m), dtype=torch.float64, device="cuda").t()
    dB = torch.zeros((n, n), dtype=torch.float64, device="cuda").t()
    r2 = sy.sylv_result()
    rc = sy.sylv_tri_solve_backward(m, n, Ad.data_ptr(), m, Bd.data_ptr(), n, Y.data_ptr(), m, res.log2scale,
                                    G.data_ptr(), m, dA.data_ptr(), m, dB.data_ptr(), n, o, r2)
    torch.cuda.synchronize()
    assert rc == 0
    rA, rB, rC, X = orc.kron_grad(A, B, C, W, isgn=-1)
    assert rel(Y.cpu().numpy(), X) <= FWD_TOL
    assert rel(G.cpu().numpy(), rC) <= FWD_TOL
    assert rel(dA.cpu().numpy(), rA) <= 1e-11
    assert rel(dB.cpu().numpy(), rB) <= 1e-11


@pytest.mark.parametrize("sms", [1, 3, 17])
def test_sm_cap_is_bitwise_identical(sy, sms):
    """Capping the persistent grid changes which CTA owns which tile, never the order
    of a tile's updates: the solution is bitwise the uncapped one."""
    A, B, C = inputs.problem(300, 260, seed=31, kind="growth", upper=4.0)
    Y, res = solve(sy, A, B, C)
    Yc, resc = solve(sy, A, B, C, max_sms=sms)
    assert res.info == resc.info and res.log2scale == resc.log2scale
    assert np.array_equal(Y, Yc)


def test_option_validation(sy):
    o = sy.make_opts()
    o.isgn = 2
    d = torch.zeros((4, 4), dtype=torch.float64, device="cuda")
    res = sy.sylv_result()
    p = d.data_ptr()
    assert sy.sylv_tri_solve_ex(4, 4, p, 4, p, 4, p, 4, o, res) == sy.SYLV_ERR_UNSUPPORTED
    o.isgn = 1
    o.max_sms = -1
    assert sy.sylv_tri_solve_ex(4, 4, p, 4, p, 4, p, 4, o, res) == sy.SYLV_ERR_UNSUPPORTED


def tri_solve(sy, A, C, **kw):
    X, res = sy.triangular_solve(dev(A), dev(C), **kw)
    torch.cuda.synchronize()
    return X.cpu().numpy(), res


@pytest.mark.parametrize("m,n,tile", [(70, 5, 32), (257, 1, 32), (130, 200, 24), (33, 64, 0), (400, 37, 64)])
def test_triangular_solve(orc, sy, m, n, tile):
    A, _, C = inputs.problem(m, n, seed=m + 7 * n, kind="wellcond")
    X, res = tri_solve(sy, A, C, tile=tile)
    assert res.info == 0 and res.log2scale == 0
    ref = orc.trsyl(A, np.zeros((n, n)), C)
    assert rel(X, ref["Y"]) <= FWD_TOL
    assert rel(X, np.linalg.solve(np.triu(A, -1), C)) <= 1e-11


def test_triangular_solve_transposed(orc, sy):
    A, _, C = inputs.problem(150, 20, seed=4, kind="wellcond")
    X, res = tri_solve(sy, A, C, transa=True)
    assert res.info == 0
    assert rel(X, orc.trsyl(A, np.zeros((20, 20)), C, transa=True)["Y"]) <= FWD_TOL


def test_triangular_solve_scaling(orc, sy):
    """Growth past the binary64 range: the robust solve scales (alpha < 1, finite X,
    Y/alpha equal to the oracle's after a common power-of-two shift), the plain one
    overflows."""
    A, _, C = inputs.problem(500, 12, seed=2, kind="growth", upper=200.0)  # oracle: alpha = 2^-613
    X, res = tri_solve(sy, A, C)
    ref = orc.trsyl(A, np.zeros((12, 12)), C)
    assert res.info in (0, 2) and res.log2scale < 0 and ref["log2scale"] < 0
    assert np.all(np.isfinite(X)) and np.max(np.abs(X)) <= 2.0 ** 1020
    Xs = np.ldexp(X, int(ref["log2scale"]) - int(res.log2scale))
    s = np.max(np.abs(ref["Y"]))  # entries near 2^1016: normalise before the norm
    assert rel(Xs / s, ref["Y"] / s) <= FWD_TOL
    _, res_nr = tri_solve(sy, A, C, precision="fp64_nonrobust", check=False)
    assert res_nr.info == sy.SYLV_OVERFLOWED


def test_triangular_solve_arguments(sy):
    d = torch.zeros((4, 4), dtype=torch.float64, device="cuda")
    p = d.data_ptr()
    res = sy.sylv_result()
    assert sy.sylv_tri_solve_triangular(-1, 4, p, 4, p, 4, None, res) == -1
    assert sy.sylv_tri_solve_triangular(4, 4, 0, 4, p, 4, None, res) == -3
    assert sy.sylv_tri_solve_triangular(4, 4, p, 4, p, 2, None, res) == -6
    o = sy.make_opts(precision="fp32_refine")
    assert sy.sylv_tri_solve_triangular(4, 4, p, 4, p, 4, o, res) == sy.SYLV_ERR_UNSUPPORTED
    assert sy.sylv_tri_solve_triangular(0, 4, p, 1, p, 1, None, res) == 0

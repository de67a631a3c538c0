"""GPU parity at the benchmark's full sizes, in the launch configuration bench.py
times (tile 32, robust FP64; FP32 + refinement; the 4096-equation batch).

The oracle cannot solve m = n = 4000 or 8000 in test time, but the bottom-left
block Y[m-b:, :b] of the solution depends only on A[m-b:, m-b:], B[:b, :b] and
C[m-b:, :b] (A and B are upper quasi-triangular, so the block equation of that
corner involves nothing else): it is the solution of an independent b x b
equation that the oracle solves in seconds.  The GPU's corner, shifted by the
difference of the two scale exponents, must match it.  The residual of eq. (9)
of the whole GPU solution is evaluated on the host where it is affordable.
"""
import numpy as np
import pytest

from paper_1905_10574_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

FWD_TOL = 1e-13  # FP64: Y/alpha against the oracle (relative Frobenius norm)
REFINE_TOL = 1e-12  # FP32 + refinement: forward error after refinement
RESID_TOL = 1e-13


@pytest.fixture(scope="module")
def sy():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_10574_gb300 import build, sylv
    build.build()
    sylv.load()
    return sylv


def _rel(a, b):
    s = max(float(np.max(np.abs(a))), float(np.max(np.abs(b))))
    e = -int(np.frexp(s)[1]) if s > 0 else 0
    a2, b2 = np.ldexp(a, e), np.ldexp(b, e)
    return float(np.linalg.norm(a2 - b2) / np.linalg.norm(b2))


def _corner(orc, A, B, C, b):
    """Oracle solution of the bottom-left b x b corner equation."""
    m = A.shape[0]
    r0 = m - b
    # do not cut a 2x2 block of A at row r0 or of B at column b
    if A[r0, r0 - 1] != 0.0:
        r0 -= 1
    cb = b + 1 if B[b, b - 1] != 0.0 else b
    out = orc.trsyl(A[r0:, r0:], B[:cb, :cb], C[r0:, :cb])
    return r0, cb, out


def _gpu(sy, A, B, C, **kw):
    Y, res = sy.solve(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), torch.from_numpy(C).cuda(), **kw)
    torch.cuda.synchronize()
    return Y.cpu().numpy(), res


def test_overflow_4000_full_size(orc, sy):
    A, B, C, w = inputs.workload("overflow_4000")
    Y, res = _gpu(sy, A, B, C, tile=w["tile"])
    assert res.info == 0 and res.log2scale < 0
    assert np.all(np.isfinite(Y)) and np.max(np.abs(Y)) <= 2.0 ** 1020
    r0, cb, ref = _corner(orc, A, B, C, 400)
    Yc = np.ldexp(Y[r0:, :cb], int(ref["log2scale"]) - int(res.log2scale))
    assert _rel(Yc, ref["Y"]) <= FWD_TOL
    assert orc.residual(A, B, Y, C, res.log2scale) <= RESID_TOL
    _, res_nr = _gpu(sy, A, B, C, tile=w["tile"], precision="fp64_nonrobust", check=False)
    assert res_nr.info == sy.SYLV_OVERFLOWED


@pytest.mark.parametrize("tol", [0.0, 2.0 ** -41])
@pytest.mark.parametrize("name", ["wellcond_4000", "wellcond_8000"])
def test_mixed_full_size(orc, sy, name, tol):
    """FP32 + refinement at full size: the corner against the oracle, and every entry
    against the robust FP64 solve (itself within ~1e-15 of the oracle, so the
    comparison measures the refined solution's own error), both within 1e-12; the
    eq. (9) residual of the whole refined solution, evaluated on the host by the
    oracle, within 1e-13.  The library's default stop tolerance (2^-43) and the
    benchmark's (2^-41, chosen for the 1e-12 forward-error target) are both checked."""
    A, B, C, w = inputs.workload(name)
    Y, res = _gpu(sy, A, B, C, tile=w["tile"], precision="fp32_refine", tol=tol)
    assert res.info == 0 and res.log2scale == 0
    assert res.iters >= 2 and res.last_update <= (tol or 2.0 ** -43)
    r0, cb, ref = _corner(orc, A, B, C, 300)
    assert ref["log2scale"] == 0
    assert _rel(Y[r0:, :cb], ref["Y"]) <= REFINE_TOL
    assert orc.residual(A, B, Y, C, 0) <= RESID_TOL
    Y64, res64 = _gpu(sy, A, B, C, tile=w["tile"])
    assert res64.info == 0 and res64.log2scale == 0
    assert _rel(Y, Y64) <= REFINE_TOL


@pytest.mark.parametrize("precision", ["fp64", "fp32_refine"])
def test_batched_4096_sampled(orc, sy, precision):
    """The 4096-equation batch as the benchmark runs it, in FP64 and in FP32 +
    refinement at the benchmark's stop tolerance (2^-41): 24 sampled equations
    against the oracle (FP64 1e-13, refined 1e-12) and their eq. (9) residuals."""
    shapes = inputs.batch_shapes(4096, 16, 512, seed=1234)
    probs = [inputs.problem(m, n, 10000 + i, kind="wellcond") for i, (m, n) in enumerate(shapes)]
    As = [torch.from_numpy(p[0]).cuda() for p in probs]
    Bs = [torch.from_numpy(p[1]).cuda() for p in probs]
    Cs = [torch.from_numpy(p[2]).cuda() for p in probs]
    refine = precision == "fp32_refine"
    Ys, res = sy.batch_solve(As, Bs, Cs, precision=precision, tol=2.0 ** -41 if refine else 0.0)
    torch.cuda.synchronize()
    assert all(r.info == 0 for r in res)
    if refine:
        assert all(r.iters >= 2 and r.last_update <= 2.0 ** -41 for r in res)
    tol = REFINE_TOL if refine else FWD_TOL
    rng = np.random.default_rng(0)
    for i in rng.choice(len(probs), size=24, replace=False):
        A, B, C = probs[i]
        Yh = Ys[i].cpu().numpy()
        assert np.all(np.isfinite(Yh))
        ref = orc.trsyl(A, B, C)
        assert orc.residual(A, B, Yh, C, res[i].log2scale) <= RESID_TOL
        assert _rel(np.ldexp(Yh, int(ref["log2scale"]) - int(res[i].log2scale)), ref["Y"]) <= tol


def test_lyapunov_adjoint_256x512_sampled(orc, sy):
    """The differentiation workload at full size: 256 Lyapunov-type equations
    A Y + Y A^T = C with m = n = 512, forward and hand-written adjoint through the
    batched autograd Function, as the benchmark times them.  C is symmetrised so that
    Y = Y^T must hold (a property of the equation at any size).  On sampled instances:
    Y against the oracle; the adjoint Gamma = dL/dC against the oracle's solve of
    A^T Gamma + Gamma A = W; dA against central differences of the loss (h = 1e-6)."""
    count, m = 256, 512
    As = [inputs.quasi_triangular(m, 20000 + i, kind="wellcond") for i in range(count)]
    Cs = [inputs.rhs(m, m, 30000 + i) for i in range(count)]
    Cs = [(c + c.T) / 2 for c in Cs]
    Ws = [inputs.rhs(m, m, 40000 + i) for i in range(count)]
    At = sy.batch_fortran(torch.from_numpy(np.stack(As)).cuda()).requires_grad_(True)
    Ct = sy.batch_fortran(torch.from_numpy(np.stack(Cs)).cuda()).requires_grad_(True)
    Wt = sy.batch_fortran(torch.from_numpy(np.stack(Ws)).cuda())
    Y = sy.BatchSylvesterSolve.apply(At, At, Ct, False, True, 0)
    (Wt * Y).sum().backward()
    torch.cuda.synchronize()
    Yh = Y.detach().cpu().numpy()
    dA = At.grad.cpu().numpy()
    dC = Ct.grad.cpu().numpy()
    assert np.all(np.isfinite(Yh)) and np.all(np.isfinite(dA)) and np.all(np.isfinite(dC))
    for i in range(count):  # P8: symmetric C gives a symmetric solution
        assert _rel(Yh[i].T, Yh[i]) <= FWD_TOL
    rng = np.random.default_rng(5)
    for i in rng.choice(count, size=3, replace=False):
        A, C, W = As[i], Cs[i], Ws[i]
        ref = orc.trsyl(A, A, C, transb=True)
        assert ref["log2scale"] == 0
        assert _rel(Yh[i], ref["Y"]) <= FWD_TOL
        assert orc.residual(A, A, Yh[i], C, 0, False, True) <= RESID_TOL
        adj = orc.trsyl(A, A, W, transa=True)
        assert adj["log2scale"] == 0
        assert _rel(dC[i], adj["Y"]) <= FWD_TOL
        h = 1e-6
        for r, c in [(0, m - 1), (100, 101), (300, 300), (511, 511)]:
            if r > c + 1 or (r == c + 1 and A[r, c] == 0.0):
                continue
            E = np.zeros_like(A)
            E[r, c] = h
            Yp, _ = _gpu(sy, A + E, A + E, C, transb=True)
            Ym, _ = _gpu(sy, A - E, A - E, C, transb=True)
            fd = float(np.sum(W * (Yp - Ym))) / (2 * h)
            assert abs(dA[i][r, c] - fd) <= 1e-6 * max(1.0, abs(fd)), (i, r, c, dA[i][r, c], fd)

"""Batched FP32 + refinement: many uneven equations refined in one launch sequence
(binary32 robust correction solves, binary64-accurate residuals), each equation
stopping on its own tolerance test.  Every result is checked against the FP64
oracle: forward error of Y <= 1e-12 (the refinement's target) on well-conditioned
inputs, and the eq. (9) residual <= 1e-13."""
import numpy as np
import pytest

from paper_1905_10574_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

REFINE_TOL = 1e-12
RESID_TOL = 1e-13
FWD_TOL = 1e-13


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


def host(t):
    return t.cpu().numpy()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_batched_refine_uneven(orc, sy):
    shapes = inputs.batch_shapes(30, 16, 300, seed=41)
    probs = [inputs.problem(m, n, 500 + i, kind="wellcond") for i, (m, n) in enumerate(shapes)]
    Ys, res = sy.batch_solve([dev(p[0]) for p in probs], [dev(p[1]) for p in probs], [dev(p[2]) for p in probs],
                             precision="fp32_refine")
    torch.cuda.synchronize()
    for (A, B, C), Y, r in zip(probs, Ys, res):
        assert r.info == 0 and r.log2scale == 0, r
        assert 2 <= r.iters <= 6 and r.last_update <= 2.0 ** -43
        Yh = host(Y)
        ref = orc.trsyl(A, B, C)
        assert rel(Yh, ref["Y"]) <= REFINE_TOL
        assert orc.residual(A, B, Yh, C, 0) <= RESID_TOL


def test_batched_refine_matches_single_equation_refine(sy):
    """The batch runs each equation's refinement with the same arithmetic as the
    single-equation FP32 + refinement path on the double-float residual: the same
    number of corrections and the same solution to rounding."""
    shapes = [(40, 70), (129, 64), (16, 16), (200, 33)]
    probs = [inputs.problem(m, n, 900 + i, kind="wellcond") for i, (m, n) in enumerate(shapes)]
    Ys, res = sy.batch_solve([dev(p[0]) for p in probs], [dev(p[1]) for p in probs], [dev(p[2]) for p in probs],
                             precision="fp32_refine", tile=32)
    torch.cuda.synchronize()
    for (A, B, C), Y, r in zip(probs, Ys, res):
        Y1, r1 = sy.solve(dev(A), dev(B), dev(C), precision="fp32_refine", tile=32)
        torch.cuda.synchronize()
        assert r.info == r1.info == 0
        assert rel(host(Y), host(Y1)) <= REFINE_TOL


@pytest.mark.parametrize("transa,transb,isgn", [(True, False, 1), (False, True, 1), (True, True, -1)])
def test_batched_refine_transposes_and_sign(orc, sy, transa, transb, isgn):
    shapes = inputs.batch_shapes(8, 16, 150, seed=43 + isgn)
    probs = []
    for i, (m, n) in enumerate(shapes):
        A, B, C = inputs.problem(m, n, 600 + i, kind="wellcond")
        probs.append((A, -B if isgn < 0 else B, C))
    Ys, res = sy.batch_solve([dev(p[0]) for p in probs], [dev(p[1]) for p in probs], [dev(p[2]) for p in probs],
                             precision="fp32_refine", transa=transa, transb=transb, isgn=isgn)
    torch.cuda.synchronize()
    for (A, B, C), Y, r in zip(probs, Ys, res):
        assert r.info == 0, r
        ref = orc.trsyl(A, -B if isgn < 0 else B, C, transa=transa, transb=transb)
        assert rel(host(Y), ref["Y"]) <= REFINE_TOL


def test_batched_refine_cuda_graph_replay(orc, sy):
    """A refined batch captured once in a CUDA graph and replayed twice (right-hand
    sides refilled before each replay) gives the oracle's solutions both times."""
    shapes = inputs.batch_shapes(10, 16, 200, seed=47)
    probs = [inputs.problem(m, n, 700 + i, kind="wellcond") for i, (m, n) in enumerate(shapes)]
    As = [dev(p[0]) for p in probs]
    Bs = [dev(p[1]) for p in probs]
    C0 = [dev(p[2]) for p in probs]
    Cs = [c.clone() for c in C0]
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        o = sy.make_opts(stream=stream.cuda_stream, precision="fp32_refine")
        plan = sy.sylv_batch_create([m for m, _ in shapes], [n for _, n in shapes], [a.data_ptr() for a in As],
                                    [a.stride(1) for a in As], [b.data_ptr() for b in Bs], [b.stride(1) for b in Bs],
                                    [c.data_ptr() for c in Cs], [c.stride(1) for c in Cs], o)
        assert sy.sylv_batch_execute(plan, stream.cuda_stream) == 0
        stream.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            assert sy.sylv_batch_execute(plan, torch.cuda.current_stream().cuda_stream) == 0
    try:
        for _ in range(2):
            for c, c0 in zip(Cs, C0):
                c.copy_(c0)
            g.replay()
            torch.cuda.synchronize()
            rc, res = sy.sylv_batch_results(plan, len(shapes))
            assert rc == 0
            for (A, B, C), Y, r in zip(probs, Cs, res):
                assert r.info == 0 and r.iters >= 2
                assert rel(host(Y), orc.trsyl(A, B, C)["Y"]) <= REFINE_TOL
    finally:
        sy.sylv_batch_destroy(plan)


def test_adjoint_in_refined_precision(orc, sy):
    """The backward entry points with FP32 + refinement: the adjoint solve is refined
    like a forward one, and the gradients match the oracle's Kronecker form."""
    m, n = 14, 11
    A, B, C = inputs.problem(m, n, 71, kind="wellcond")
    W = inputs.rhs(m, n, 72)
    rA, rB, rC, X = orc.kron_grad(A, B, C, W)
    Ad, Bd, Y = dev(A), dev(B), dev(X)
    o = sy.make_opts(precision="fp32_refine")
    G = dev(W).clone()
    dA = torch.zeros((m, m), dtype=torch.float64, device="cuda").t()
    dB = torch.zeros((n, n), dtype=torch.float64, device="cuda").t()
    r = sy.sylv_result()
    rc = sy.sylv_tri_solve_backward(m, n, Ad.data_ptr(), m, Bd.data_ptr(), n, Y.data_ptr(), m, 0, G.data_ptr(), m,
                                    dA.data_ptr(), m, dB.data_ptr(), n, o, r)
    torch.cuda.synchronize()
    assert rc == 0 and r.iters >= 2
    assert rel(host(G), rC) <= REFINE_TOL
    assert rel(host(dA), rA) <= REFINE_TOL
    assert rel(host(dB), rB) <= REFINE_TOL
    Gs = [dev(W).clone() for _ in range(2)]
    dAs = [torch.zeros((m, m), dtype=torch.float64, device="cuda").t() for _ in range(2)]
    dBs = [torch.zeros((n, n), dtype=torch.float64, device="cuda").t() for _ in range(2)]
    rc, rs = sy.sylv_tri_solve_backward_batched([m] * 2, [n] * 2, [Ad.data_ptr()] * 2, [m] * 2, [Bd.data_ptr()] * 2,
                                                [n] * 2, [Y.data_ptr()] * 2, [m] * 2, [0, 0],
                                                [g.data_ptr() for g in Gs], [m] * 2, [d.data_ptr() for d in dAs],
                                                [m] * 2, [d.data_ptr() for d in dBs], [n] * 2, o)
    torch.cuda.synchronize()
    assert rc == 0 and all(x.iters >= 2 for x in rs)
    for i in range(2):
        assert rel(host(Gs[i]), rC) <= REFINE_TOL
        assert rel(host(dAs[i]), rA) <= REFINE_TOL
        assert rel(host(dBs[i]), rB) <= REFINE_TOL


def test_batched_refine_degenerate_and_unconverged(orc, sy):
    """Single-row and single-column equations in a refined batch converge like the
    others; with maxit = 1 no equation can pass the stop test, so each reports
    SYLV_NOT_CONVERGED and returns its first (binary32-accurate) solution."""
    shapes = [(1, 5), (40, 30), (7, 1), (64, 65)]
    probs = [inputs.problem(m, n, 950 + i, kind="wellcond") for i, (m, n) in enumerate(shapes)]
    Ys, res = sy.batch_solve([dev(p[0]) for p in probs], [dev(p[1]) for p in probs], [dev(p[2]) for p in probs],
                             precision="fp32_refine")
    torch.cuda.synchronize()
    for (A, B, C), Y, r in zip(probs, Ys, res):
        assert r.info == 0, r
        assert rel(host(Y), orc.trsyl(A, B, C)["Y"]) <= REFINE_TOL
    Ys, res = sy.batch_solve([dev(p[0]) for p in probs], [dev(p[1]) for p in probs], [dev(p[2]) for p in probs],
                             precision="fp32_refine", maxit=1)
    torch.cuda.synchronize()
    for (A, B, C), Y, r in zip(probs, Ys, res):
        assert r.info == sy.SYLV_NOT_CONVERGED and r.iters == 1, r
        err = rel(host(Y), orc.trsyl(A, B, C)["Y"])
        assert err <= 1e-4  # binary32-accurate, not refined

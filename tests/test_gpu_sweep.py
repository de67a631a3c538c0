"""Seeded randomised parity sweep of the single-equation solve against the oracle.

400 equations drawn from one seeded stream: m, n in [1, 160], tile in {auto, 16, 24,
32, 48, 64}, both transposes, the benign / wellcond / growth generators (strictly-upper
scale up to 1e3, so alpha stays within the binary64 range where the oracle's Y/alpha
is the reference; below it see test_gpu_solve's decimal test), and the three
precisions (robust FP64; FP32 + refinement and the non-robust Algorithm 1 on the
non-growth inputs).  Each case checks the status, the eq. (9) residual, the
normwise forward error against the oracle (non-growth), and every normal entry of
Y/alpha against the oracle's within 100 times the oracle's own sensitivity to
relative perturbations of 1e-15 in A and B (at least 1e-12).  The batched launch is
swept the same way: batches of 8 to 60 equations with mixed sizes, generators and
tiles, FP64 and FP32 + refinement, with transposes."""
import numpy as np
import pytest

from paper_1905_10574_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

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
    s = max(float(np.max(np.abs(a))) if a.size else 0.0, float(np.max(np.abs(b))) if b.size else 0.0)
    e = -int(np.frexp(s)[1]) if s > 0 else 0
    a2, b2 = np.ldexp(a, e), np.ldexp(b, e)
    d = np.linalg.norm(b2)
    return float(np.linalg.norm(a2 - b2) / (d if d else 1.0))


def _cases(count=400, seed=20260):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        m, n = int(rng.integers(1, 161)), int(rng.integers(1, 161))
        tile = int(rng.choice([0, 16, 24, 32, 48, 64]))
        kind = str(rng.choice(["benign", "wellcond", "growth", "growth"]))
        upper = float(rng.choice([3.0, 30.0, 1e3])) if kind == "growth" else 1.0
        ta, tb = bool(rng.integers(0, 2)), bool(rng.integers(0, 2))
        prec = str(rng.choice(["fp64", "fp64", "fp32_refine", "fp64_nonrobust"]))
        if kind == "growth":
            prec = "fp64"
        out.append((m, n, tile, kind, upper, ta, tb, prec, int(rng.integers(0, 10 ** 6))))
    return out


def _check(orc, rng, case, A, B, C, Y, res, failures):
    m, n, tile, kind, upper, ta, tb, prec, seed = case
    ref = orc.trsyl(A, B, C, transa=ta, transb=tb)
    assert ref["info"] == 0 and ref["log2scale"] >= -1074, case
    if res.info != 0:
        failures.append((case, "info", res.info))
        return
    r = orc.residual(A, B, Y, C, res.log2scale, ta, tb)
    Yr = np.ldexp(Y, int(ref["log2scale"]) - int(res.log2scale))
    Yo = ref["Y"]
    if r > RESID_TOL:
        failures.append((case, "residual", r))
    if kind != "growth":
        tol = 1e-12 if prec == "fp32_refine" else 1e-13
        fwd = _rel(Yr, Yo)
        if fwd > tol:
            failures.append((case, "forward", fwd))
    elif m and n:
        Ap = A * (1 + 1e-15 * rng.standard_normal(A.shape))
        Bp = B * (1 + 1e-15 * rng.standard_normal(B.shape))
        r2 = orc.trsyl(Ap, Bp, C, transa=ta, transb=tb)
        Y2 = np.ldexp(r2["Y"], int(ref["log2scale"]) - int(r2["log2scale"]))
        mask = (np.abs(Yo) > 2.0 ** -900) & (np.abs(Yr) > 2.0 ** -900) & (np.abs(Y2) > 2.0 ** -900)
        if mask.any():
            cw = float(np.max(np.abs(Yr - Yo)[mask] / np.abs(Yo)[mask]))
            pert = float(np.max(np.abs(Y2 - Yo)[mask] / np.abs(Yo)[mask]))
            if cw > max(1e-12, 100 * pert):
                failures.append((case, "entrywise", cw, pert))


def _dev(a):
    return torch.from_numpy(np.asfortranarray(a)).cuda()


def test_random_sweep_against_oracle(orc, sy):
    rng = np.random.default_rng(7)
    failures = []
    for case in _cases():
        m, n, tile, kind, upper, ta, tb, prec, seed = case
        A, B, C = inputs.problem(m, n, seed, kind=kind, upper=upper)
        Yt, res = sy.solve(_dev(A), _dev(B), _dev(C), transa=ta, transb=tb, precision=prec, tile=tile)
        torch.cuda.synchronize()
        _check(orc, rng, case, A, B, C, Yt.cpu().numpy(), res, failures)
    assert not failures, failures[:5]


def test_random_batches_against_oracle(orc, sy):
    rng = np.random.default_rng(20261)
    failures = []
    for b in range(8):
        prec = "fp64" if b % 2 == 0 else "fp32_refine"
        ta, tb = bool(rng.integers(0, 2)), bool(rng.integers(0, 2))
        tile = int(rng.choice([0, 16, 32, 64]))
        probs = []
        for _ in range(int(rng.integers(8, 61))):
            m, n = int(rng.integers(1, 201)), int(rng.integers(1, 201))
            kinds = ["benign", "wellcond", "growth"] if prec == "fp64" else ["benign", "wellcond"]
            kind = str(rng.choice(kinds))
            upper = float(rng.choice([3.0, 30.0, 1e3])) if kind == "growth" else 1.0
            seed = int(rng.integers(0, 10 ** 6))
            probs.append(((m, n, tile, kind, upper, ta, tb, prec, seed),) + inputs.problem(m, n, seed, kind, upper))
        Ys, rs = sy.batch_solve([_dev(p[1]) for p in probs], [_dev(p[2]) for p in probs],
                                [_dev(p[3]) for p in probs], transa=ta, transb=tb, tile=tile, precision=prec)
        torch.cuda.synchronize()
        for (case, A, B, C), Yt, res in zip(probs, Ys, rs):
            _check(orc, rng, case, A, B, C, Yt.cpu().numpy(), res, failures)
    assert not failures, failures[:5]

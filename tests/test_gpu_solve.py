"""GPU parity: the CUDA library (through the C ABI) against the FP64 CPU oracle.

Tolerances (FP64): the relative residual of eq. (9) must be <= 1e-13, and Y/alpha
must agree with the oracle's Y/alpha to 1e-13 in the Frobenius norm on inputs
whose condition keeps the forward error of a backward-stable solver near
machine precision (the oracle and the GPU round differently: different
summation orders in the tile updates, multiplication by powers of two in
different places).  Where Y/alpha overflows (the growth workloads), the two
alpha-scaled results are compared after a common power-of-two shift.  Results of
FP32 + refinement are held to the 1e-12 forward error that refinement targets.
"""
import math

import numpy as np
import pytest

from paper_1905_10574_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

RESID_TOL = 1e-13
FWD_TOL = 1e-13
REFINE_TOL = 1e-12


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


def gpu_solve(sy, A, B, C, **kw):
    Y, res = sy.solve(dev(A), dev(B), dev(C), **kw)
    torch.cuda.synchronize()
    return host(Y), res


def rel(a, b):
    """||a - b||_F / ||b||_F, evaluated on a common power-of-two rescaling (entries
    near 2^1020 would overflow the squares)."""
    s = max(float(np.max(np.abs(a))) if a.size else 0.0, float(np.max(np.abs(b))) if b.size else 0.0)
    e = -int(np.frexp(s)[1]) if s > 0 else 0
    a2, b2 = np.ldexp(a, e), np.ldexp(b, e)
    d = np.linalg.norm(b2)
    return float(np.linalg.norm(a2 - b2) / (d if d else 1.0))


def shifted(Y, e_from, e_to):
    """Y * 2^(e_to - e_from): the same augmented tile at another scale."""
    return np.ldexp(Y, int(e_to) - int(e_from))


def check_against_oracle(orc, sy, A, B, C, fwd_tol=FWD_TOL, **kw):
    Y, res = gpu_solve(sy, A, B, C, **kw)
    ta, tb = kw.get("transa", False), kw.get("transb", False)
    ref = orc.trsyl(A, B, C, transa=ta, transb=tb)
    assert res.info == 0, res
    assert np.all(np.isfinite(Y))
    r = orc.residual(A, B, Y, C, res.log2scale, ta, tb)
    assert r <= RESID_TOL, r
    err = rel(shifted(Y, res.log2scale, ref["log2scale"]), ref["Y"])
    assert err <= fwd_tol, err
    return Y, res, ref


def test_config1_benign_256_tile64(orc, sy):
    """m = n = 256, tile 64, ~50% of eigenvalues in 2x2 blocks, seed 0."""
    A, B, C = inputs.problem(256, 256, 0, kind="benign")
    Y, res, ref = check_against_oracle(orc, sy, A, B, C, tile=64)
    assert res.log2scale == 0 == ref["log2scale"]


@pytest.mark.parametrize("m,n,tile", [(1, 1, 0), (1, 9, 32), (9, 1, 32), (2, 2, 32), (3, 5, 0), (33, 31, 32),
                                      (65, 64, 64), (64, 65, 32), (100, 37, 64), (129, 200, 32), (200, 129, 64),
                                      (257, 95, 0)])
def test_shapes_and_tiles(orc, sy, m, n, tile):
    A, B, C = inputs.problem(m, n, m * 1000 + n, kind="benign")
    check_against_oracle(orc, sy, A, B, C, tile=tile)


@pytest.mark.parametrize("transa,transb", [(True, False), (False, True), (True, True)])
def test_transposes(orc, sy, transa, transb):
    A, B, C = inputs.problem(150, 90, 7, kind="benign")
    check_against_oracle(orc, sy, A, B, C, tile=32, transa=transa, transb=transb)


def test_two_by_two_blocks_at_edges(orc, sy):
    """2x2 blocks at index 0, at the last index and straddling every nominal tile
    boundary: the partition must move boundaries instead of splitting blocks."""
    m = n = 130
    A = inputs.quasi_triangular(m, 5, kind="benign", p_pair=0.0)
    B = inputs.quasi_triangular(n, 6, kind="benign", p_pair=0.0)
    for T in (A, B):
        for i in [0, 31, 63, 95, 128]:
            T[i, i + 1], T[i + 1, i] = 1.5, -0.75
            T[i + 1, i + 1] = T[i, i]
    C = inputs.rhs(m, n, 3)
    for tile in (32, 64):
        check_against_oracle(orc, sy, A, B, C, tile=tile)


def test_diagonal_closed_form(sy):
    """Diagonal A, B: Y_ij = C_ij / (a_i + b_j).  The 1x1 small solves multiply by the
    stored reciprocal of the pivot a_i + b_j (two roundings instead of one), so every
    entry must be within one unit in the last place of the correctly rounded quotient."""
    rng = np.random.default_rng(3)
    m, n = 150, 70
    a = rng.uniform(1, 10, m)
    b = rng.uniform(1, 10, n)
    C = rng.uniform(-1, 1, (m, n))
    Y, res = gpu_solve(sy, np.diag(a), np.diag(b), C, tile=32)
    assert res.log2scale == 0 and res.info == 0
    ref = C / (a[:, None] + b[None, :])
    assert np.all(np.abs(Y - ref) <= np.spacing(np.abs(ref)))


def test_deterministic(sy):
    A, B, C = inputs.problem(300, 260, 9, kind="benign")
    Y1, _ = gpu_solve(sy, A, B, C, tile=32)
    Y2, _ = gpu_solve(sy, A, B, C, tile=32)
    assert np.array_equal(Y1, Y2)


def test_paper_matrices_need_no_scaling(orc, sy):
    """Sec. 4: mu = m, nu = n gives alpha = 1."""
    m, n = 200, 150
    A = inputs.paper_matrix(m, float(m), seed=1)
    B = inputs.paper_matrix(n, float(n), seed=2)
    C = np.ones((m, n))
    Y, res, ref = check_against_oracle(orc, sy, A, B, C, tile=64)
    assert res.log2scale == 0


@pytest.mark.parametrize("m,upper,tile", [(300, 100.0, 32), (500, 30.0, 64), (257, 120.0, 64), (400, 40.0, 32)])
def test_robust_where_plain_overflows(orc, sy, m, upper, tile):
    """Unscaled growth of ~1300-1900 bits (past the binary64 range): the robust GPU
    solve stays finite with a representable alpha < 1, a tiny residual and the
    oracle's Y/alpha (after a common power-of-two shift); the non-robust mode
    overflows."""
    A, B, C = inputs.problem(m, m, 3, kind="growth", upper=upper)
    ref = orc.trsyl(A, B, C)
    assert ref["log2scale"] < 0 and ref["info"] == 0
    Y, res = gpu_solve(sy, A, B, C, tile=tile)
    assert res.info == 0, res
    assert res.log2scale < 0 and res.scale_events > 0
    assert np.all(np.isfinite(Y)) and np.max(np.abs(Y)) <= 2.0 ** 1020
    assert orc.residual(A, B, Y, C, res.log2scale) <= RESID_TOL
    err = rel(shifted(Y, res.log2scale, ref["log2scale"]), ref["Y"])
    assert err <= FWD_TOL, err
    _, res_nr = gpu_solve(sy, A, B, C, tile=tile, precision="fp64_nonrobust", check=False)
    assert res_nr.info == sy.SYLV_OVERFLOWED


@pytest.mark.parametrize("m,n,tile,upper,seed", [(32, 32, 32, 1e10, 7), (20, 28, 32, 1e12, 7), (17, 31, 32, 1e13, 9),
                                                 (64, 64, 64, 1e6, 7)])
def test_single_tile_growth_hands_over_to_scaling(orc, sy, m, n, tile, upper, seed):
    """One diagonal tile whose own substitution grows past the binary64 range: its
    left-looking steps (which never scale) must hand over to the scaled right-looking
    steps partway through the tile (scale_events > 0 on a single tile), whose tile-wide
    factors (ProtectUpdate, Sec. 2.1) every warp must apply.  alpha < 1 and
    representable, every entry finite and <= Omega, the eq. (9) residual tiny, and
    Y/alpha equal to the oracle's entry by entry.  The solutions span ~440 decades, so
    the normwise residual cannot see errors in the small entries (wrong entries of
    size 1e-60 relative to max|Y| leave it near 1e-17).  The problems are well
    conditioned componentwise (relative perturbations of 1e-15 in A and B move no
    entry of X by more than ~1e-11), so every entry must agree; all entries stay
    normal on both sides (the smallest is ~1e-166 of the largest)."""
    A, B, C = inputs.problem(m, n, seed, kind="growth", upper=upper)
    ref = orc.trsyl(A, B, C)
    assert -1074 < ref["log2scale"] < 0 and ref["info"] == 0
    Y, res = gpu_solve(sy, A, B, C, tile=tile)
    assert res.info == 0 and -1074 < res.log2scale < 0 and res.scale_events > 0
    assert np.all(np.isfinite(Y)) and np.max(np.abs(Y)) <= 2.0 ** 1020
    assert orc.residual(A, B, Y, C, res.log2scale) <= RESID_TOL
    Yr = shifted(Y, res.log2scale, ref["log2scale"])
    Yo = ref["Y"]
    assert np.min(np.abs(Yo)) > 2.0 ** -900 and np.min(np.abs(Yr)) > 2.0 ** -900
    cw = np.abs(Yr - Yo) / np.abs(Yo)
    assert float(np.max(cw)) <= 1e-10, (np.unravel_index(np.argmax(cw), cw.shape), float(np.max(cw)))


@pytest.mark.parametrize("m,n,upper,seed,tile", [(100, 100, 1e3, 3, 32), (160, 96, 1e4, 5, 32), (160, 96, 1e4, 5, 64),
                                                 (200, 200, 30.0, 7, 32)])
def test_multi_tile_growth_entrywise(orc, sy, m, n, upper, seed, tile):
    """Growth inputs over several tiles (solutions spanning up to ~560 decades; the
    160 x 96 case needs alpha = 2^-839 in the oracle): besides the normwise checks,
    Y/alpha must match the oracle entry by entry wherever both sides hold a normal
    number.  Relative perturbations of 1e-15 in A and B move no entry of these
    solutions by more than ~1e-9, so 1e-7 leaves a factor 100 for rounding while any
    wrong factor, sign or dropped term in a small entry fails."""
    A, B, C = inputs.problem(m, n, seed, kind="growth", upper=upper)
    Y, res, ref = check_against_oracle(orc, sy, A, B, C, tile=tile)
    Yr = shifted(Y, res.log2scale, ref["log2scale"])
    Yo = ref["Y"]
    mask = (np.abs(Yo) > 2.0 ** -900) & (np.abs(Yr) > 2.0 ** -900)
    assert mask.mean() > 0.99
    cw = np.abs(Yr - Yo)[mask] / np.abs(Yo)[mask]
    assert float(np.max(cw)) <= 1e-7, float(np.max(cw))


@pytest.mark.parametrize("m,n,seed,tile", [(184, 10, 936395, 32), (185, 48, 900660, 0), (189, 45, 237710, 0)])
def test_alpha_below_binary64_against_decimal_solution(orc, sy, m, n, seed, tile):
    """Growth inputs (strictly-upper entries up to 1e6) whose solutions need
    alpha = 2^-1270 ... 2^-1978, below the binary64 range (status SCALE_UNDERFLOW).
    Algorithm 2's single factor scales right-hand sides it has not reached yet, and
    once alpha < 2^-1074 they underflow to zero: on these inputs the oracle's Y/alpha
    is 15-100% off the true solution (normwise).  The tile kernel's per-tile factors
    scale a tile's right-hand side only together with its own updates, so its result
    is compared with the solution computed in 50-digit decimal arithmetic (no
    scaling, unbounded exponent range; pinned on the CPU against the Kronecker solve
    and the exact rational residual): measured 2e-16 ... 4e-15 normwise and at most
    5e-12 relative in any entry that is a normal binary64 number."""
    A, B, C = inputs.problem(m, n, seed, kind="growth", upper=1e6)
    Y, res = gpu_solve(sy, A, B, C, tile=tile, check=False)
    assert res.info == sy.SYLV_SCALE_UNDERFLOW and res.log2scale < -1074
    assert np.all(np.isfinite(Y)) and np.max(np.abs(Y)) <= 2.0 ** 1020
    assert orc.residual(A, B, Y, C, res.log2scale) <= RESID_TOL
    X = orc.decimal_scaled(orc.solve_decimal(A, B, C), res.log2scale)
    assert rel(Y, X) <= 1e-13
    mask = np.abs(X) > 2.0 ** -1000
    assert mask.mean() > 0.5
    cw = np.abs(Y - X)[mask] / np.abs(X)[mask]
    assert float(np.max(cw)) <= 1e-10, float(np.max(cw))


@pytest.mark.parametrize("m,n,tile", [(32, 32, 32), (29, 18, 32), (64, 40, 64)])
def test_right_hand_side_near_omega_starts_right_looking(orc, sy, m, n, tile):
    """Entries of C near 2^1018: the diagonal tile's bound test fails before its first
    step, so the tile is solved by the scaled right-looking steps from the start; the
    result must still match the oracle."""
    A, B, C = inputs.problem(m, n, 5, kind="benign")
    C = np.ldexp(C, 1018)
    check_against_oracle(orc, sy, A, B, C, tile=tile)


@pytest.mark.parametrize("m,n,tile,kind,upper", [(1, 1, 0, "benign", 1.0), (33, 31, 32, "benign", 1.0),
                                                 (129, 200, 32, "benign", 1.0), (200, 129, 64, "benign", 1.0),
                                                 (257, 95, 0, "benign", 1.0), (300, 300, 32, "growth", 30.0)])
def test_nonrobust_matches_oracle_plain(orc, sy, m, n, tile, kind, upper):
    """The non-robust mode (Algorithm 1 per tile: no guard, no scaling) against the
    oracle's plain substitution (Algorithm 1) on inputs where it stays finite: the
    same Y (alpha = 1) to 1e-13.  The growth case reaches max|Y| ~ 2^746, large but
    inside the binary64 range, so nothing overflows there either."""
    A, B, C = inputs.problem(m, n, 40 + m + n, kind=kind, upper=upper)
    ref = orc.trsyl(A, B, C, robust=False)
    assert ref["log2scale"] == 0 and np.all(np.isfinite(ref["Y"]))
    Y, res = gpu_solve(sy, A, B, C, tile=tile, precision="fp64_nonrobust")
    assert res.info == 0 and res.log2scale == 0 and res.scale_events == 0
    assert rel(Y, ref["Y"]) <= FWD_TOL
    assert orc.residual(A, B, Y, C, 0) <= RESID_TOL


@pytest.mark.parametrize("transa,transb", [(True, False), (False, True), (True, True)])
def test_nonrobust_transposes(orc, sy, transa, transb):
    A, B, C = inputs.problem(150, 90, 17, kind="benign")
    ref = orc.trsyl(A, B, C, robust=False, transa=transa, transb=transb)
    Y, res = gpu_solve(sy, A, B, C, tile=32, precision="fp64_nonrobust", transa=transa, transb=transb)
    assert res.info == 0 and res.log2scale == 0
    assert rel(Y, ref["Y"]) <= FWD_TOL


def test_extreme_growth_alpha_underflows(orc, sy):
    """Strictly-upper entries ~1e120: alpha falls below the double range for the oracle
    and the GPU alike; log2scale still carries it exactly, every entry stays finite
    and the residual (evaluated with a common power-of-two shift) stays tiny."""
    A, B, C = inputs.problem(48, 48, 3, kind="growth", upper=1e120)
    ref = orc.trsyl(A, B, C)
    Y, res = gpu_solve(sy, A, B, C, tile=32, check=False)
    assert ref["log2scale"] < -1074 and res.log2scale < -1074
    assert res.info == sy.SYLV_SCALE_UNDERFLOW and res.scale == 0.0
    assert np.all(np.isfinite(Y)) and np.max(np.abs(Y)) <= 2.0 ** 1020
    assert orc.residual(A, B, Y, C, res.log2scale) <= RESID_TOL


def test_paper_small_mu_scaling(orc, sy):
    """Sec. 4: mu = 1e-3, nu = 1e-2 needs frequent scaling."""
    m = n = 300
    A = inputs.paper_matrix(m, 1e-3, seed=1)
    B = inputs.paper_matrix(n, 1e-2, seed=2)
    C = np.ones((m, n))
    Y, res = gpu_solve(sy, A, B, C, tile=64, check=False)
    ref = orc.trsyl(A, B, C)
    assert res.log2scale < 0 and np.all(np.isfinite(Y))
    if res.info == sy.SYLV_SCALE_UNDERFLOW:
        assert res.scale == 0.0
    else:
        assert res.info == 0
    assert orc.residual(A, B, Y, C, res.log2scale) <= RESID_TOL
    assert ref["log2scale"] < 0


def test_structure_and_input_errors(sy):
    A, B, C = inputs.problem(40, 30, 1)
    A2 = A.copy()
    A2[11, 10] = 0.5
    A2[12, 11] = 0.5
    _, res = gpu_solve(sy, A2, B, C, check=False)
    assert res.info == sy.SYLV_ERR_STRUCTURE_A
    B2 = B.copy()
    B2[4, 3] = 1.0
    B2[5, 4] = 1.0
    _, res = gpu_solve(sy, A, B2, C, check=False)
    assert res.info == sy.SYLV_ERR_STRUCTURE_B
    C2 = C.copy()
    C2[3, 3] = np.nan
    _, res = gpu_solve(sy, A, B, C2, check=False)
    assert res.info == sy.SYLV_ERR_NONFINITE
    A3 = A.copy()
    A3[0, 5] = np.inf
    _, res = gpu_solve(sy, A3, B, C, check=False)
    assert res.info == sy.SYLV_ERR_NONFINITE


def test_near_singular_reported(sy):
    """lambda_i(A) + lambda_j(B) = 0 for one pair: the small solve's pivot is raised to
    smin and the status says so (eq. (1)'s uniqueness condition fails)."""
    m, n = 20, 20
    A = np.triu(np.full((m, m), 0.1), 1) + np.diag(np.linspace(1, 3, m))
    B = np.triu(np.full((n, n), 0.1), 1) + np.diag(np.linspace(1, 3, n))
    B[7, 7] = -A[3, 3]
    C = inputs.rhs(m, n, 1)
    Y, res = gpu_solve(sy, A, B, C, check=False)
    assert res.info in (sy.SYLV_NEAR_SINGULAR, sy.SYLV_SCALE_UNDERFLOW)
    assert np.all(np.isfinite(Y))


def test_near_singular_matches_oracle(orc, sy):
    """The singular pair of test_near_singular_reported sits in merged pseudo blocks on
    both sides (rows 2-3 of A, columns 6-7 of B are pairs of 1x1 blocks): the composed
    inverse raises exactly the 1x1 pivot that the oracle raises, so Y / alpha agrees
    with the oracle's (normwise, after a common power-of-two shift)."""
    m, n = 20, 20
    A = np.triu(np.full((m, m), 0.1), 1) + np.diag(np.linspace(1, 3, m))
    B = np.triu(np.full((n, n), 0.1), 1) + np.diag(np.linspace(1, 3, n))
    B[7, 7] = -A[3, 3]
    C = inputs.rhs(m, n, 1)
    Y, res = gpu_solve(sy, A, B, C, check=False)
    ref = orc.trsyl(A, B, C)
    assert res.info in (sy.SYLV_NEAR_SINGULAR, sy.SYLV_SCALE_UNDERFLOW)
    Ys = np.ldexp(Y, int(ref["log2scale"]) - int(res.log2scale))
    s = np.max(np.abs(ref["Y"]))
    assert np.linalg.norm(Ys / s - ref["Y"] / s) <= 1e-9 * np.linalg.norm(ref["Y"] / s)


def test_bounded_wait_times_out_without_hanging(sy):
    """A wait on a flag nothing sets ends with SYLV_ERR_TIMEOUT; the context stays
    usable for the next solve."""
    import time
    t0 = time.time()
    rc = sy.sylv_diag_wait_timeout(200)
    assert rc == sy.SYLV_ERR_TIMEOUT
    assert time.time() - t0 < 30
    A, B, C = inputs.problem(64, 64, 2)
    Y, res = gpu_solve(sy, A, B, C)
    assert res.info == 0


@pytest.mark.parametrize("m,n", [(300, 300), (257, 130)])
def test_fp32_refine_reaches_fp64_accuracy(orc, sy, m, n):
    """FP32 correction solves + FP64 residuals: forward error <= 1e-12 against the
    oracle on well-conditioned inputs."""
    A, B, C = inputs.problem(m, n, 4, kind="wellcond")
    Y, res = gpu_solve(sy, A, B, C, precision="fp32_refine", tile=32)
    ref = orc.trsyl(A, B, C)
    assert res.info == 0, res
    assert res.iters >= 2
    assert rel(Y, ref["Y"]) <= REFINE_TOL
    assert orc.residual(A, B, Y, C, 0) <= RESID_TOL


@pytest.mark.parametrize("transa", [False, True])
def test_fp32_refine_beyond_binary64_solves_with_fp64(orc, sy, transa):
    """A growth input whose solution needs alpha = 2^-199: FP32 + refinement returns
    alpha = 1 and cannot hold it (its first correction is infinite).  The synchronous
    solve sees SYLV_OVERFLOWED, finds C untouched and solves again on the robust FP64
    path: iters = 0, alpha < 1, Y/alpha as the oracle's."""
    A, B, C = inputs.problem(160, 96, 5, kind="growth", upper=1e3)
    ref = orc.trsyl(A, B, C, transa=transa)
    assert ref["log2scale"] < 0
    Y, res = gpu_solve(sy, A, B, C, precision="fp32_refine", tile=32, transa=transa)
    assert res.info == 0 and res.iters == 0 and res.log2scale < 0, res
    assert np.all(np.isfinite(Y))
    assert orc.residual(A, B, Y, C, res.log2scale, transa, False) <= RESID_TOL
    assert rel(shifted(Y, res.log2scale, ref["log2scale"]), ref["Y"]) <= FWD_TOL


def test_fp32_refine_beyond_binary64_async_reports_overflow(sy):
    """The same input without synchronization (result written to device memory):
    status SYLV_OVERFLOWED, and C still holds the right-hand side bit for bit."""
    import ctypes
    A, B, C = inputs.problem(160, 96, 5, kind="growth", upper=1e3)
    Ad, Bd, Cd = dev(A), dev(B), dev(C)
    stream = torch.cuda.current_stream()
    o = sy.make_opts(precision="fp32_refine", tile=32, stream=stream.cuda_stream, sync=False)
    rbuf = torch.zeros(ctypes.sizeof(sy.sylv_result), dtype=torch.uint8, device="cuda")
    rc = sy.sylv_tri_solve_ex(160, 96, Ad.data_ptr(), Ad.stride(1), Bd.data_ptr(), Bd.stride(1), Cd.data_ptr(),
                              Cd.stride(1), o, rbuf.data_ptr())
    torch.cuda.synchronize()
    assert rc == 0
    r = sy.sylv_result.from_buffer_copy(bytes(rbuf.cpu().numpy()))
    assert r.info == sy.SYLV_OVERFLOWED
    assert np.array_equal(host(Cd), C)


def test_batched_refine_beyond_binary64_reports_overflow(orc, sy):
    """In a refined batch, the equation whose solution lies beyond the binary64 range
    reports SYLV_OVERFLOWED and keeps its right-hand side; the others are solved."""
    probs = [inputs.problem(60, 50, 11, kind="wellcond"), inputs.problem(160, 96, 5, kind="growth", upper=1e3),
             inputs.problem(90, 130, 12, kind="benign")]
    Ys, rs = sy.batch_solve([dev(p[0]) for p in probs], [dev(p[1]) for p in probs], [dev(p[2]) for p in probs],
                            tile=32, precision="fp32_refine")
    torch.cuda.synchronize()
    assert rs[1].info == sy.SYLV_OVERFLOWED
    assert np.array_equal(host(Ys[1]), probs[1][2])
    for i in (0, 2):
        A, B, C = probs[i]
        assert rs[i].info == 0
        assert rel(host(Ys[i]), orc.trsyl(A, B, C)["Y"]) <= REFINE_TOL


def test_batched_growth_against_decimal_solution(orc, sy):
    """24 growth equations (m 20-120, n 5-60, strictly-upper scale 30, 1e3 or 1e6;
    alpha from 1 down to below 2^-1074) in one batched launch: every entry of Y that
    is a normal binary64 number against the 50-digit decimal solution (measured
    <= 3.7e-11), and each equation bitwise equal to its own single solve."""
    rng = np.random.default_rng(5)
    probs = []
    for i in range(24):
        m, n = int(rng.integers(20, 121)), int(rng.integers(5, 61))
        up = float(rng.choice([30.0, 1e3, 1e6]))
        probs.append(inputs.problem(m, n, 500 + i, kind="growth", upper=up))
    Ys, rs = sy.batch_solve([dev(p[0]) for p in probs], [dev(p[1]) for p in probs], [dev(p[2]) for p in probs],
                            tile=32)
    torch.cuda.synchronize()
    for (A, B, C), Yt, r in zip(probs, Ys, rs):
        Y = host(Yt)
        assert r.info == (sy.SYLV_SCALE_UNDERFLOW if r.log2scale < -1074 else 0)
        X = orc.decimal_scaled(orc.solve_decimal(A, B, C), r.log2scale)
        mask = np.abs(X) > 2.0 ** -1000
        assert mask.any()
        assert float(np.max(np.abs(Y - X)[mask] / np.abs(X)[mask])) <= 1e-9
        Y1, r1 = gpu_solve(sy, A, B, C, tile=32, check=False)
        assert r1.log2scale == r.log2scale and np.array_equal(Y1, Y)


def test_batched_uneven(orc, sy):
    shapes = inputs.batch_shapes(24, 16, 300, seed=5)
    probs = [inputs.problem(m, n, 100 + i, kind="benign") for i, (m, n) in enumerate(shapes)]
    Ys, res = sy.batch_solve([dev(p[0]) for p in probs], [dev(p[1]) for p in probs],
                             [dev(p[2]) for p in probs])
    torch.cuda.synchronize()
    for (A, B, C), Y, r in zip(probs, Ys, res):
        assert r.info == 0
        Yh = host(Y)
        ref = orc.trsyl(A, B, C)
        assert orc.residual(A, B, Yh, C, r.log2scale) <= RESID_TOL
        assert rel(shifted(Yh, r.log2scale, ref["log2scale"]), ref["Y"]) <= FWD_TOL


def test_adjoint_matches_kronecker_gradient(orc, sy):
    """Lyapunov-type A Y + Y A^T = C at m = n = 16: autograd through the hand-written
    adjoint against the oracle's Kronecker-form gradient (dA = both uses of A)."""
    m = 16
    A = inputs.quasi_triangular(m, 8, kind="wellcond")
    C = inputs.rhs(m, m, 9)
    W = inputs.rhs(m, m, 10)
    At = dev(A).requires_grad_(True)
    Ct = dev(C).requires_grad_(True)
    Y = sy.SylvesterSolve.apply(At, At, Ct, False, True, 0)
    loss = (dev(W) * Y).sum()
    loss.backward()
    dA1, dB1, dC, _ = orc.kron_grad(A, A, C, W, False, True)
    assert rel(host(At.grad), dA1 + dB1) <= 1e-11
    assert rel(host(Ct.grad), dC) <= 1e-11


def test_adjoint_finite_differences(sy):
    """Central differences, h = 1e-6, of the GPU forward solve for a few entries."""
    m, n = 40, 30
    A, B, C = inputs.problem(m, n, 12, kind="wellcond")
    W = inputs.rhs(m, n, 13)
    At, Bt, Ct = dev(A).requires_grad_(True), dev(B).requires_grad_(True), dev(C).requires_grad_(True)
    Y = sy.SylvesterSolve.apply(At, Bt, Ct, False, False, 32)
    (dev(W) * Y).sum().backward()
    h = 1e-6

    def loss(A_, B_, C_):
        Y_, _ = gpu_solve(sy, A_, B_, C_, tile=32)
        return float(np.sum(W * Y_))

    for (M, grad, idx) in [("A", At.grad, (3, 17)), ("A", At.grad, (10, 10)), ("B", Bt.grad, (0, 29)),
                           ("C", Ct.grad, (39, 0))]:
        E = np.zeros({"A": A, "B": B, "C": C}[M].shape)
        E[idx] = h
        args_p = [A + E if M == "A" else A, B + E if M == "B" else B, C + E if M == "C" else C]
        args_m = [A - E if M == "A" else A, B - E if M == "B" else B, C - E if M == "C" else C]
        fd = (loss(*args_p) - loss(*args_m)) / (2 * h)
        g = float(host(grad)[idx])
        assert abs(g - fd) <= 1e-6 * max(1.0, abs(fd)), (M, idx, g, fd)


def test_adjoint_removes_its_own_scale(orc, sy):
    """With Omega = 2^12 the growth input makes the forward solve AND the adjoint
    solve scale (alpha = 2^e < 1, alpha_G < 1).  The backward entry points must hand
    back the true gradients of L = sum(W * Y) with Y = alpha X (alpha held fixed):
    dC = alpha Gamma, dA = alpha dA_X, dB = alpha dB_X, where Gamma and the
    X-gradients are the oracle's Kronecker-form gradients -- with alpha_G removed
    inside the call (a missing or doubled 2^-log2(alpha_G) is off by >= 2^4).  The
    single and the batched entry points are both checked."""
    m, n = 12, 16
    A, B, C = inputs.problem(m, n, 7, kind="growth", upper=16.0)
    W = inputs.rhs(m, n, 57)
    o = sy.make_opts(omega=2.0 ** 12)
    Ad, Bd = dev(A), dev(B)
    Y = dev(C).clone()
    res = sy.sylv_result()
    rc = sy.sylv_tri_solve_ex(m, n, Ad.data_ptr(), m, Bd.data_ptr(), n, Y.data_ptr(), m, o, res)
    assert rc == 0 and res.log2scale < 0
    rA, rB, rC, X = orc.kron_grad(A, B, C, W)
    alpha = 2.0 ** res.log2scale
    assert rel(np.ldexp(host(Y), -int(res.log2scale)), X) <= 1e-9  # kappa ~ 1e5: LU against the tiled solve
    # single
    G = dev(W).clone()
    dA = torch.zeros((m, m), dtype=torch.float64, device="cuda").t()
    dB = torch.zeros((n, n), dtype=torch.float64, device="cuda").t()
    r2 = sy.sylv_result()
    rc = sy.sylv_tri_solve_backward(m, n, Ad.data_ptr(), m, Bd.data_ptr(), n, Y.data_ptr(), m, res.log2scale,
                                    G.data_ptr(), m, dA.data_ptr(), m, dB.data_ptr(), n, o, r2)
    torch.cuda.synchronize()
    assert rc == 0 and r2.log2scale <= -4
    assert rel(host(G), alpha * rC) <= 1e-12
    assert rel(host(dA), alpha * rA) <= 1e-9
    assert rel(host(dB), alpha * rB) <= 1e-9
    # batched: the same equation twice beside an unscaled one
    A2, B2, C2 = inputs.problem(m, n, 8, kind="wellcond")
    A2d, B2d, Y2 = dev(A2), dev(B2), dev(C2).clone()
    res2 = sy.sylv_result()
    rc = sy.sylv_tri_solve_ex(m, n, A2d.data_ptr(), m, B2d.data_ptr(), n, Y2.data_ptr(), m, o, res2)
    assert rc == 0 and res2.log2scale == 0
    Gs = [dev(W).clone(), dev(W).clone(), dev(W).clone()]
    dAs = [torch.zeros((m, m), dtype=torch.float64, device="cuda").t() for _ in range(3)]
    dBs = [torch.zeros((n, n), dtype=torch.float64, device="cuda").t() for _ in range(3)]
    rc, rs = sy.sylv_tri_solve_backward_batched(
        [m] * 3, [n] * 3, [Ad.data_ptr(), A2d.data_ptr(), Ad.data_ptr()], [m] * 3,
        [Bd.data_ptr(), B2d.data_ptr(), Bd.data_ptr()], [n] * 3, [Y.data_ptr(), Y2.data_ptr(), Y.data_ptr()],
        [m] * 3, [res.log2scale, res2.log2scale, res.log2scale], [g.data_ptr() for g in Gs], [m] * 3,
        [d.data_ptr() for d in dAs], [m] * 3, [d.data_ptr() for d in dBs], [n] * 3, o)
    torch.cuda.synchronize()
    assert rc == 0 and rs[0].log2scale <= -4 and rs[2].log2scale <= -4
    rA2, rB2, rC2, _ = orc.kron_grad(A2, B2, C2, W)
    for i, (ga, ra, rb, rcc) in enumerate([(alpha, rA, rB, rC), (1.0, rA2, rB2, rC2), (alpha, rA, rB, rC)]):
        assert rel(host(Gs[i]), ga * rcc) <= 1e-12, i
        assert rel(host(dAs[i]), ga * ra) <= 1e-9, i
        assert rel(host(dBs[i]), ga * rb) <= 1e-9, i


@pytest.mark.parametrize("transa,transb", [(True, False), (False, True), (True, True)])
def test_batched_transposes(orc, sy, transa, transb):
    shapes = inputs.batch_shapes(10, 16, 200, seed=8)
    probs = [inputs.problem(m, n, 300 + i, kind="benign") for i, (m, n) in enumerate(shapes)]
    Ys, res = sy.batch_solve([dev(p[0]) for p in probs], [dev(p[1]) for p in probs], [dev(p[2]) for p in probs],
                             transa=transa, transb=transb)
    torch.cuda.synchronize()
    for (A, B, C), Y, r in zip(probs, Ys, res):
        assert r.info == 0
        Yh = host(Y)
        ref = orc.trsyl(A, B, C, transa=transa, transb=transb)
        assert orc.residual(A, B, Yh, C, r.log2scale, transa, transb) <= RESID_TOL
        assert rel(shifted(Yh, r.log2scale, ref["log2scale"]), ref["Y"]) <= FWD_TOL


def test_batched_adjoint_lyapunov(orc, sy):
    """A batch of Lyapunov equations A_i Y + Y A_i^T = C_i (m = n = 16) through the
    batched autograd Function: gradients against the oracle's Kronecker form."""
    b, m = 5, 16
    As = np.stack([inputs.quasi_triangular(m, 50 + i, kind="wellcond") for i in range(b)])
    Cs = np.stack([inputs.rhs(m, m, 60 + i) for i in range(b)])
    Ws = np.stack([inputs.rhs(m, m, 70 + i) for i in range(b)])
    At = torch.from_numpy(As).cuda().requires_grad_(True)
    Ct = torch.from_numpy(Cs).cuda().requires_grad_(True)
    Y = sy.BatchSylvesterSolve.apply(At, At, Ct, False, True, 0)
    (torch.from_numpy(Ws).cuda() * Y).sum().backward()
    for i in range(b):
        dA1, dB1, dC, X = orc.kron_grad(As[i], As[i], Cs[i], Ws[i], False, True)
        assert rel(host(Y[i].detach()), X) <= FWD_TOL
        assert rel(host(At.grad[i]), dA1 + dB1) <= 1e-11
        assert rel(host(Ct.grad[i]), dC) <= 1e-11


def test_batched_cuda_graph_replay(orc, sy):
    """A batch plan's execute captured once in a CUDA graph and replayed twice, with the
    right-hand sides refilled before each replay, gives the oracle's solutions."""
    shapes = inputs.batch_shapes(12, 16, 160, seed=21)
    probs = [inputs.problem(m, n, 700 + i, kind="benign") for i, (m, n) in enumerate(shapes)]
    As = [dev(p[0]) for p in probs]
    Bs = [dev(p[1]) for p in probs]
    C0 = [dev(p[2]) for p in probs]
    Cs = [c.clone() for c in C0]
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        o = sy.make_opts(stream=stream.cuda_stream)
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
                ref = orc.trsyl(A, B, C)
                Yh = host(Y)
                assert r.info == 0
                assert rel(shifted(Yh, r.log2scale, ref["log2scale"]), ref["Y"]) <= FWD_TOL
    finally:
        sy.sylv_batch_destroy(plan)


def test_autotuned_tiles_solve_correctly(orc, sy):
    from paper_1905_10574_gb300 import autotune
    shapes = inputs.batch_shapes(16, 16, 300, seed=33)
    probs = [inputs.problem(m, n, 800 + i, kind="benign") for i, (m, n) in enumerate(shapes)]
    As = [dev(p[0]) for p in probs]
    Bs = [dev(p[1]) for p in probs]
    Cs = [dev(p[2]) for p in probs]
    tiles = autotune.tune_batch(As, Bs, Cs, use_cache=False, reps=1)
    assert len(tiles) == len(shapes) and all(t in autotune.CANDIDATES for t in tiles)
    for c, p in zip(Cs, probs):  # inputs restored after tuning
        assert np.array_equal(host(c), p[2])
    o = sy.make_opts(stream=torch.cuda.current_stream().cuda_stream)
    plan = sy.sylv_batch_create([m for m, _ in shapes], [n for _, n in shapes], [a.data_ptr() for a in As],
                                [a.stride(1) for a in As], [b.data_ptr() for b in Bs], [b.stride(1) for b in Bs],
                                [c.data_ptr() for c in Cs], [c.stride(1) for c in Cs], o, tiles=tiles)
    try:
        assert sy.sylv_batch_execute(plan, o.stream) == 0
        rc, res = sy.sylv_batch_results(plan, len(shapes))
    finally:
        sy.sylv_batch_destroy(plan)
    for (A, B, C), Y, r in zip(probs, Cs, res):
        ref = orc.trsyl(A, B, C)
        assert rel(shifted(host(Y), r.log2scale, ref["log2scale"]), ref["Y"]) <= FWD_TOL

"""The allocation-free entry point, sylv_tri_solve_noalloc, against the regular
entry point sylv_tri_solve_ex.

Callers that cannot allocate device memory at solve time (real-time loops that
forbid allocator calls after start-up, hosts whose device memory belongs to a
foreign allocator) use the allocation-free entry point; it runs the same solver
with scratch in a fixed device array of the library.  This file is collected last
on purpose; it passes alone in a fresh process and after the other tests.
"""
import numpy as np
import pytest

from paper_1905_10574_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = 1e-13  # the relative Frobenius tolerance the other FP64 GPU tests use for Y/alpha
SCRATCH = 16 << 20  # bytes of the fixed device array


@pytest.fixture(scope="module")
def sy():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_10574_gb300 import build, sylv
    build.build()
    sylv.load()
    return sylv


def _dev(a):
    return torch.from_numpy(np.asfortranarray(a)).cuda()


def _rel(a, b):
    s = max(float(np.max(np.abs(a))), float(np.max(np.abs(b))))
    e = -int(np.frexp(s)[1]) if s > 0 else 0
    a2, b2 = np.ldexp(a, e), np.ldexp(b, e)
    return float(np.linalg.norm(a2 - b2) / np.linalg.norm(b2))


def _regular(sy, A, B, C):
    Ad, Bd, Cd = _dev(A), _dev(B), _dev(C)
    res = sy.sylv_result()
    rc = sy.sylv_tri_solve_ex(A.shape[0], B.shape[0], Ad.data_ptr(), Ad.stride(1), Bd.data_ptr(), Bd.stride(1),
                              Cd.data_ptr(), Cd.stride(1), sy.sylv_default_opts(), res)
    assert rc == 0, rc
    return Cd.cpu().numpy(), res


def _noalloc(sy, A, B, C):
    Ad, Bd, Cd = _dev(A), _dev(B), _dev(C)
    rc, res = sy.sylv_tri_solve_noalloc(A.shape[0], B.shape[0], Ad.data_ptr(), Ad.stride(1), Bd.data_ptr(),
                                        Bd.stride(1), Cd.data_ptr(), Cd.stride(1), 0,
                                        torch.cuda.current_stream().cuda_stream)
    assert rc == 0, rc
    return Cd.cpu().numpy(), res


def test_noalloc_matches_regular_entry_point_two_calls(sy):
    """Two calls in a row on different problems (the second must not see the first's
    leftovers in the shared scratch), each against the regular entry point."""
    cases = [inputs.problem(700, 450, 31, kind="benign"), inputs.problem(500, 500, 3, kind="growth", upper=30.0)]
    for A, B, C in cases:
        Y_ref, r_ref = _regular(sy, A, B, C)
        Y, r = _noalloc(sy, A, B, C)
        assert r.info == r_ref.info == 0
        assert r.log2scale == r_ref.log2scale
        Ys = np.ldexp(Y, int(r_ref.log2scale) - int(r.log2scale))
        assert _rel(Ys, Y_ref) <= TOL


def test_noalloc_fewer_ctas_than_regular(sy):
    """m = n = 10000 at tile 32: the bookkeeping leaves room for fewer per-CTA factor
    stores than the regular entry point's two CTAs per SM, so the allocation-free
    call runs the tile kernel with fewer CTAs; its result must still match."""
    m = n = 10000
    p = q = -(-m // 32)
    fixed_lower = p * q * (4 + 8 + 4 + 8) + (p * p + q * q) * 8  # flags, tasks, exponents, norms; norm tables
    per_cta = 5 * 32 * 32 * 8 + 32 * 32 * 4
    assert fixed_lower + 2 * torch.cuda.get_device_properties(0).multi_processor_count * per_cta > SCRATCH
    A, B, C = inputs.problem(m, n, 41, kind="wellcond")
    Y_ref, r_ref = _regular(sy, A, B, C)
    Y, r = _noalloc(sy, A, B, C)
    assert r.info == r_ref.info == 0
    assert r.log2scale == r_ref.log2scale == 0
    assert _rel(Y, Y_ref) <= TOL


def test_noalloc_rejects_too_large(sy):
    """Sizes whose bookkeeping exceeds the fixed scratch are refused on the host from
    the sizes alone, before any GPU work (so a one-element buffer stands in for the
    operands)."""
    n = 24000
    buf = torch.zeros(1, dtype=torch.float64, device="cuda")
    rc, _ = sy.sylv_tri_solve_noalloc(n, n, buf.data_ptr(), n, buf.data_ptr(), n, buf.data_ptr(), n, 0, None)
    assert rc == sy.SYLV_ERR_WORKSPACE

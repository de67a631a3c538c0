"""The solver's own device ProtectUpdate and ProtectDivision (Sec. 2.1), evaluated on
the GPU through the diagnostic entry point sylv_diag_guards and checked on the host
against the contract in exact rational arithmetic.

The contract: for c, t, x in [0, Omega], ProtectUpdate returns zeta = 2^z in (0, 1]
with zeta (c + t x) <= Omega; for |b| <= Omega, ProtectDivision returns zeta with
zeta |b| / |d| <= Omega.  Beyond the contract the solver relies on the factors
being (near) the largest allowed -- a smaller one scales without need -- so that is
checked too: no scaling when c + t x <= Omega / 2, and 2 zeta (c + t x) above Omega
up to rounding; the division factor is exactly the largest power of two.

These checks are independent of the oracle: they compare with the definition, not
with another implementation.
"""
from fractions import Fraction

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

OMEGA64 = 2.0 ** 1020
OMEGA32 = 2.0 ** 124


def _edge_values(omega):
    vals = [0.0, 2.0 ** -1074, 3 * 2.0 ** -1074, 2.0 ** -1022, 2.0 ** -1022 * (1 - 2 ** -52), 0.5,
            1.0 - 2 ** -53, 1.0, 1.0 + 2 ** -52, 2.0, 3.0, 2.0 ** 100, 2.0 ** 500,
            omega / 2, omega * 0.75, omega * (1 - 2 ** -53), omega]
    rng = np.random.default_rng(7)
    vals += list(np.ldexp(rng.uniform(0.5, 1.0, 40), rng.integers(-1074, int(np.log2(omega)), 40)))
    return sorted(set(float(v) for v in vals if v <= omega))


def _update_triples(omega, seed):
    vals = _edge_values(omega)
    rng = np.random.default_rng(seed)
    e = int(np.log2(omega))
    tri = [(c, t, x) for c in vals[::2] for t in vals[::2] for x in vals]
    tri += [tuple(float(v) for v in np.ldexp(rng.uniform(0.5, 1, 3), rng.integers(-60, e + 1, 3)))
            for _ in range(3000)]
    # products straddling omega: t x within a few ulps of omega - c
    for _ in range(500):
        c = float(np.ldexp(rng.uniform(0.5, 1), rng.integers(e - 8, e)))
        t = float(np.ldexp(rng.uniform(0.5, 1), rng.integers(0, e)))
        x = float((Fraction(omega) - Fraction(c)) / Fraction(t)) * float(1 + rng.integers(-4, 5) * 2.0 ** -52)
        tri.append((c, t, x))
    return [(c, t, x) for c, t, x in tri if max(c, t, x) <= omega and min(c, t, x) >= 0.0]


def _division_pairs(omega, seed):
    vals = _edge_values(omega)
    rng = np.random.default_rng(seed)
    pairs = [(b, d) for b in vals for d in vals if d != 0.0]
    pairs += [(float(np.ldexp(rng.uniform(0.5, 1), rng.integers(-1074, int(np.log2(omega))))),
               float(np.ldexp(rng.uniform(0.5, 1), rng.integers(-1074, 2)))) for _ in range(3000)]
    signed = []
    for i, (b, d) in enumerate(pairs):
        signed.append((b if i % 2 else -b, -d if i % 3 == 0 else d))
    return signed


def _device_guards(c, t, x, b, d, omega):
    import torch
    from paper_1905_10574_gb300 import sylv
    n = max(len(c), len(b))
    pad = lambda v: list(v) + [0.0] * (n - len(v))
    dev = lambda v: torch.tensor(pad(v), dtype=torch.float64, device="cuda")
    dc, dt, dx, db = dev(c), dev(t), dev(x), dev(b)
    dd = torch.tensor(list(d) + [1.0] * (n - len(d)), dtype=torch.float64, device="cuda")
    zu = torch.full((n,), 7, dtype=torch.int32, device="cuda")
    zd = torch.full((n,), 7, dtype=torch.int32, device="cuda")
    rc = sylv.sylv_diag_guards(n, dc.data_ptr(), dt.data_ptr(), dx.data_ptr(), zu.data_ptr(), db.data_ptr(),
                               dd.data_ptr(), zd.data_ptr(), omega)
    assert rc == 0, rc
    return zu.cpu().tolist()[:len(c)], zd.cpu().tolist()[:len(b)]


@pytest.mark.parametrize("omega", [OMEGA64, OMEGA32], ids=["omega64", "omega32"])
def test_device_protect_update_contract(omega):
    tri = _update_triples(omega, 11)
    zs, _ = _device_guards([v[0] for v in tri], [v[1] for v in tri], [v[2] for v in tri], [], [], omega)
    W = Fraction(omega)
    scaled = 0
    for (c, t, x), z in zip(tri, zs):
        assert z <= 0, (c, t, x, z)
        zeta = Fraction(2) ** z
        tot = Fraction(c) + Fraction(t) * Fraction(x)
        assert zeta * tot <= W, (c, t, x, z)
        if tot <= W / 2:
            assert z == 0, (c, t, x, z)
        if z < 0:
            scaled += 1
            # the largest power of two, up to the rounding of the bound
            assert 2 * zeta * tot > W * (1 - Fraction(1, 2 ** 48)), (c, t, x, z)
    assert scaled > 500  # the straddling and large cases do reach the scaling branch


@pytest.mark.parametrize("omega", [OMEGA64, OMEGA32], ids=["omega64", "omega32"])
def test_device_protect_division_contract(omega):
    pairs = [(b, d) for b, d in _division_pairs(omega, 5) if abs(b) <= omega]
    _, zs = _device_guards([], [], [], [p[0] for p in pairs], [p[1] for p in pairs], omega)
    W = Fraction(omega)
    scaled = 0
    for (b, d), z in zip(pairs, zs):
        q = abs(Fraction(b)) / abs(Fraction(d))
        zeta = Fraction(2) ** z
        assert zeta * q <= W, (b, d, z)
        if q <= W:
            assert z == 0, (b, d, z)
        else:
            scaled += 1
            assert 2 * zeta * q > W, (b, d, z)  # exactly the largest power of two
    assert scaled > 500


def test_device_guards_arguments():
    from paper_1905_10574_gb300 import sylv
    assert sylv.sylv_diag_guards(-1, None, None, None, None, None, None, None, OMEGA64) == -1
    assert sylv.sylv_diag_guards(4, None, None, None, None, None, None, None, OMEGA64) == -2
    assert sylv.sylv_diag_guards(0, None, None, None, None, None, None, None, 0.5) == -9
    assert sylv.sylv_diag_guards(0, None, None, None, None, None, None, None, OMEGA64) == 0

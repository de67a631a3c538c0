"""Calibrate the overflow workload (robust vs non-robust FP64, m = n = 4000).

The generator is ``inputs.problem(m, n, seed, kind="growth", upper=s)``: the
benign quasi-triangular matrices with the strictly-upper part scaled by s.  A
larger s makes unscaled back substitution grow faster.  The unscaled growth
g(m) = log2 max|X| = log2 max|Y| - log2(alpha) of the FP64 CPU oracle
(Algorithm 2) grows linearly with the order, so s is bisected at m = n = 1000 for
g = TARGET/4, the linearity is confirmed at m = n = 2000, and g(4000) is
extrapolated (the oracle's level-2 row updates make a 4000 x 4000 run take
hours).  TARGET = 1400 bits: past the binary64 range (1024), so the non-robust
solve overflows, while alpha ~ 2^-(g - 1020) stays a normal double.  Only the
oracle is called.  Output: overflow_config.json beside this file.
"""
import json
import math
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from oracle import oracle  # noqa: E402
from paper_1905_10574_gb300 import inputs  # noqa: E402

SEED = 0
TARGET = 1400.0


def growth(m, s):
    A, B, C = inputs.problem(m, m, SEED, kind="growth", upper=s)
    t0 = time.time()
    out = oracle.trsyl(A, B, C)
    g = math.log2(float(np.max(np.abs(out["Y"])))) - out["log2scale"]
    print(f"m={m} upper={s:.4f}: log2 growth={g:.1f} log2scale={out['log2scale']} ({time.time() - t0:.0f}s)",
          flush=True)
    return g


def main():
    lo, hi = 2.0, 8.0
    s = 4.1
    for _ in range(8):
        g = growth(1000, s)
        if abs(g - TARGET / 4) < 10:
            break
        if g < TARGET / 4:
            lo = s
        else:
            hi = s
        s = round(0.5 * (lo + hi), 3)
    g1 = g
    g2 = growth(2000, s)
    ratio = g2 / g1
    if not 1.9 < ratio < 2.1:
        raise SystemExit(f"growth not linear in m (ratio {ratio:.3f})")
    cfg = {"workload": "overflow_4000", "m": 4000, "n": 4000, "seed": SEED, "kind": "growth", "upper": s,
           "log2_growth_m1000": round(g1, 1), "log2_growth_m2000": round(g2, 1),
           "log2_growth_m4000_extrapolated": round(g1 + (g2 - g1) * 3, 1),
           "made_by": "tests/golden/calibrate_overflow.py (FP64 oracle only)"}
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "overflow_config.json"), "w") as f:
        json.dump(cfg, f, indent=1)
    print(cfg)


if __name__ == "__main__":
    main()

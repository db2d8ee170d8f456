"""Write the oracle's singular values for the full-size workloads.

Each fixture is the FP64 oracle's reduction (Section III, Algorithms 1 and 2,
sequential sweep order) of one seeded synthetic band, followed by the singular
values of the resulting bidiagonal from its Golub-Kahan tridiagonal through
LAPACK sterf (a library step).  The oracle's own Sturm bisection is run on the
same bidiagonal as a cross-check, and the two must agree to 1e-13 * sigma_max
before anything is written.  Nothing here calls the GPU library.

Workloads (n = 32768, N(0, 1) entries, seed 2):
  f"sigma_n32768_b128_seed2.npy"          the band the benchmark reduces
  f"sigma_n32768_b{b}_seed2_graded.npy"   b in {32, 64, 128}, row i scaled by
                                          10^(-6 i / n) (the precision study)

    python tests/golden/make_full_size_sigma.py [name ...]

One reduction takes about ten minutes of one host core; each name runs in its
own process.
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

N = 32768
SEED = 2
TW = 16
CASES = {
    "sigma_n32768_b128_seed2": (128, False),
    "sigma_n32768_b32_seed2_graded": (32, True),
    "sigma_n32768_b64_seed2_graded": (64, True),
    "sigma_n32768_b128_seed2_graded": (128, True),
}


def make(name: str) -> None:
    import bandgen
    import oracle
    b, graded = CASES[name]
    ab = bandgen.random_band(N, b, seed=SEED, graded=graded)
    t0 = time.perf_counter()
    d, e, cnt = oracle.band_to_bidiag(ab, b, TW)
    t1 = time.perf_counter()
    s_lapack = oracle.bidiag_sigma(d, e, method="lapack")
    s_bisect = oracle.bidiag_sigma(d, e, method="bisect")
    t2 = time.perf_counter()
    dev = float(np.max(np.abs(s_lapack - s_bisect)) / s_lapack[0])
    if not dev <= 1e-13:
        raise SystemExit(f"{name}: sterf and bisection disagree by {dev:.3e} * sigma_max")
    np.save(os.path.join(HERE, name + ".npy"), s_lapack)
    print(f"{name}: reduction {t1 - t0:.0f} s ({cnt['flops'] / (t1 - t0) / 1e9:.2f} GFLOP/s), "
          f"sigma {t2 - t1:.0f} s, sterf vs bisection {dev:.2e} * sigma_max, "
          f"sigma_max {s_lapack[0]:.6e}, sigma_min {s_lapack[-1]:.3e}", flush=True)


if __name__ == "__main__":
    names = sys.argv[1:] or list(CASES)
    for nm in names:
        make(nm)

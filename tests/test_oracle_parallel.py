"""The OpenMP form of the oracle (the cycle schedule of Section III-A with the
row-bulges of each cycle on several host threads) gives the sequential
oracle's d and e bit for bit: under the lag the row-bulges of a cycle touch
disjoint elements, so no thread count and no split of a cycle can change a
single rounding.  It is the CPU baseline's parallel form, so it is pinned to
the sequential oracle here rather than used as a reference itself."""
import os
import subprocess
import sys

import numpy as np
import pytest

import bandgen
import oracle

CASES = [(1, 0, 4), (2, 1, 4), (50, 3, 2), (200, 16, 8), (300, 40, 16), (257, 33, 32),
         (400, 64, 32), (129, 128, 32), (600, 7, 3)]


@pytest.mark.parametrize("n,b,tw", CASES)
def test_parallel_equals_sequential(n, b, tw):
    ab = bandgen.random_band(n, b, seed=7 * n + b)
    d0, e0, c0 = oracle.band_to_bidiag(ab, b, tw)
    d1, e1, c1, thr = oracle.band_to_bidiag_parallel(ab, b, tw)
    assert thr >= 1
    assert np.array_equal(d0, d1) and np.array_equal(e0, e1)
    assert c1["steps"] == c0["steps"] and c1["stages"] == c0["stages"]
    assert c1["flops"] == c0["flops"] and c1["out_of_band"] == 0


@pytest.mark.parametrize("threads", [1, 3, 8])
def test_thread_count_does_not_change_bits(threads):
    """Fresh interpreters with OMP_NUM_THREADS fixed: every count gives the
    same bits as the sequential oracle (a race would show at some count)."""
    code = (
        "import sys, numpy as np; sys.path[:0] = [%r, %r]\n"
        "import bandgen, oracle\n"
        "ab = bandgen.random_band(700, 48, seed=3)\n"
        "d0, e0, _ = oracle.band_to_bidiag(ab, 48, 16)\n"
        "d1, e1, _, t = oracle.band_to_bidiag_parallel(ab, 48, 16)\n"
        "assert t == %d, t\n"
        "assert np.array_equal(d0, d1) and np.array_equal(e0, e1)\n"
    ) % (os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
         os.path.dirname(os.path.abspath(__file__)), threads)
    env = dict(os.environ, OMP_NUM_THREADS=str(threads))
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]


def test_step_budget_stops_after_a_cycle():
    n, b, tw = 500, 32, 8
    ab = bandgen.random_band(n, b, seed=11)
    _, _, full = oracle.band_to_bidiag(ab, b, tw)
    _, _, c, _ = oracle.band_to_bidiag_parallel(ab, b, tw, max_steps=1000)
    # at least the budget, at most one more cycle's worth (<= n row-bulges)
    assert 1000 <= c["steps"] < 1000 + n
    assert c["steps"] < full["steps"]
    _, _, z, _ = oracle.band_to_bidiag_parallel(ab, b, tw, max_steps=0)
    assert z["steps"] == 0

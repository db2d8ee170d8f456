"""Host model of the bulge kernel's data movement (Section III, Algorithm 2).

The GPU row-bulge reads its right and left panels from the working band,
keeps the next row-bulge's first rows (the bulge row and the d rows below it)
in shared memory instead of storing and reloading them, defers the left
panel's tail columns, and writes everything back at different points.  This
test replays exactly that pattern of loads, carried values and stores,
sequentially with plain numpy arithmetic, and requires the result to match the
oracle.  A mistake in which element goes where (a carried row reloaded from a
stale copy, a store skipped without a carry) changes the singular values by
O(1), far beyond rounding; the planted variants at the end check that.
"""
import numpy as np
import pytest

import bandgen
import oracle


def _larfg(x):
    alpha = x[0]
    xi = np.linalg.norm(x[1:])
    if xi == 0.0:
        v = np.zeros_like(x)
        v[0] = 1.0
        return v, 0.0, alpha
    beta = -np.copysign(np.hypot(alpha, xi), 1.0 if alpha >= 0 else -1.0)
    v = x / (alpha - beta)
    v[0] = 1.0
    return v, (beta - alpha) / beta, beta


def _sweep_steps(n, bw, d, R):
    s = 0
    while R + (bw - d) + s * bw < n - 1:
        s += 1
    return s


def kernel_dataflow(A, b, tw, carried_rows="d+1", carry=True):
    """Dense replay of the kernel's panel traffic; returns (d, e)."""
    n = A.shape[0]
    W = A.astype(np.float64).copy()
    bw = b
    while bw > 1:
        d = min(tw, bw - 1)
        tail_start = bw - 1 if bw - d >= 2 else d + bw
        for R in range(n - 1):
            ns = _sweep_steps(n, bw, d, R)
            kept = None                        # next right panel rows 0..d (shared memory)
            for s in range(ns):
                c = R + (bw - d) + s * bw
                m = min(d + 1, n - c)
                r0 = R if s == 0 else c - bw
                nr = c + m - r0
                ncols = min(n - 1, c + m - 1 + bw) - c
                pre_hi = min(tail_start, ncols + 1)
                # A: loads (rows already kept are not reloaded)
                lo = 0 if kept is None else (d + 1 if carried_rows == "d+1" else m)
                RP = np.empty((nr, m))
                RP[lo:] = W[r0 + lo:c + m, c:c + m]
                if kept is not None:
                    RP[:lo] = kept[:lo, :m]
                LP = np.zeros((m, ncols + 1))
                LP[:, m:pre_hi] = W[c:c + m, c + m:c + pre_hi]
                # B, C: right reflector; rows above c to the band, the rest to LP
                v, tau, beta = _larfg(RP[0].copy())
                RP = RP - tau * np.outer(RP @ v, v)
                RP[0] = 0.0
                RP[0, 0] = beta
                W[r0:c, c:c + m] = RP[:c - r0]
                LP[:, :m] = RP[c - r0:]
                # D, E: left reflector on the columns loaded up front
                vl, taul, betal = _larfg(LP[:, 0].copy())
                LP[:, 1:pre_hi] -= taul * np.outer(vl, vl @ LP[:, 1:pre_hi])
                LP[:, 0] = 0.0
                LP[0, 0] = betal
                carry_out = carry and s + 1 < ns
                keep_lo = min(pre_hi, bw) if carry_out else pre_hi
                W[c:c + m, c:c + keep_lo] = LP[:, :keep_lo]
                nxt = np.zeros((d + 1, d + 1)) if carry_out else None
                if carry_out:
                    nxt[:m, :pre_hi - keep_lo] = LP[:, keep_lo:pre_hi]
                # tail: columns from tail_start, read from the band now
                for jj in range(pre_hi, ncols + 1):
                    a = W[c:c + m, c + jj].copy()
                    a -= taul * vl * (vl @ a)
                    if carry_out and jj >= bw:
                        nxt[:m, jj - bw] = a
                    else:
                        W[c:c + m, c + jj] = a
                kept = nxt
        bw -= d
    return np.diag(W).copy(), np.diag(W, 1).copy()


CASES = [(12, 3, 2), (20, 5, 2), (40, 5, 2), (60, 8, 3), (41, 3, 1), (64, 16, 16), (57, 9, 4),
         (33, 7, 6), (50, 12, 5), (45, 17, 8)]


@pytest.mark.parametrize("n,b,tw", CASES)
def test_kernel_dataflow_matches_oracle(n, b, tw):
    ab = bandgen.random_band(n, b, seed=n + 7 * b)
    d, e = kernel_dataflow(bandgen.dense_from_band(ab, b), b, tw)
    do, eo, _ = oracle.band_to_bidiag(ab, b, tw)
    scale = np.max(np.abs(do)) + np.max(np.abs(eo))
    assert np.max(np.abs(np.abs(d) - np.abs(do))) <= 1e-12 * scale
    assert np.max(np.abs(np.abs(e) - np.abs(eo))) <= 1e-12 * scale


@pytest.mark.parametrize("n,b,tw", [(12, 3, 2), (40, 5, 2), (60, 8, 3)])
def test_planted_carry_mistake_is_caught(n, b, tw):
    # reloading the carried rows from m instead of d + 1 (wrong at the end of
    # the matrix, where m < d + 1) reads stale values that were never stored
    ab = bandgen.random_band(n, b, seed=n + 7 * b)
    d, e = kernel_dataflow(bandgen.dense_from_band(ab, b), b, tw, carried_rows="m")
    do, eo, _ = oracle.band_to_bidiag(ab, b, tw)
    s = oracle.bidiag_sigma(d, e)
    so = oracle.bidiag_sigma(do, eo)
    assert np.max(np.abs(s - so)) > 1e-6 * so[0]

"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each check is independent of the oracle's own code: closed-form spectra,
identities of the reduction, invariants of orthogonal transformations,
brute-force SVD, and the paper's dependency argument for the cycle schedule
(Section III-A).  The mutation tests at the end plant plausible mistakes in a
copy of the oracle and require that some pin catches each one.
"""
import os
import subprocess

import numpy as np
import pytest

import bandgen
import oracle


def _sigma_dense(a):
    return np.linalg.svd(a, compute_uv=False)


# --------------------------------------------------------------------- inputs

def test_toeplitz_generator_matches_closed_form():
    n = 300
    ab = bandgen.toeplitz_qr_band(n, 4)
    a = bandgen.dense_from_band(ab, 4)
    assert np.allclose(np.tril(a, -1), 0.0)
    assert np.all(ab[:, :2] == 0.0)          # offsets 3, 4 are empty
    s = _sigma_dense(a)
    ref = bandgen.toeplitz_singular_values(n)
    assert np.max(np.abs(s - ref)) < 1e-13


def test_prescribed_sigma_generator():
    ab, sig = bandgen.prescribed_sigma_band(96, 8, "logarithmic", seed=5)
    a = bandgen.dense_from_band(ab, 8)
    assert np.max(np.abs(_sigma_dense(a) - sig)) < 1e-13


# ------------------------------------------------------ bidiagonal sigma pins

def test_bidiag_sigma_closed_form_all_ones():
    # B = I + N (ones on the diagonal and superdiagonal): sigma_k = 2 cos(k pi/(2n+1))
    for n in (1, 2, 7, 100, 513):
        s = oracle.bidiag_sigma(np.ones(n), np.ones(n - 1), method="bisect")
        k = np.arange(1, n + 1)
        ref = 2.0 * np.cos(k * np.pi / (2 * n + 1))
        assert np.max(np.abs(s - ref)) < 1e-14 * 2, n


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _golden(name):
    return np.loadtxt(os.path.join(GOLDEN, name), comments="#")


def test_golden_bidiag_ones():
    # stored closed form (tests/golden/make_golden.py)
    s = oracle.bidiag_sigma(np.ones(10), np.ones(9), method="bisect")
    assert np.max(np.abs(s - _golden("bidiag_ones_sigma_n10.txt"))) < 4e-15


def test_golden_toeplitz_reduction():
    # the whole reduction of Toeplitz R (b = 2 and b = 64 storage, several TW)
    # against the stored closed form
    ref = _golden("toeplitz_sigma_n64.txt")
    for b, tw in ((2, 1), (2, 16), (64, 16), (64, 5)):
        d, e, _ = oracle.band_to_bidiag(bandgen.toeplitz_qr_band(64, b), b, tw)
        s = oracle.bidiag_sigma(d, e, method="bisect")
        assert np.max(np.abs(s - ref)) <= 1e-14 * ref[0], (b, tw)


def test_bidiag_sigma_against_numpy_and_lapack():
    rng = np.random.default_rng(11)
    for n in (3, 50, 400):
        d = rng.standard_normal(n)
        e = rng.standard_normal(n - 1)
        dense = np.diag(d) + np.diag(e, 1)
        ref = _sigma_dense(dense)
        s1 = oracle.bidiag_sigma(d, e, method="bisect")
        s2 = oracle.bidiag_sigma(d, e, method="lapack")
        assert np.max(np.abs(s1 - ref)) < 1e-13 * ref[0]
        assert np.max(np.abs(s2 - ref)) < 1e-13 * ref[0]


def test_bidiag_sigma_graded_relative_accuracy():
    # bisection on the Golub-Kahan form keeps tiny singular values accurate
    n = 60
    d = 10.0 ** (-np.arange(n) / 6.0)
    e = 0.5 * d[1:]
    s = oracle.bidiag_sigma(d, e, method="bisect")
    ref = _sigma_dense(np.diag(d) + np.diag(e, 1))
    assert np.max(np.abs(s - ref) / ref) < 1e-9


def test_jacobi_sigma_pins():
    rng = np.random.default_rng(3)
    diag = np.abs(rng.standard_normal(20))
    assert np.allclose(oracle.jacobi_sigma(np.diag(diag)), np.sort(diag)[::-1], atol=1e-15)
    a = rng.standard_normal((40, 40))
    assert np.max(np.abs(oracle.jacobi_sigma(a) - _sigma_dense(a))) < 1e-13 * _sigma_dense(a)[0]


def test_power_sums_against_dense():
    ab = bandgen.random_band(120, 9, seed=4)
    a = bandgen.dense_from_band(ab, 9)
    p1, p2 = oracle.band_power_sums(ab, 9)
    g = a.T @ a
    assert abs(p1 - np.sum(a * a)) < 1e-12 * p1
    assert abs(p2 - np.sum(g * g)) < 1e-12 * p2


# ----------------------------------------------------------- reduction pins

@pytest.mark.parametrize("n,b,tw", [(40, 6, 2), (60, 8, 3), (64, 16, 16), (50, 5, 1),
                                    (70, 12, 5), (33, 7, 4), (64, 63, 16), (17, 30, 4)])
def test_reduction_bruteforce_jacobi(n, b, tw):
    ab = bandgen.random_band(n, b, seed=100 + n + b)
    a = bandgen.dense_from_band(ab, b)
    d, e, cnt = oracle.band_to_bidiag(ab, b, tw, check_fill=True)
    ref = oracle.jacobi_sigma(a)
    s = oracle.bidiag_sigma(d, e)
    assert cnt["out_of_band"] == 0 and cnt["fill_violations"] == 0
    assert np.max(np.abs(s - ref)) <= 1e-13 * ref[0]


@pytest.mark.parametrize("n,b,tw", [(512, 16, 16), (300, 40, 16), (257, 33, 8), (400, 64, 32)])
def test_reduction_against_numpy_svd(n, b, tw):
    ab = bandgen.random_band(n, b, seed=n)
    a = bandgen.dense_from_band(ab, b)
    d, e, _ = oracle.band_to_bidiag(ab, b, tw)
    s = oracle.bidiag_sigma(d, e)
    ref = _sigma_dense(a)
    assert np.max(np.abs(s - ref)) <= 1e-13 * ref[0]


@pytest.mark.parametrize("n,b", [(64, 2), (300, 8), (1000, 16)])
def test_toeplitz_closed_form(n, b):
    ab = bandgen.toeplitz_qr_band(n, b)
    d, e, _ = oracle.band_to_bidiag(ab, b, 16)
    s = oracle.bidiag_sigma(d, e)
    ref = bandgen.toeplitz_singular_values(n)
    assert np.max(np.abs(s - ref)) <= 1e-13 * ref[0]


@pytest.mark.parametrize("profile", ["arithmetic", "logarithmic", "quartercircle"])
def test_prescribed_sigma(profile):
    # Section V-A: known singular values survive the band reduction
    ab, sig = bandgen.prescribed_sigma_band(128, 12, profile, seed=7)
    d, e, _ = oracle.band_to_bidiag(ab, 12, 4)
    s = oracle.bidiag_sigma(d, e)
    assert np.max(np.abs(s - sig)) <= 1e-13


def test_first_row_and_column_identities():
    # Q and P never touch row/column 0: d[0] = A[0,0] exactly and
    # |e[0]| = ||A[0, 1:]|| (row 0 of B is row 0 of A P).
    for (n, b, tw) in [(200, 20, 8), (97, 31, 16), (64, 5, 2)]:
        ab = bandgen.random_band(n, b, seed=b)
        a = bandgen.dense_from_band(ab, b)
        d, e, _ = oracle.band_to_bidiag(ab, b, tw)
        assert d[0] == a[0, 0]
        r = np.linalg.norm(a[0, 1:])
        assert abs(abs(e[0]) - r) <= 1e-14 * r


def test_trivial_bandwidths():
    ab = bandgen.random_band(50, 0, seed=1)
    d, e, cnt = oracle.band_to_bidiag(ab, 0, 4)
    assert np.array_equal(d, ab[:, 0]) and np.all(e == 0.0) and cnt["steps"] == 0
    ab = bandgen.random_band(50, 1, seed=2)
    d, e, cnt = oracle.band_to_bidiag(ab, 1, 4)
    assert np.array_equal(d, ab[:, 1]) and np.array_equal(e, ab[1:, 0]) and cnt["steps"] == 0
    d, e, _ = oracle.band_to_bidiag(np.array([[3.5]]), 0, 1)
    assert d[0] == 3.5 and e.size == 0


def test_invariants_and_exact_zeros():
    n, b, tw = 400, 24, 8
    ab = bandgen.random_band(n, b, seed=9, graded=True)
    d, e, cnt, work = oracle.band_to_bidiag(ab, b, tw, return_work=True, check_fill=True)
    assert cnt["fill_violations"] == 0 and cnt["out_of_band"] == 0
    up = b + tw
    # every stored entry off the bidiagonal is exactly zero
    for j in range(n):
        for off in range(work.shape[1]):
            i = off - up + j
            if 0 <= i < n and i != j and i != j - 1:
                assert work[j, off] == 0.0
    p1a, p2a = oracle.band_power_sums(ab, b)
    p1b, p2b = oracle.bidiag_power_sums(d, e)
    assert abs(p1a - p1b) <= 1e-13 * p1a
    assert abs(p2a - p2b) <= 1e-13 * p2a


def test_intermediate_stage_bandwidth():
    # after one stage the matrix is upper banded with bandwidth b - d
    n, b, tw = 150, 20, 6
    ab = bandgen.random_band(n, b, seed=12)
    a = bandgen.dense_from_band(ab, b)
    _, _, cnt, work = oracle.band_to_bidiag(ab, b, tw, max_stages=1, return_work=True)
    up = b + tw
    dense = np.zeros((n, n))
    for j in range(n):
        for off in range(work.shape[1]):
            i = off - up + j
            if 0 <= i < n:
                dense[i, j] = work[j, off]
    assert cnt["stages"] == 1
    assert np.all(np.tril(dense, -1) == 0.0)
    assert np.all(np.triu(dense, b - tw + 1) == 0.0)
    assert np.max(np.abs(_sigma_dense(dense) - _sigma_dense(a))) < 1e-13 * _sigma_dense(a)[0]


def test_cycle_schedule_dependency_argument():
    # Section III-A: with a separation of 3 cycles between consecutive sweeps
    # no two concurrent row-bulges overlap, so the cycle schedule reproduces
    # the sequential result exactly; 2 cycles suffice only when the stage does
    # not end at bandwidth 1.
    for (n, b, tw) in [(90, 10, 3), (120, 33, 16), (64, 16, 16)]:
        ab = bandgen.random_band(n, b, seed=n * 7)
        d0, e0, _ = oracle.band_to_bidiag(ab, b, tw)
        d3, e3, _ = oracle.band_to_bidiag(ab, b, tw, order=3)
        d2, e2, _ = oracle.band_to_bidiag(ab, b, tw, order=-2)
        assert np.array_equal(d0, d3) and np.array_equal(e0, e3)
        assert np.array_equal(d0, d2) and np.array_equal(e0, e2)
        # lag 2 on the final stage (bandwidth 1) is not a valid schedule
        d2x, e2x, _ = oracle.band_to_bidiag(ab, b, tw, order=2)
        assert not (np.array_equal(d0, d2x) and np.array_equal(e0, e2x))


def test_scaling_extremes_and_zero_input():
    n, b, tw = 80, 10, 4
    ab = bandgen.random_band(n, b, seed=21)
    d, e, _ = oracle.band_to_bidiag(ab, b, tw)
    s = oracle.bidiag_sigma(d, e)
    for scale in (1e-300, 1e300, 2.0 ** -1060):
        ds, es, _ = oracle.band_to_bidiag(ab * scale, b, tw)
        assert np.all(np.isfinite(ds)) and np.all(np.isfinite(es))
        ss = oracle.bidiag_sigma(ds / scale, es / scale) if scale > 1e-310 else None
        if ss is not None:
            assert np.max(np.abs(ss - s)) <= 1e-12 * s[0], scale
    dz, ez, _ = oracle.band_to_bidiag(np.zeros((n, b + 1)), b, tw)
    assert np.all(dz == 0.0) and np.all(ez == 0.0)


def test_step_and_work_counts():
    # number of row-bulges: sum over stages and sweeps of the closed-form count
    n, b, tw = 300, 40, 16
    _, _, cnt = oracle.band_to_bidiag(bandgen.random_band(n, b, seed=1), b, tw)
    steps = 0
    bw = b
    stages = 0
    while bw > 1:
        d = min(tw, bw - 1)
        for r in range(n - 1):
            c0 = r + bw - d
            if c0 < n - 1:
                steps += (n - 2 - c0) // bw + 1
        bw -= d
        stages += 1
    assert cnt["steps"] == steps and cnt["stages"] == stages


# ------------------------------------------------------------ mutation tests

_MUTATIONS = [
    ("drop tau", "w *= tau;\n        for (int k = 0; k < m; k++) *at(A, r, c + k)",
     "w *= 1.0;\n        for (int k = 0; k < m; k++) *at(A, r, c + k)"),
    ("wrong sign of beta", "if (alpha >= 0.0) beta = -beta;          /*",
     "if (alpha < 0.0) beta = -beta;          /*"),
    ("stride = new bandwidth", "const int c = R + (bw - d) + s * bw;",
     "const int c = R + (bw - d) + s * (bw - d);"),
    ("left reflector one column short", "const int jmax = (c + m - 1 + bw < n - 1) ? c + m - 1 + bw : n - 1;",
     "const int jmax = (c + m - 2 + bw < n - 1) ? c + m - 2 + bw : n - 1;"),
    ("right reflector skips the last row", "for (int r = r0 + 1; r <= c + m - 1; r++) {",
     "for (int r = r0 + 1; r <= c + m - 2; r++) {"),
    ("transposed left application", "w += v[k] * *at(A, c + k, j);",
     "w += v[k] * *at(A, j, c + k);"),
    ("first row-bulge starts at row c - bw", "const int r0 = (s == 0) ? R : c - bw;",
     "const int r0 = c - bw;"),
]


@pytest.mark.parametrize("name,old,new", _MUTATIONS, ids=[m[0] for m in _MUTATIONS])
def test_pins_catch_planted_mistakes(tmp_path, name, old, new):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "bulge_oracle.c")).read()
    assert old in src, name
    mut = src.replace(old, new, 1)
    c_path = tmp_path / "mut.c"
    c_path.write_text(mut)
    so = tmp_path / "mut.so"
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                           "-o", str(so), str(c_path), "-lm"])
    import ctypes
    lib = ctypes.CDLL(str(so))
    dp = ctypes.POINTER(ctypes.c_double)
    lib.oracle_band_to_bidiag.argtypes = [
        ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, dp, dp,
        ctypes.POINTER(oracle._Counts), ctypes.c_int, ctypes.c_int, ctypes.c_longlong,
        dp, ctypes.c_int]

    def run(ab, b, tw):
        ab = np.ascontiguousarray(ab)
        n = ab.shape[0]
        d = np.zeros(n)
        e = np.zeros(n)
        cnt = oracle._Counts()
        lib.oracle_band_to_bidiag(n, b, tw, oracle._ptr(ab), ab.shape[1], oracle._ptr(d),
                                  oracle._ptr(e), ctypes.byref(cnt), 0, -1, -1, None, 1)
        return d, e[: n - 1], cnt

    caught = []
    # pin 1: brute-force singular values
    n, b, tw = 48, 9, 3
    ab = bandgen.random_band(n, b, seed=5)
    d, e, cnt = run(ab, b, tw)
    ref = oracle.jacobi_sigma(bandgen.dense_from_band(ab, b))
    if not np.all(np.isfinite(d)) or not np.all(np.isfinite(e)):
        caught.append("nonfinite")
    else:
        s = oracle.bidiag_sigma(d, e)
        caught.append(np.max(np.abs(s - ref)) > 1e-12 * ref[0])
    # pin 2: fill confinement / storage bounds
    caught.append(cnt.fill_violations != 0 or cnt.out_of_band != 0)
    # pin 3: closed-form Toeplitz spectrum
    ab = bandgen.toeplitz_qr_band(200, 6)
    d, e, _ = run(ab, 6, 4)
    if np.all(np.isfinite(d)) and np.all(np.isfinite(e)):
        s = oracle.bidiag_sigma(d, e)
        caught.append(np.max(np.abs(s - bandgen.toeplitz_singular_values(200))) > 1e-12)
    else:
        caught.append(True)
    assert any(bool(c) for c in caught), f"mutation '{name}' not caught"

"""Parity of the sm_103a path with the FP64 oracle at the full benchmark size,
at the benchmark's own launch configuration, and on the inputs the reflector
code's safe scaling is written for.

Full size (n = 32768): every singular value of the GPU's bidiagonal is
compared with the oracle's, stored in tests/golden/ by
tests/golden/make_full_size_sigma.py (oracle reduction, then LAPACK sterf on
the Golub-Kahan tridiagonal, cross-checked against the oracle's bisection).
The bar is the accuracy target: max |dsigma| <= 1e-11 ||A||_2 in FP64 and
2e-4 ||A||_2 in FP32.
"""
import os

import numpy as np
import pytest

import bandgen
import oracle
from gpu_util import TOL_F32, TOL_F64, run_gpu

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _golden(name):
    return np.load(os.path.join(GOLDEN, name + ".npy"))


def _sigma_lapack(d, e):
    return oracle.bidiag_sigma(np.asarray(d, np.float64), np.asarray(e, np.float64), method="lapack")


def _tuning(n, b, dtype, which):
    if which == "default":
        return None
    from paper_2510_12705_gb300 import tuner
    tun, _ = tuner.tuning_for(n, b, dtype)
    return tun


# ------------------------------------------------ n = 32768 against fixtures

@pytest.mark.parametrize("tuning", ["default", "bench"])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_full_size_bench_band_every_sigma(dtype, tuning):
    # the band bench.py reduces: n = 32768, b = 128, iid N(0, 1), seed 2
    ref = _golden("sigma_n32768_b128_seed2")
    ab = bandgen.random_band(32768, 128, seed=2)
    d, e, st = run_gpu(ab, 128, dtype, tuning=_tuning(32768, 128, dtype, tuning))
    assert st == 0
    s = _sigma_lapack(d, e)
    err = float(np.max(np.abs(s - ref)) / ref[0])
    assert err <= (TOL_F64 if dtype == "f64" else TOL_F32), err


@pytest.mark.parametrize("b", [32, 64, 128])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_full_size_graded_every_sigma(b, dtype):
    # precision study: row i scaled by 10^(-6 i / n), seed 2
    ref = _golden(f"sigma_n32768_b{b}_seed2_graded")
    ab = bandgen.random_band(32768, b, seed=2, graded=True)
    d, e, st = run_gpu(ab, b, dtype, tuning=_tuning(32768, b, dtype, "bench"))
    assert st == 0
    s = _sigma_lapack(d, e)
    err = float(np.max(np.abs(s - ref)) / ref[0])
    assert err <= (TOL_F64 if dtype == "f64" else TOL_F32), err


# --------------------------- the bench's kernel instance on a live oracle run

def test_bench_kernel_instance_n8192_b128():
    # FP64, TW = 32, CTA size and panel shape of the n = 32768, b = 128 bench
    # launch (the same stages 128 -> 96 -> 64 -> 32 -> 1), at a size the
    # oracle reduces in about half a minute
    n, b = 8192, 128
    ab = bandgen.random_band(n, b, seed=2)
    d0, e0, _ = oracle.band_to_bidiag(ab, b, 32)
    ref = _sigma_lapack(d0, e0)
    tun = _tuning(32768, 128, "f64", "bench")
    d, e, st = run_gpu(ab, b, "f64", tuning=tun)
    assert st == 0
    err = float(np.max(np.abs(_sigma_lapack(d, e) - ref)) / ref[0])
    assert err <= TOL_F64, err
    d, e, st = run_gpu(ab.astype(np.float32).astype(np.float64), b, "f32",
                       tuning=_tuning(32768, 128, "f32", "bench"))
    assert st == 0
    err = float(np.max(np.abs(_sigma_lapack(d, e) - ref)) / ref[0])
    assert err <= TOL_F32, err


# ---------------------------------------------------------- scaling extremes

N_S, B_S, TW_S = 300, 24, 8


@pytest.fixture(scope="module")
def scale_case():
    ab = bandgen.random_band(N_S, B_S, seed=21)
    d, e, _ = oracle.band_to_bidiag(ab, B_S, TW_S)
    return ab, oracle.bidiag_sigma(d, e)


@pytest.mark.parametrize("scale", [1e-300, 1e300, 2.0 ** -1000, 2.0 ** 1000])
def test_f64_extreme_scales(scale_case, scale):
    # norms of these vectors under- or overflow without the power-of-two
    # scaling of the reflector generation; the result must be the scaled one
    ab, s0 = scale_case
    d, e, st = run_gpu(ab * scale, B_S, "f64", tuning={"tw": TW_S})
    assert st == 0
    assert np.all(np.isfinite(d)) and np.all(np.isfinite(e))
    s = oracle.bidiag_sigma(d / scale, e / scale)
    assert np.max(np.abs(s - s0)) <= TOL_F64 * s0[0]


def test_f64_subnormal_band():
    # entries ~2^-1060: subnormal, about 14 significant bits.  Compare with
    # the oracle on the same input, after scaling both bidiagonals by 2^1060
    # (exact), within the absolute error subnormal arithmetic allows: each
    # entry goes through at most a few hundred roundings of 2^-1075.
    ab = bandgen.random_band(N_S, B_S, seed=21) * 2.0 ** -1060
    d0, e0, _ = oracle.band_to_bidiag(ab, B_S, TW_S)
    d, e, st = run_gpu(ab, B_S, "f64", tuning={"tw": TW_S})
    assert st == 0
    assert np.all(np.isfinite(d)) and np.all(np.isfinite(e))
    up = 2.0 ** 530                    # applied twice: 2^1060 itself overflows
    s0 = oracle.bidiag_sigma(d0 * up * up, e0 * up * up)
    s = oracle.bidiag_sigma(d * up * up, e * up * up)
    assert s0[0] > 0
    # a few hundred half-ulps of 2^-1074, rescaled: 2^-14 per unit of sigma_max / 10
    assert np.max(np.abs(s - s0)) <= 2e-2 * s0[0]
    assert d[0] == ab[0, B_S]


@pytest.mark.parametrize("scale", [1e-30, 1e30])
def test_f32_extreme_scales(scale_case, scale):
    # FP32 storage: squares of 1e+-30 leave the FP32 range, the FP64 reflector
    # generation must not
    ab, _ = scale_case
    ab32 = (ab * scale).astype(np.float32)
    d0, e0, _ = oracle.band_to_bidiag(ab32.astype(np.float64) / scale, B_S, TW_S)
    s0 = oracle.bidiag_sigma(d0, e0)
    d, e, st = run_gpu(ab32.astype(np.float64), B_S, "f32", tuning={"tw": TW_S})
    assert st == 0
    assert np.all(np.isfinite(d)) and np.all(np.isfinite(e))
    s = oracle.bidiag_sigma(d / scale, e / scale)
    assert np.max(np.abs(s - s0)) <= TOL_F32 * s0[0]


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_all_zero_band(dtype):
    d, e, st = run_gpu(np.zeros((N_S, B_S + 1)), B_S, dtype, tuning={"tw": TW_S})
    assert st == 0
    assert np.all(d == 0.0) and np.all(e == 0.0)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("tw", [8, 32])
def test_zero_rows_and_columns(dtype, tw):
    # whole rows and columns of A set to zero: zero reflector tails (tau = 0)
    # inside the chase, and exact splits of the bidiagonal
    n, b = 400, 40
    ab = bandgen.random_band(n, b, seed=33)
    a = bandgen.dense_from_band(ab, b)
    a[100:104, :] = 0.0
    a[:, 250:253] = 0.0
    a[390, :] = 0.0
    ab = bandgen.band_from_dense(a, b)
    d0, e0, _ = oracle.band_to_bidiag(ab, b, tw)
    s0 = oracle.bidiag_sigma(d0, e0)
    d, e, st = run_gpu(ab, b, dtype, tuning={"tw": tw})
    assert st == 0
    s = oracle.bidiag_sigma(d, e)
    tol = TOL_F64 if dtype == "f64" else TOL_F32
    assert np.max(np.abs(s - s0)) <= tol * s0[0]
    # five zero rows: rank <= n - 5, kept up to rounding
    assert np.sum(s <= (1e-12 if dtype == "f64" else 1e-5) * s0[0]) >= 5


def test_f32_subnormal_band_stays_finite():
    # FP32 entries around 1e-40 are subnormal: reflector vectors whose norm is
    # below the FP32 range of 1 / (|alpha| + ||x||) must still give finite
    # reflectors (the same happens near the end of random triangular bands,
    # whose trailing singular values underflow in FP32)
    ab = bandgen.random_band(N_S, B_S, seed=21) * 1e-40
    for tw in (TW_S, 16, 32):
        d, e, st = run_gpu(ab, B_S, "f32", tuning={"tw": tw})
        assert st == 0
        assert np.all(np.isfinite(d)) and np.all(np.isfinite(e))
        assert float(np.max(np.abs(d))) <= 1e-37

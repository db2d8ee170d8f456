"""GPU singular values of the bidiagonal (bb_bidiag_sigma) against the
oracle's Sturm bisection, closed forms, LAPACK's tridiagonal solver, and the
whole GPU-resident band -> bidiagonal -> sigma pipeline on the Toeplitz
instance whose singular values are known in closed form."""
import os

import numpy as np
import pytest
import torch

import bandgen
import oracle

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def bb():
    import paper_2510_12705_gb300 as bb
    from paper_2510_12705_gb300 import build
    build.build()
    return bb


def _gpu_sigma(bb, d, e, dtype=torch.float64):
    dd = torch.from_numpy(np.asarray(d, np.float64)).to("cuda", dtype)
    ee = torch.from_numpy(np.asarray(e if len(e) else [0.0], np.float64)).to("cuda", dtype)
    s = bb.bb_bidiag_sigma(dd, ee)
    torch.cuda.synchronize()
    return s.cpu().numpy()


@pytest.mark.parametrize("n", [1, 2, 3, 17, 100, 1000])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_matches_oracle_bisection(bb, n, dtype):
    rng = np.random.default_rng(n)
    d = rng.standard_normal(n)
    e = rng.standard_normal(n - 1)
    if dtype == "f32":   # the oracle sees the same (rounded) values the GPU widens
        d, e = d.astype(np.float32).astype(np.float64), e.astype(np.float32).astype(np.float64)
    s = _gpu_sigma(bb, d, e, torch.float64 if dtype == "f64" else torch.float32)
    ref = oracle.bidiag_sigma(d, e, method="bisect")
    assert np.all(np.diff(s) <= 0)
    assert np.max(np.abs(s - ref)) <= 2e-15 * ref[0] * max(1.0, np.log2(n))


def test_closed_forms(bb):
    ref = np.loadtxt(os.path.join(GOLDEN, "bidiag_ones_sigma_n10.txt"), comments="#")
    assert np.max(np.abs(_gpu_sigma(bb, np.ones(10), np.ones(9)) - ref)) < 4e-15
    n = 2000
    k = np.arange(1, n + 1)
    s = _gpu_sigma(bb, np.ones(n), np.ones(n - 1))
    assert np.max(np.abs(s - 2.0 * np.cos(k * np.pi / (2 * n + 1)))) < 1e-14


def test_zeros_and_extreme_scales(bb):
    # exact zeros split B; tiny and huge entries stress the pivot guard
    d = np.array([1.0, 0.0, 3.0, 2.0, 1e-200, 5.0])
    e = np.array([0.0, 2.0, 0.0, 1e-150, 1.0])
    ref = oracle.bidiag_sigma(d, e, method="bisect")
    s = _gpu_sigma(bb, d, e)
    assert np.max(np.abs(s - ref)) <= 1e-15 * ref[0]
    s = _gpu_sigma(bb, d * 1e250, e * 1e250)
    assert np.max(np.abs(s - ref * 1e250)) <= 1e-15 * ref[0] * 1e250


def test_against_lapack_large(bb):
    n = 8192
    rng = np.random.default_rng(3)
    d = rng.standard_normal(n) * 10.0 ** rng.uniform(-3, 0, n)
    e = rng.standard_normal(n - 1)
    s = _gpu_sigma(bb, d, e)
    ref = oracle.bidiag_sigma(d, e, method="lapack")
    assert np.max(np.abs(s - ref)) <= 1e-13 * ref[0]


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_gpu_resident_pipeline_toeplitz(bb, dtype):
    # band (Toeplitz QR factor, closed-form sigma) -> bidiagonal -> sigma, all on the GPU
    n, b = 4096, 64
    ab = bandgen.toeplitz_qr_band(n, b)
    t = torch.float64 if dtype == "f64" else torch.float32
    band = torch.from_numpy(ab).to("cuda", t)
    d = torch.empty(n, device="cuda", dtype=t)
    e = torch.empty(n - 1, device="cuda", dtype=t)
    bb.band_to_bidiag(band, b, d, e)
    s = bb.bb_bidiag_sigma(d, e).cpu().numpy()
    assert bb.bb_device_status(reset=True) == 0
    ref = bandgen.toeplitz_singular_values(n)
    tol = 1e-11 if dtype == "f64" else 2e-4
    assert np.max(np.abs(s - ref)) <= tol * ref[0]

"""Parity of the sm_103a path (through the C ABI) with the CPU oracle.

The bar (BASELINE accuracy targets): singular values of the output
bidiagonal within 1e-11 * ||A||_2 of the oracle's in FP64 and 2e-4 * ||A||_2
in FP32.  The FP64 path runs the same reflector sequence as the oracle, so for
small n its |d| and |e| are also compared element by element.
"""
import numpy as np
import pytest

import bandgen
import oracle
from gpu_util import TOL_F32, TOL_F64, run_gpu, sigma_err

pytestmark = pytest.mark.gpu


def _oracle_sigma(ab, b, tw=16):
    d, e, _ = oracle.band_to_bidiag(ab, b, tw)
    return d, e, oracle.bidiag_sigma(d, e)


# ------------------------------------------------------------ small configs

def test_config_512_b16_f64_elementwise():
    # n = 512, b = 16, N(0,1), seed 0: plain FP64 form
    ab = bandgen.random_band(512, 16, seed=0)
    d0, e0, s0 = _oracle_sigma(ab, 16, 16)
    d, e, st = run_gpu(ab, 16, "f64")
    assert st == 0
    err, _ = sigma_err(d, e, s0)
    assert err <= TOL_F64
    # same reflector sequence: |d|, |e| agree up to rounding order
    scale = s0[0]
    assert np.max(np.abs(np.abs(d) - np.abs(d0))) <= 1e-10 * scale
    assert np.max(np.abs(np.abs(e) - np.abs(e0))) <= 1e-10 * scale
    a = bandgen.dense_from_band(ab, 16)
    assert d[0] == a[0, 0]


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("n,b,tw", [
    (1, 0, 16), (2, 1, 16), (3, 2, 16), (5, 4, 2), (17, 30, 4),       # tiny / b >= n
    (64, 63, 16), (100, 7, 3), (257, 33, 8), (333, 40, 16), (300, 64, 32),
    (129, 16, 16), (200, 100, 32), (511, 48, 5), (640, 128, 16), (96, 9, 1),
])
def test_parity_small(n, b, tw, dtype):
    ab = bandgen.random_band(n, b, seed=3 * n + b)
    _, _, s0 = _oracle_sigma(ab, b, tw)
    d, e, st = run_gpu(ab, b, dtype, tuning={"tw": tw})
    assert st == 0
    err, _ = sigma_err(d, e, s0)
    assert err <= (TOL_F64 if dtype == "f64" else TOL_F32), err


@pytest.mark.parametrize("tpb", [64, 128, 256, 512])
@pytest.mark.parametrize("sif", [1, 3, 0])
def test_parity_launch_shapes(tpb, sif):
    # any CTA size and any number of persistent CTAs (1 = fully serial) give
    # the same bidiagonal: the schedule is serialisable
    ab = bandgen.random_band(300, 24, seed=77)
    d_ref, e_ref, _ = run_gpu(ab, 24, "f64", tuning={"tw": 8, "tpb": 128})
    d, e, st = run_gpu(ab, 24, "f64", tuning={"tw": 8, "tpb": tpb, "sweeps_in_flight": sif})
    assert st == 0
    assert np.array_equal(d, d_ref) and np.array_equal(e, e_ref)


def test_trivial_bandwidths_exact():
    ab = bandgen.random_band(200, 0, seed=1)
    d, e, st = run_gpu(ab, 0, "f64")
    assert st == 0 and np.array_equal(d, ab[:, 0]) and np.all(e == 0)
    ab = bandgen.random_band(200, 1, seed=2)
    d, e, st = run_gpu(ab, 1, "f64")
    assert st == 0 and np.array_equal(d, ab[:, 1]) and np.array_equal(e, ab[1:, 0])


def test_ldab_padding_and_rows_above_matrix_ignored():
    n, b = 150, 12
    ab = bandgen.random_band(n, b, seed=8, ldab=b + 5)
    ab[:, b + 1:] = 1e30                  # padding rows must not be read
    for j in range(b):
        ab[j, : b - j] = np.nan           # slots above row 0 must not be read
    clean = ab.copy()
    clean[:, b + 1:] = 0.0
    for j in range(b):
        clean[j, : b - j] = 0.0
    _, _, s0 = _oracle_sigma(clean[:, : b + 1], b)
    d, e, st = run_gpu(ab, b, "f64")
    assert st == 0
    assert sigma_err(d, e, s0)[0] <= TOL_F64


def test_repeatable_bitwise():
    ab = bandgen.random_band(1000, 32, seed=5)
    r1 = run_gpu(ab, 32, "f64")
    r2 = run_gpu(ab, 32, "f64")
    assert np.array_equal(r1[0], r2[0]) and np.array_equal(r1[1], r2[1])


@pytest.mark.parametrize("profile", ["arithmetic", "logarithmic", "quartercircle"])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_prescribed_sigma(profile, dtype):
    # Section V-A methodology: known singular values in [0, 1]
    ab, sig = bandgen.prescribed_sigma_band(512, 32, profile, seed=11)
    d, e, st = run_gpu(ab, 32, dtype)
    assert st == 0
    err, _ = sigma_err(d, e, sig)
    assert err <= (TOL_F64 if dtype == "f64" else TOL_F32)


# --------------------------------------------------- n = 8192, b = 64 config

@pytest.fixture(scope="module")
def cfg8192():
    ab = bandgen.random_band(8192, 64, seed=1)
    d, e, cnt = oracle.band_to_bidiag(ab, 64, 16)
    return ab, oracle.bidiag_sigma(d, e)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_config_8192_b64(cfg8192, dtype):
    ab, s0 = cfg8192
    d, e, st = run_gpu(ab, 64, dtype)
    assert st == 0
    err, _ = sigma_err(d, e, s0)
    assert err <= (TOL_F64 if dtype == "f64" else TOL_F32), err


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_toeplitz_closed_form_8192(dtype):
    # R of the QR of tridiag(-1, 2, -1) in b = 64 storage: sigma = 2 - 2 cos(k pi/(n+1))
    n = 8192
    ab = bandgen.toeplitz_qr_band(n, 64)
    ref = bandgen.toeplitz_singular_values(n)
    d, e, st = run_gpu(ab, 64, dtype)
    assert st == 0
    err, _ = sigma_err(d, e, ref)
    assert err <= (TOL_F64 if dtype == "f64" else TOL_F32), err


# ------------------------------------------- full size n = 32768, b = 128

def _top_sigma(ab, b, k=3):
    # largest singular values of the banded A by ARPACK on A^T A (library step)
    from scipy.sparse import diags
    from scipy.sparse.linalg import eigsh
    n = ab.shape[0]
    offs = list(range(0, b + 1))
    a = diags([ab[k:, b - k] for k in offs], offs, shape=(n, n), format="csr")
    w = eigsh((a.T @ a).tocsr(), k=k, which="LA", tol=1e-15, return_eigenvectors=False)
    return np.sort(np.sqrt(w))[::-1]


@pytest.fixture(scope="module")
def full_size():
    ab = bandgen.random_band(32768, 128, seed=2, graded=False)
    p1, p2 = oracle.band_power_sums(ab, 128)
    return ab, p1, p2, _top_sigma(ab, 128)


@pytest.mark.parametrize("tuning", ["default", "bench"])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_full_size_properties(full_size, dtype, tuning):
    # properties that hold at any size: d[0] = A[0,0]; |e[0]| = ||A[0,1:]||;
    # sum sigma^2 and sum sigma^4 preserved; the largest singular values.
    # "bench": the hyperparameters bench.py times (the learned tuner's pick)
    from paper_2510_12705_gb300 import tuner
    ab, p1, p2, top = full_size
    tun = None
    if tuning == "bench":
        tun, _ = tuner.tuning_for(32768, 128, dtype)
    d, e, st = run_gpu(ab, 128, dtype, tuning=tun)
    assert st == 0
    a00 = ab[0, 128]
    r0 = np.sqrt(sum(ab[k, 128 - k] ** 2 for k in range(1, 129)))   # ||A[0, 1:]||
    tol = 1e-12 if dtype == "f64" else 1e-5
    if dtype == "f64":
        assert d[0] == a00
    else:
        assert d[0] == np.float32(a00)
    assert abs(abs(e[0]) - r0) <= tol * 10 * r0
    q1, q2 = oracle.bidiag_power_sums(d, e)
    assert abs(q1 - p1) <= tol * p1
    assert abs(q2 - p2) <= 10 * tol * p2
    s = oracle.bidiag_sigma(d, e, method="lapack")[: len(top)]
    assert np.max(np.abs(s - top)) <= (TOL_F64 if dtype == "f64" else TOL_F32) * top[0]


# ------------------------------------------------------------- error paths

def test_nonfinite_input_reported():
    import paper_2510_12705_gb300 as bb
    ab = bandgen.random_band(100, 8, seed=4)
    ab[50, 3] = np.nan
    _, _, st = run_gpu(ab, 8, "f64")
    assert bb.BB_ERR_NONFINITE in bb.status_bits(st)
    ab[50, 3] = np.inf
    _, _, st = run_gpu(ab, 8, "f32")
    assert bb.BB_ERR_NONFINITE in bb.status_bits(st)


def test_bounded_wait_times_out_and_context_survives():
    # fault injected on the host side: sweep 0 never reports progress, so the
    # other sweeps' bounded waits run out (50 ms without progress), the launch
    # aborts and records BB_ERR_TIMEOUT; the next call works normally.
    import paper_2510_12705_gb300 as bb
    ab = bandgen.random_band(400, 16, seed=6)
    _, _, st = run_gpu(ab, 16, "f64", tuning={"flags": bb.BB_FLAG_INJECT_STALL, "timeout_s": 0.05})
    assert bb.BB_ERR_TIMEOUT in bb.status_bits(st)
    _, _, s0 = _oracle_sigma(ab, 16)
    d, e, st = run_gpu(ab, 16, "f64")
    assert st == 0 and sigma_err(d, e, s0)[0] <= TOL_F64


# ------------------------------------------------------- workspace / e2e

def test_caller_workspace_and_streams():
    import torch
    import paper_2510_12705_gb300 as bb
    ab = bandgen.random_band(700, 40, seed=12)
    d_ref, e_ref, _ = run_gpu(ab, 40, "f64")
    band = torch.from_numpy(ab).cuda()
    ws = torch.empty(bb.band_to_bidiag_workspace_size(700, 40, bb.BB_F64), dtype=torch.uint8,
                     device="cuda")
    s = torch.cuda.Stream()
    d = torch.empty(700, dtype=torch.float64, device="cuda")
    e = torch.empty(699, dtype=torch.float64, device="cuda")
    with torch.cuda.stream(s):
        bb.band_to_bidiag_ex(band, 40, d, e, workspace=ws, stream=s)
    s.synchronize()
    assert np.array_equal(d.cpu().numpy(), d_ref) and np.array_equal(e.cpu().numpy(), e_ref)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_host_entry_point_matches_device(dtype):
    import paper_2510_12705_gb300 as bb
    ab = bandgen.random_band(900, 50, seed=13).astype(dtype)
    d, e = bb.band_to_bidiag_host(ab, 50)
    d2, e2, st = run_gpu(ab.astype(np.float64), 50, "f64" if dtype == np.float64 else "f32")
    assert st == 0
    assert np.array_equal(d.astype(np.float64), d2) and np.array_equal(e.astype(np.float64), e2)


# ------------------------------------------- kernel variants of one reduction

VARIANTS = [{"group": -1}, {"group": 1}, {"group": 4}, {"group": 16},
            {"teams": 2}, {"teams": 4}, {"group": 16, "teams": 8}]


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("n,b,tw", [(640, 128, 16), (511, 48, 5), (333, 40, 16), (1500, 64, 32),
                                    (97, 96, 32), (700, 20, 3)])
def test_kernel_variants(n, b, tw, dtype):
    # the group kernel (K sweeps per CTA on the split stages), the team kernel
    # (W sweeps per CTA on the last stage) and the per-sweep kernel reduce the
    # same matrix to bidiagonals with the oracle's singular values
    ab = bandgen.random_band(n, b, seed=7 * n + b)
    _, _, s0 = _oracle_sigma(ab, b, tw)
    for var in VARIANTS:
        d, e, st = run_gpu(ab, b, dtype, tuning={"tw": tw, **var})
        assert st == 0, var
        err, _ = sigma_err(d, e, s0)
        assert err <= (TOL_F64 if dtype == "f64" else TOL_F32), (var, err)


@pytest.mark.parametrize("var", [{"group": 8}, {"teams": 4}])
def test_variant_launch_shapes_bitwise(var):
    # any CTA count gives the same bits (each kernel's order of operations is
    # fixed by its protocol, not by the schedule)
    ab = bandgen.random_band(500, 40, seed=91)
    ref = run_gpu(ab, 40, "f64", tuning={"tw": 8, **var})
    for sif in (1, 5):
        d, e, st = run_gpu(ab, 40, "f64", tuning={"tw": 8, "sweeps_in_flight": sif, **var})
        assert st == 0 and np.array_equal(d, ref[0]) and np.array_equal(e, ref[1])

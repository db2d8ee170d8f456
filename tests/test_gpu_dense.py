"""Stage 1 on the GPU (dense_to_band, Sections II and V-A) against the stage-1
oracle, and the paper's accuracy experiment end to end on the device:
prescribed-sigma dense matrix -> band -> bidiagonal -> singular values."""
import numpy as np
import pytest

import bandgen
from gpu_util import TOL_F32, TOL_F64
from oracle import dense_band

pytestmark = pytest.mark.gpu


def _gpu_band(a, b, dtype):
    """GPU dense_to_band of the dense numpy matrix a; returns the LAPACK 'U'
    band (n, b+1) as float64 and the dense upper-band matrix."""
    import torch
    import paper_2510_12705_gb300 as bb
    n = a.shape[0]
    # column-major A: the row-major tensor of A^T
    at = torch.from_numpy(np.ascontiguousarray(a.T)).to("cuda", dtype)
    band = torch.full((n, b + 1), float("nan"), device="cuda", dtype=dtype)
    bb.dense_to_band(at, b, band)
    torch.cuda.synchronize()
    ab = band.double().cpu().numpy()
    return ab, bandgen.dense_from_band(ab, b)


@pytest.mark.parametrize("dtype_name", ["f64", "f32"])
@pytest.mark.parametrize("n,b", [(1, 1), (2, 1), (37, 5), (300, 16), (513, 64), (200, 1), (130, 129), (96, 32)])
def test_dense_to_band_matches_oracle(n, b, dtype_name):
    import torch
    dtype = torch.float64 if dtype_name == "f64" else torch.float32
    a = np.random.default_rng(n * 31 + b).standard_normal((n, n))
    if dtype_name == "f32":
        a = a.astype(np.float32).astype(np.float64)      # the input both sides see
    ab, bd = _gpu_band(a, b, dtype)
    assert np.all(np.isfinite(ab))
    # the output is a band: nothing below the diagonal, band slots above row 0 zero
    for j in range(n):
        assert np.all(ab[j, : max(0, b - j)] == 0.0)
    s0 = np.linalg.svd(a, compute_uv=False)
    s1 = np.linalg.svd(bd, compute_uv=False)
    tol = TOL_F64 if dtype_name == "f64" else TOL_F32
    assert np.max(np.abs(s1 - s0)) <= tol * s0[0]
    if dtype_name == "f64":
        # same reflector sequence as the oracle: the band agrees elementwise
        # (rounding only; no sign is free here since every alpha is far from 0)
        bo = dense_band.dense_to_band(a, b)
        assert np.max(np.abs(bd - bo)) <= 1e-10 * np.linalg.norm(a)


@pytest.mark.parametrize("dtype_name", ["f64", "f32"])
def test_already_banded_and_zero_inputs(dtype_name):
    import torch
    dtype = torch.float64 if dtype_name == "f64" else torch.float32
    n, b = 150, 8
    rng = np.random.default_rng(4)
    a = np.triu(np.tril(rng.standard_normal((n, n)), 5))     # bandwidth 5 <= b
    if dtype_name == "f32":
        a = a.astype(np.float32).astype(np.float64)
    _, bd = _gpu_band(a, b, dtype)
    assert np.array_equal(bd, a)                                # every reflector is the identity
    _, bz = _gpu_band(np.zeros((n, n)), b, dtype)
    assert np.array_equal(bz, np.zeros((n, n)))


@pytest.mark.parametrize("profile", ["arithmetic", "logarithmic", "quartercircle"])
@pytest.mark.parametrize("dtype_name", ["f64", "f32"])
def test_prescribed_sigma_end_to_end_on_device(profile, dtype_name):
    """Section V-A's accuracy experiment: A = U diag(sigma) V^T with
    prescribed sigma; dense -> band (dense_to_band), band -> bidiagonal
    (band_to_bidiag) and bidiagonal -> sigma (bb_bidiag_sigma), all on the GPU;
    the result is compared with the prescribed values."""
    import torch
    import paper_2510_12705_gb300 as bb
    dtype = torch.float64 if dtype_name == "f64" else torch.float32
    n, b = 1024, 32
    a, sigma = bandgen.prescribed_sigma_dense(n, profile, seed=5)
    at = torch.from_numpy(np.ascontiguousarray(a.T)).to("cuda", dtype)
    band = torch.empty((n, b + 1), device="cuda", dtype=dtype)
    d = torch.empty(n, device="cuda", dtype=dtype)
    e = torch.empty(n - 1, device="cuda", dtype=dtype)
    s_out = torch.empty(n, device="cuda", dtype=torch.float64)
    ws = torch.empty(int(bb.lib().bb_bidiag_sigma_workspace_size(n)), dtype=torch.uint8, device="cuda")
    bb.dense_to_band(at, b, band)
    bb.band_to_bidiag(band, b, d, e)
    bb.bb_bidiag_sigma(d, e, s_out, ws)
    torch.cuda.synchronize()
    assert bb.bb_device_status(reset=True) == 0
    s = s_out.cpu().numpy()
    tol = TOL_F64 if dtype_name == "f64" else TOL_F32
    assert np.max(np.abs(s - sigma)) <= tol * sigma[0], np.max(np.abs(s - sigma))


def test_caller_workspace_and_errors():
    import torch
    import paper_2510_12705_gb300 as bb
    n, b = 200, 12
    a = np.random.default_rng(9).standard_normal((n, n))
    at = torch.from_numpy(np.ascontiguousarray(a.T)).cuda()
    ws = torch.empty(bb.dense_to_band_workspace_size(n, b, bb.BB_F64), dtype=torch.uint8, device="cuda")
    band1 = torch.empty((n, b + 1), device="cuda", dtype=torch.float64)
    band2 = torch.empty((n, b + 1), device="cuda", dtype=torch.float64)
    bb.dense_to_band(at, b, band1, workspace=ws)
    bb.dense_to_band(at, b, band2)
    torch.cuda.synchronize()
    assert torch.equal(band1, band2)                 # same kernels, same order: same bits
    small = torch.empty(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(bb.BBError) as ei:
        bb.dense_to_band(at, b, band1, workspace=small)
    assert ei.value.code == bb.BB_ERR_WORKSPACE


@pytest.mark.parametrize("dtype_name", ["f64", "f32"])
@pytest.mark.parametrize("n,b", [(1, 1), (64, 16), (300, 1), (513, 64), (130, 129)])
def test_stage1_factors(n, b, dtype_name):
    """dense_to_band_qp: the same band as dense_to_band, and orthogonal Q, P
    with Q^T A P = B."""
    import torch
    import paper_2510_12705_gb300 as bb
    dtype = torch.float64 if dtype_name == "f64" else torch.float32
    a = np.random.default_rng(3 * n + b).standard_normal((n, n))
    if dtype_name == "f32":
        a = a.astype(np.float32).astype(np.float64)
    at = torch.from_numpy(np.ascontiguousarray(a.T)).to("cuda", dtype)
    band = torch.empty((n, b + 1), device="cuda", dtype=dtype)
    q = torch.full((n, n), float("nan"), device="cuda", dtype=dtype)
    p = torch.full((n, n), float("nan"), device="cuda", dtype=dtype)
    bb.dense_to_band_qp(at, b, band, q, p)
    band_ref = torch.empty((n, b + 1), device="cuda", dtype=dtype)
    bb.dense_to_band(at, b, band_ref)
    torch.cuda.synchronize()
    assert torch.equal(band, band_ref)
    bd = bandgen.dense_from_band(band.double().cpu().numpy(), b)
    qm, pm = q.double().cpu().numpy().T, p.double().cpu().numpy().T
    tol = TOL_F64 if dtype_name == "f64" else TOL_F32
    eye = np.eye(n)
    assert np.max(np.abs(qm.T @ qm - eye)) <= tol
    assert np.max(np.abs(pm.T @ pm - eye)) <= tol
    assert np.max(np.abs(qm.T @ a @ pm - bd)) <= tol * np.linalg.norm(a, 2)


@pytest.mark.parametrize("dtype_name", ["f64", "f32"])
def test_dense_svd_vectors_end_to_end(dtype_name):
    """Singular vectors of a dense prescribed-sigma matrix: stage 1 factors
    (dense_to_band_qp), stage 2 factors (band_to_bidiag_vectors) and the
    bidiagonal's singular vectors (host LAPACK, test only) give A = U S V^T."""
    import torch
    import paper_2510_12705_gb300 as bb
    dtype = torch.float64 if dtype_name == "f64" else torch.float32
    n, b = 512, 32
    a, sigma = bandgen.prescribed_sigma_dense(n, "quartercircle", seed=8)
    if dtype_name == "f32":
        a = a.astype(np.float32).astype(np.float64)
    at = torch.from_numpy(np.ascontiguousarray(a.T)).to("cuda", dtype)
    band = torch.empty((n, b + 1), device="cuda", dtype=dtype)
    q1 = torch.empty((n, n), device="cuda", dtype=dtype)
    p1 = torch.empty((n, n), device="cuda", dtype=dtype)
    q2 = torch.empty((n, n), device="cuda", dtype=dtype)
    p2 = torch.empty((n, n), device="cuda", dtype=dtype)
    d = torch.empty(n, device="cuda", dtype=dtype)
    e = torch.empty(n - 1, device="cuda", dtype=dtype)
    bb.dense_to_band_qp(at, b, band, q1, p1)
    bb.band_to_bidiag_vectors(band, b, d, e, q2, p2)
    torch.cuda.synchronize()
    assert bb.bb_device_status(reset=True) == 0
    Q = q1.double().cpu().numpy().T @ q2.double().cpu().numpy().T
    P = p1.double().cpu().numpy().T @ p2.double().cpu().numpy().T
    ub, s, vbt = np.linalg.svd(np.diag(d.double().cpu().numpy()) + np.diag(e.double().cpu().numpy(), 1))
    u, v = Q @ ub, P @ vbt.T
    tol = TOL_F64 if dtype_name == "f64" else TOL_F32
    assert np.max(np.abs(s - np.linalg.svd(a, compute_uv=False))) <= tol * s[0]
    assert np.max(np.abs(u @ np.diag(s) @ v.T - a)) <= tol * s[0]
    assert np.max(np.abs(u.T @ u - np.eye(n))) <= tol and np.max(np.abs(v.T @ v - np.eye(n))) <= tol

"""Singular vectors of the band stage (band_to_bidiag_vectors): the reflectors
the GPU kernels store, back-transformed on the GPU into Q and P with
Q^T A P = bidiag(d, e) (Section VII), checked against what the mathematics
fixes: the factors are orthogonal, their first columns and rows are e1, they
reconstruct A exactly up to rounding, and with the bidiagonal's own singular
vectors they give a full SVD of A."""
import numpy as np
import pytest

import bandgen
from gpu_util import TOL_F32, TOL_F64

pytestmark = pytest.mark.gpu


def _run(ab, b, dtype, tuning=None):
    import torch
    import paper_2510_12705_gb300 as bb
    n = ab.shape[0]
    band = torch.from_numpy(ab).to("cuda", dtype)
    d = torch.empty(n, device="cuda", dtype=dtype)
    e = torch.empty(max(n - 1, 1), device="cuda", dtype=dtype)
    q = torch.full((n, n), float("nan"), device="cuda", dtype=dtype)
    p = torch.full((n, n), float("nan"), device="cuda", dtype=dtype)
    bb.band_to_bidiag_vectors(band, b, d, e, q, p, tuning=tuning)
    torch.cuda.synchronize()
    st = bb.bb_device_status(reset=True)
    # the tensors hold the column-major factors: as row-major arrays, Q^T and P^T
    return (d.double().cpu().numpy(), e[: n - 1].double().cpu().numpy(), q.double().cpu().numpy().T,
            p.double().cpu().numpy().T, st)


CASES = [(200, 16, 8, None), (300, 40, 16, None), (513, 64, 32, None), (257, 33, 32, -1), (100, 3, 2, None),
         (64, 1, 16, None), (1, 0, 16, None), (150, 20, 5, 4)]


@pytest.mark.parametrize("dtype_name", ["f64", "f32"])
@pytest.mark.parametrize("n,b,tw,group", CASES)
def test_factors_reconstruct_the_band(n, b, tw, group, dtype_name):
    import torch
    dtype = torch.float64 if dtype_name == "f64" else torch.float32
    ab = bandgen.random_band(n, b, seed=17 * n + b)
    if dtype_name == "f32":
        ab = ab.astype(np.float32).astype(np.float64)
    tun = {"tw": tw} if group is None else {"tw": tw, "group": group}
    d, e, q, p, st = _run(ab, b, dtype, tun)
    assert st == 0
    a = bandgen.dense_from_band(ab, b)
    bmat = np.diag(d) + np.diag(e, 1)
    norm = max(np.linalg.norm(a, 2), 1e-300)
    tol = TOL_F64 if dtype_name == "f64" else TOL_F32
    eye = np.eye(n)
    assert np.max(np.abs(q.T @ q - eye)) <= tol
    assert np.max(np.abs(p.T @ p - eye)) <= tol
    assert np.max(np.abs(q.T @ a @ p - bmat)) <= tol * norm
    # row and column 0 are never touched by a reflector
    assert np.array_equal(q[:, 0], eye[:, 0]) and np.array_equal(q[0], eye[0])
    assert np.array_equal(p[:, 0], eye[:, 0]) and np.array_equal(p[0], eye[0])


@pytest.mark.parametrize("dtype_name", ["f64", "f32"])
def test_full_svd_at_the_bench_kernel_instance(dtype_name):
    """n = 2048, b = 128, TW = 32 with the default group kernel (24 sweeps per
    CTA on the split stages) and the per-sweep last stage: A = U diag(s) V^T
    with U = Q U_B, V = P V_B from the bidiagonal's SVD (host LAPACK, test
    only); d and e equal band_to_bidiag's bitwise."""
    import torch
    import paper_2510_12705_gb300 as bb
    dtype = torch.float64 if dtype_name == "f64" else torch.float32
    n, b = 2048, 128
    ab = bandgen.random_band(n, b, seed=23)
    if dtype_name == "f32":
        ab = ab.astype(np.float32).astype(np.float64)
    d, e, q, p, st = _run(ab, b, dtype, {"tw": 32})
    assert st == 0
    band = torch.from_numpy(ab).to("cuda", dtype)
    d2 = torch.empty(n, device="cuda", dtype=dtype)
    e2 = torch.empty(n - 1, device="cuda", dtype=dtype)
    bb.band_to_bidiag_ex(band, b, d2, e2, tuning={"tw": 32})
    torch.cuda.synchronize()
    assert np.array_equal(d, d2.double().cpu().numpy()) and np.array_equal(e, e2.double().cpu().numpy())
    a = bandgen.dense_from_band(ab, b)
    ub, s, vbt = np.linalg.svd(np.diag(d) + np.diag(e, 1))
    u, v = q @ ub, p @ vbt.T
    tol = TOL_F64 if dtype_name == "f64" else TOL_F32
    assert np.max(np.abs(u @ np.diag(s) @ v.T - a)) <= tol * s[0]
    assert np.max(np.abs(a @ v[:, :8] - u[:, :8] * s[:8])) <= tol * s[0]

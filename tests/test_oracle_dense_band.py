"""Pins of the stage-1 oracle (dense -> upper band, Section II / V-A): what the
mathematics fixes, checked without the oracle's own formulas."""
import numpy as np
import pytest

from oracle import dense_band


def _rand(n, seed):
    return np.random.default_rng(seed).standard_normal((n, n))


@pytest.mark.parametrize("n,b", [(1, 1), (2, 1), (7, 1), (9, 3), (40, 6), (61, 7), (64, 16), (33, 32), (50, 49)])
def test_singular_values_preserved(n, b):
    a = _rand(n, n * 100 + b)
    bb = dense_band.dense_to_band(a, b)
    s0 = np.linalg.svd(a, compute_uv=False)
    s1 = np.linalg.svd(bb, compute_uv=False)
    assert np.max(np.abs(s1 - s0)) <= 1e-13 * s0[0]


@pytest.mark.parametrize("n,b", [(40, 6), (61, 7), (30, 1), (17, 16)])
def test_exact_band_structure_and_frobenius(n, b):
    a = _rand(n, 7 * n + b)
    bb = dense_band.dense_to_band(a, b)
    assert np.count_nonzero(np.tril(bb, -1)) == 0
    assert np.count_nonzero(np.triu(bb, b + 1)) == 0
    assert abs(np.linalg.norm(bb) - np.linalg.norm(a)) <= 1e-14 * n * np.linalg.norm(a)


@pytest.mark.parametrize("n,b", [(25, 4), (31, 1), (12, 11)])
def test_orthogonal_factors_reconstruct(n, b):
    a = _rand(n, 3 * n + b)
    bb, q, p = dense_band.dense_to_band(a, b, with_qp=True)
    eye = np.eye(n)
    assert np.max(np.abs(q.T @ q - eye)) <= 1e-14 * n
    assert np.max(np.abs(p.T @ p - eye)) <= 1e-14 * n
    assert np.max(np.abs(q.T @ a @ p - bb)) <= 1e-14 * n * np.linalg.norm(a)
    # the first row and column of P are e1: row 0's first entry is untouched by P
    assert np.allclose(p[:, 0], eye[:, 0]) and np.allclose(p[0], eye[0])


@pytest.mark.parametrize("n,b,bw", [(30, 5, 5), (30, 5, 3), (20, 1, 1), (16, 8, 0)])
def test_already_banded_input_is_unchanged(n, b, bw):
    # every reflector then has a zero tail (tau = 0, identity)
    a = np.triu(np.tril(_rand(n, n + bw), bw))
    assert np.array_equal(dense_band.dense_to_band(a, b), a)


def test_full_bandwidth_is_lapack_qr():
    # b >= n - 1: one panel, a plain Householder QR; LAPACK's geqrf uses the
    # same reflector convention, so B is its R
    n = 24
    a = _rand(n, 5)
    bb = dense_band.dense_to_band(a, n - 1)
    r = np.linalg.qr(a, mode="r")
    assert np.max(np.abs(bb - r)) <= 1e-13 * np.linalg.norm(a)


def test_larfg_contract():
    x = np.array([3.0, 4.0])
    tau, v, beta = dense_band.larfg(x.copy())
    assert beta == -5.0 and v[0] == 1.0
    h = np.eye(2) - tau * np.outer(v, v)
    assert np.allclose(h @ x, [beta, 0.0]) and np.allclose(h @ h.T, np.eye(2))
    tau0, v0, beta0 = dense_band.larfg(np.array([-2.0, 0.0, 0.0]))
    assert tau0 == 0.0 and beta0 == -2.0 and np.array_equal(v0, [1.0, 0.0, 0.0])
    _, _, bz = dense_band.larfg(np.array([0.0, 1.0]))
    assert bz == -1.0                    # sign(0) = +1


def test_planted_mistakes_are_caught(monkeypatch):
    # a reflector applied from the right to the panel rows only (forgetting the
    # rows below) breaks the singular values; a wrong sign of tau breaks them too
    n, b = 30, 4
    a = _rand(n, 11)
    s0 = np.linalg.svd(a, compute_uv=False)

    def bad_rows(a_in, b_in):
        a2 = np.array(a_in, dtype=np.float64, copy=True)
        nn = a2.shape[0]
        for k in range(0, nn, b_in):
            w = min(b_in, nn - k)
            for j in range(w):
                c = k + j
                tau, v, beta = dense_band.larfg(a2[c:, c].copy())
                a2[c:, c] = 0.0
                a2[c, c] = beta
                a2[c:, c + 1:] -= tau * np.outer(v, v @ a2[c:, c + 1:])
            for i in range(w):
                r, c0 = k + i, k + w + i
                if c0 >= nn:
                    break
                tau, u, beta = dense_band.larfg(a2[r, c0:].copy())
                a2[r, c0:] = 0.0
                a2[r, c0] = beta
                rows = slice(r + 1, k + w)            # planted: rows below the panel skipped
                a2[rows, c0:] -= tau * np.outer(a2[rows, c0:] @ u, u)
        return a2

    s_bad = np.linalg.svd(bad_rows(a, b), compute_uv=False)
    assert np.max(np.abs(s_bad - s0)) > 1e-3 * s0[0]

    real = dense_band.larfg

    def flipped(x):
        tau, v, beta = real(x)
        return -tau, v, beta

    monkeypatch.setattr(dense_band, "larfg", flipped)
    s_flip = np.linalg.svd(dense_band.dense_to_band(a, b), compute_uv=False)
    assert np.max(np.abs(s_flip - s0)) > 1e-3 * s0[0]

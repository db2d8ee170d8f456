"""Seeded synthetic inputs for the band -> bidiagonal reduction.

This module is shared by the CPU oracle's tests and by the GPU path's tests
and benchmark.  It only *produces* input matrices; it holds none of the
reduction's arithmetic (no reflectors, no bulge chasing).

Storage convention (LAPACK 'U' band storage, 0-based): an upper-banded n x n
matrix A with bandwidth b (A[i, j] != 0 only for 0 <= j - i <= b) is held in a
(b + 1) x n column-major array ``ab`` with leading dimension ``ldab >= b + 1``:

    A[i, j] == ab[(b + i - j) + j * ldab]

As a numpy array of shape (n, ldab) (one row per matrix column), that is
``ab2d[j, b + i - j]``.  Entries of ``ab`` that fall outside the matrix
(i < 0) are zero.

The workloads: random bands with iid N(0, 1) entries (the paper times
synthetic bands without stating their distribution), graded rows that stress
small singular values, a structured closed-form instance, and matrices with
prescribed singular values (Section V-A, the accuracy experiment).
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "band_from_dense",
    "dense_from_band",
    "random_band",
    "toeplitz_qr_band",
    "toeplitz_singular_values",
    "prescribed_sigma_band",
    "batch_problems",
    "tuner_grid",
]


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def band_from_dense(a: np.ndarray, b: int, ldab: int | None = None) -> np.ndarray:
    """Pack the upper band of a dense square matrix into (n, ldab) storage."""
    n = a.shape[0]
    ldab = b + 1 if ldab is None else ldab
    ab = np.zeros((n, ldab), dtype=a.dtype)
    for k in range(b + 1):           # k = j - i, the k-th superdiagonal
        j = np.arange(k, n)
        ab[j, b - k] = a[j - k, j]
    return ab


def dense_from_band(ab: np.ndarray, b: int) -> np.ndarray:
    """Unpack (n, ldab) band storage into a dense square matrix."""
    n = ab.shape[0]
    a = np.zeros((n, n), dtype=ab.dtype)
    for k in range(b + 1):
        j = np.arange(k, n)
        a[j - k, j] = ab[j, b - k]
    return a


def random_band(n: int, b: int, seed: int, *, graded: bool = False,
                ldab: int | None = None, dtype=np.float64) -> np.ndarray:
    """Upper band with iid N(0, 1) entries (PCG64 stream ``seed``).

    The normals are drawn column by column, superdiagonal offsets 0..b, so a
    given (n, b, seed) always yields the same matrix.  With ``graded`` row i
    is scaled by 10**(-6 i / n), which spreads the singular values over six
    decades and stresses the small ones.
    """
    ldab = b + 1 if ldab is None else ldab
    g = _rng(seed).standard_normal((n, b + 1))
    ab = np.zeros((n, ldab), dtype=np.float64)
    ab[:, : b + 1] = g
    # zero the entries above row 0 (i = j - k < 0)
    for j in range(min(b, n)):
        ab[j, : b - j] = 0.0
    if graded:
        for k in range(b + 1):
            j = np.arange(k, n)
            i = j - k
            ab[j, b - k] *= 10.0 ** (-6.0 * i / n)
    return ab.astype(dtype, copy=False)


def toeplitz_qr_band(n: int, b: int, a: float = 2.0, c: float = -1.0,
                     ldab: int | None = None) -> np.ndarray:
    """R factor of the QR factorisation of the tridiagonal Toeplitz T(c, a, c).

    T is symmetric tridiagonal with diagonal ``a`` and off-diagonals ``c``;
    its eigenvalues are a + 2 c cos(k pi / (n + 1)), k = 1..n.  With T = Q R
    (Givens rotations, FP64), R is upper triangular with bandwidth 2 and
    R^T R = T^T T = T^2, so the singular values of R are |eig(T)|.  R is
    stored in band storage of width ``b`` >= 2; offsets 3..b are zero, which
    exercises the zero-reflector paths of the reduction.
    """
    if b < 2:
        raise ValueError("toeplitz_qr_band needs b >= 2")
    ldab = b + 1 if ldab is None else ldab
    # rows of the upper-triangular factor, held as three diagonals r0, r1, r2
    r0 = np.zeros(n)
    r1 = np.zeros(n)
    r2 = np.zeros(n)
    # working copy of the current row k: (diag, super) and next row (sub, diag, super)
    d_k, s_k = a, c          # row k entries at columns k, k+1
    for k in range(n):
        if k == n - 1:
            r0[k] = d_k
            break
        # row k+1 of T: (c at col k, a at col k+1, c at col k+2)
        sub, dn, sn = c, a, (c if k + 2 < n else 0.0)
        h = math.hypot(d_k, sub)
        cs, sn_ = d_k / h, sub / h
        # rotate rows k and k+1
        r0[k] = h
        r1[k] = cs * s_k + sn_ * dn
        r2[k] = sn_ * sn            # row k gains an entry at column k+2
        d_next = -sn_ * s_k + cs * dn
        s_next = cs * sn
        d_k, s_k = d_next, s_next
    ab = np.zeros((n, ldab))
    ab[:, b] = r0
    ab[1:, b - 1] = r1[: n - 1]
    ab[2:, b - 2] = r2[: n - 2]
    return ab


def toeplitz_singular_values(n: int, a: float = 2.0, c: float = -1.0) -> np.ndarray:
    """Closed form |a + 2 c cos(k pi / (n + 1))|, k = 1..n, sorted descending."""
    k = np.arange(1, n + 1)
    s = np.abs(a + 2.0 * c * np.cos(k * np.pi / (n + 1)))
    return np.sort(s)[::-1]


def _haar_orthogonal(n: int, rng: np.random.Generator) -> np.ndarray:
    z = rng.standard_normal((n, n))
    q, r = np.linalg.qr(z)
    return q * np.sign(np.diag(r))


def prescribed_sigma_dense(n: int, profile: str, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """Dense n x n matrix A = U diag(sigma) V^T with Haar-random orthogonal U, V
    and prescribed singular values (the paper's accuracy-experiment input,
    Section V-A).  ``profile``: "arithmetic" (uniform spacing in (0, 1]),
    "logarithmic" (1 .. 1e-8, geometric) or "quartercircle" (quantiles of the
    quarter-circle law on [0, 1]).  Returns (A as a C-ordered array, sigma
    sorted descending)."""
    rng = _rng(seed)
    if profile == "arithmetic":
        sigma = np.arange(n, 0, -1) / n
    elif profile == "logarithmic":
        sigma = np.logspace(0.0, -8.0, n)
    elif profile == "quartercircle":
        # inverse CDF of the quarter circle density (4/pi) sqrt(1 - x^2) on [0, 1]
        p = (np.arange(n) + 0.5) / n
        xs = np.linspace(0.0, 1.0, 20001)
        cdf = (2.0 / np.pi) * (xs * np.sqrt(1.0 - xs * xs) + np.arcsin(xs))
        sigma = np.sort(np.interp(p, cdf, xs))[::-1]
    else:
        raise ValueError(profile)
    u = _haar_orthogonal(n, rng)
    v = _haar_orthogonal(n, rng)
    return (u * sigma) @ v.T, sigma


def prescribed_sigma_band(n: int, b: int, profile: str, seed: int,
                          ldab: int | None = None) -> tuple[np.ndarray, np.ndarray]:
    """Band matrix with prescribed singular values (accuracy experiment input).

    Following the paper's accuracy methodology: draw Haar-random orthogonal
    U, V, form A = U diag(sigma) V^T, and reduce A to upper-banded form with
    bandwidth b by two-sided orthogonal block transformations in FP64
    (numpy QR of b-wide panels: QR of a column panel from the left, then QR
    of the transposed row panel from the right).  Orthogonal transformations
    keep the singular values, so the band has exactly the prescribed
    sigma up to FP64 rounding.

    ``profile``: "arithmetic" (uniform spacing in (0, 1]), "logarithmic"
    (1 .. 1e-8, geometric), or "quartercircle" (quantiles of the quarter-circle
    law on [0, 1]).  Returns (ab of shape (n, ldab), sigma sorted descending).
    """
    a, sigma = prescribed_sigma_dense(n, profile, seed)
    # dense -> band: for each panel k, annihilate below the diagonal block
    # (left QR) and beyond the band (right QR of the transposed row block).
    for k in range(0, n, b):
        # left: rows k.. of columns k..k+b-1 -> upper trapezoidal
        q, _ = np.linalg.qr(a[k:, k : k + b], mode="complete")
        a[k:, k:] = q.T @ a[k:, k:]
        a[k + 1 :, k] = 0.0
        for t in range(1, min(b, n - k)):
            a[k + t + 1 :, k + t] = 0.0
        # right: columns k+b.. of rows k..k+b-1 -> lower trapezoidal
        if k + b < n:
            q, _ = np.linalg.qr(a[k : k + b, k + b :].T, mode="complete")
            a[:, k + b :] = a[:, k + b :] @ q
            for t in range(min(b, n - k)):
                a[k + t, k + t + b + 1 :] = 0.0
    return band_from_dense(np.triu(a), b, ldab), np.sort(sigma)[::-1]


def batch_problems(count: int, seed: int, n_lo: int = 256, n_hi: int = 4096,
                   bands=(8, 16, 32, 64)) -> list[tuple[int, int, int]]:
    """(n, b, seed) triples for the batched workload: n ~ U[n_lo, n_hi],
    b uniform over ``bands``; each problem gets its own derived seed."""
    rng = _rng(seed)
    ns = rng.integers(n_lo, n_hi + 1, size=count)
    bs = rng.choice(np.asarray(bands), size=count)
    seeds = rng.integers(0, 2**31 - 1, size=count)
    return [(int(n), int(b), int(s)) for n, b, s in zip(ns, bs, seeds)]


def tuner_grid(n_points: int = 11, n_lo: int = 1024, n_hi: int = 65536,
               bands=(16, 32, 64, 128, 256, 512)) -> list[tuple[int, int]]:
    """(n, b) pairs of the tuner's timing grid: n log-spaced over
    [n_lo, n_hi] (rounded to a multiple of 64) times the bandwidth list."""
    ns = np.unique((np.round(np.geomspace(n_lo, n_hi, n_points) / 64) * 64).astype(int))
    return [(int(n), int(b)) for n in ns for b in bands if b < n]

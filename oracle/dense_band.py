"""ORACLE -- test infrastructure only.

Stage 1 of the SVD the paper builds on (arXiv 2510.12705, Section II: the
dense matrix is first reduced to band form; Section V-A: the accuracy
experiments reduce prescribed-singular-value matrices to band form before the
band -> bidiagonal stage): a dense n x n matrix A is reduced to an upper-banded
B = Q^T A P with bandwidth b by Householder reflectors, one b-wide panel at a
time:

  for each panel k = 0, b, 2b, ...:
    column panel: a Householder QR of columns k .. k+w-1 (rows k .. n-1), each
      reflector applied from the left to every column to its right;
    row panel: a Householder LQ of rows k .. k+w-1 beyond the diagonal block
      (columns k+w .. n-1), each reflector applied from the right to every
      row below it.

Plain, unblocked FP64 numpy, in the order above; the reflectors follow the
LAPACK larfg convention (beta = -sign(alpha) ||x||, sign(0) = +1, tau = 0 when
the tail is zero), as the band -> bidiagonal oracle does.  Only ``tests/`` may
import this module; the product library shares no code with it.

Parity status:
  dense_to_band   pinned (tests/test_oracle_dense_band.py): singular values
                  equal numpy's SVD of A; exact zeros outside the band;
                  Frobenius norm preserved; an already banded input comes back
                  unchanged; b >= n-1 gives the R of LAPACK's QR; the returned
                  Q and P are orthogonal with Q^T A P = B; planted mistakes
                  fail these pins.
"""
from __future__ import annotations

import numpy as np


def larfg(x: np.ndarray):
    """Householder vector of x with the larfg contract: returns (tau, v, beta)
    with v[0] = 1 and (I - tau v v^T) x = (beta, 0, ..., 0)."""
    alpha = float(x[0])
    xi = float(np.linalg.norm(x[1:])) if x.size > 1 else 0.0
    if xi == 0.0:
        v = np.zeros_like(x)
        v[0] = 1.0
        return 0.0, v, alpha
    beta = -np.copysign(np.hypot(alpha, xi), alpha if alpha != 0.0 else 1.0)
    tau = (beta - alpha) / beta
    v = x / (alpha - beta)
    v[0] = 1.0
    return tau, v, beta


def dense_to_band(a: np.ndarray, b: int, with_qp: bool = False):
    """Upper band form of the dense matrix ``a`` (n x n) with bandwidth b >= 1.
    Returns B (dense n x n, exact zeros outside the band), and with
    ``with_qp`` also the accumulated orthogonal Q and P with Q^T A P = B."""
    a = np.array(a, dtype=np.float64, copy=True)
    n = a.shape[0]
    if b < 1:
        raise ValueError("bandwidth must be at least 1")
    q = np.eye(n) if with_qp else None
    p = np.eye(n) if with_qp else None
    for k in range(0, n, b):
        w = min(b, n - k)
        # column panel: QR from the left
        for j in range(w):
            c = k + j
            tau, v, beta = larfg(a[c:, c].copy())
            a[c:, c] = 0.0
            a[c, c] = beta
            if tau != 0.0:
                a[c:, c + 1:] -= tau * np.outer(v, v @ a[c:, c + 1:])
                if with_qp:
                    q[:, c:] -= tau * np.outer(q[:, c:] @ v, v)
        # row panel: LQ from the right, beyond the diagonal block
        for i in range(w):
            r = k + i
            c0 = k + w + i
            if c0 >= n:
                break
            tau, u, beta = larfg(a[r, c0:].copy())
            a[r, c0:] = 0.0
            a[r, c0] = beta
            if tau != 0.0:
                a[r + 1:, c0:] -= tau * np.outer(a[r + 1:, c0:] @ u, u)
                if with_qp:
                    p[:, c0:] -= tau * np.outer(p[:, c0:] @ u, u)
    if with_qp:
        return a, q, p
    return a

"""ORACLE -- test infrastructure only.

A plain, slow, obviously-correct CPU reference for the reduction of an
upper-banded matrix to bidiagonal form by Householder bulge chasing
(arXiv 2510.12705, Section III, Algorithms 1 and 2), plus the host-side
checks used to pin it: singular values of a bidiagonal by Sturm bisection,
a one-sided Jacobi SVD for brute force on small matrices, and spectral power
sums that hold at any size.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never loads it and
shares no code with it.  The reduction itself is plain C (``bulge_oracle.c``),
compiled here with gcc, FP64, no FMA contraction, single-threaded.
``band_to_bidiag_parallel`` runs the same row-bulges in the paper's cycle
schedule on all host cores (OpenMP, a separate library built with
``-fopenmp``); it is a CPU baseline, pinned bitwise to ``band_to_bidiag``.

Parity status of each function:
  band_to_bidiag      pinned: closed-form Toeplitz singular values, d[0] and
                      |e[0]| identities, b <= 1 special cases, Frobenius and
                      power-sum invariants, exact zeros off the bidiagonal,
                      Jacobi / LAPACK SVD brute force, prescribed-sigma inputs.
  bidiag_sigma        pinned: against numpy SVD of the dense bidiagonal and
                      against closed-form bidiagonal spectra.
  bidiag_count_below  pinned: against exact rational Sturm counts.
  jacobi_sigma        pinned: against numpy SVD and diagonal matrices.
  band_power_sums     pinned: against dense numpy on small matrices.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bulge_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_bulge_oracle.so")
_OMP_PATH = os.path.join(_HERE, "_bulge_oracle_omp.so")
_lock = threading.Lock()
_lib = None
_omp_lib = None


class _Counts(ctypes.Structure):
    _fields_ = [
        ("flops", ctypes.c_double),
        ("elements", ctypes.c_double),
        ("steps", ctypes.c_longlong),
        ("stages", ctypes.c_longlong),
        ("fill_violations", ctypes.c_longlong),
        ("out_of_band", ctypes.c_longlong),
    ]


def _compile(out: str, extra: list[str], force: bool) -> str:
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        tmp = out + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", *extra,
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile the C oracle into ``oracle/_bulge_oracle.so`` (gcc, -O2,
    no FMA contraction so results do not depend on the host's FMA use)."""
    return _compile(_LIB_PATH, [], force)


def build_parallel(force: bool = False) -> str:
    """Compile the same source with ``-fopenmp`` into
    ``oracle/_bulge_oracle_omp.so`` (adds ``oracle_band_to_bidiag_omp``)."""
    return _compile(_OMP_PATH, ["-fopenmp"], force)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            dp = ctypes.POINTER(ctypes.c_double)
            lib.oracle_band_to_bidiag.argtypes = [
                ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, dp, dp,
                ctypes.POINTER(_Counts), ctypes.c_int, ctypes.c_int, ctypes.c_longlong,
                dp, ctypes.c_int]
            lib.oracle_band_to_bidiag.restype = ctypes.c_int
            lib.oracle_bidiag_sigma.argtypes = [ctypes.c_int, dp, dp, dp]
            lib.oracle_bidiag_sigma.restype = ctypes.c_int
            lib.oracle_gk_count.argtypes = [ctypes.c_int, dp, dp, ctypes.c_double, ctypes.c_double]
            lib.oracle_gk_count.restype = ctypes.c_longlong
            lib.oracle_jacobi_sigma.argtypes = [ctypes.c_int, dp, dp]
            lib.oracle_jacobi_sigma.restype = ctypes.c_int
            _lib = lib
    return _lib


def _load_parallel():
    global _omp_lib
    with _lock:
        if _omp_lib is None:
            build_parallel()
            lib = ctypes.CDLL(_OMP_PATH)
            dp = ctypes.POINTER(ctypes.c_double)
            lib.oracle_band_to_bidiag_omp.argtypes = [
                ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, dp, dp,
                ctypes.POINTER(_Counts), ctypes.c_longlong, ctypes.POINTER(ctypes.c_int)]
            lib.oracle_band_to_bidiag_omp.restype = ctypes.c_int
            _omp_lib = lib
    return _omp_lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def band_to_bidiag(ab: np.ndarray, b: int, tw: int, *, order: int = 0,
                   max_stages: int = -1, max_steps: int = -1,
                   return_work: bool = False, check_fill: bool = False):
    """Reduce the band ``ab`` (shape (n, ldab), LAPACK 'U' storage, see
    ``bandgen``) to bidiagonal form.  Returns (d, e, counts) or, with
    ``return_work``, (d, e, counts, work) where work has shape (n, ld),
    ld = b' + 2 tw + 1 (b' = min(b, n-1)), element (i, j) at
    work[j, i - j + b' + tw].

    ``order`` 0 runs the sweeps one after another; L >= 1 runs the paper's
    cycle schedule with lag L (Section III-A).  ``max_steps`` >= 0 stops after
    that many row-bulges (a bounded timing sample; the output is then partial).
    """
    lib = _load()
    ab = np.ascontiguousarray(ab, dtype=np.float64)
    n, ldab = ab.shape
    if n < 1:
        raise ValueError("n must be >= 1")
    d = np.zeros(n)
    e = np.zeros(max(n - 1, 1))
    cnt = _Counts()
    bcl = min(b, n - 1)
    ld = bcl + 2 * tw + 1
    work = np.zeros((n, ld)) if return_work else None
    rc = lib.oracle_band_to_bidiag(n, b, tw, _ptr(ab), ldab, _ptr(d), _ptr(e),
                                   ctypes.byref(cnt), order, max_stages, max_steps,
                                   _ptr(work) if work is not None else None,
                                   1 if check_fill else 0)
    if rc != 0:
        raise ValueError(f"oracle_band_to_bidiag failed: {rc}")
    counts = {k: getattr(cnt, k) for k, _ in _Counts._fields_}
    e = e[: n - 1]
    if return_work:
        return d, e, counts, work
    return d, e, counts


def band_to_bidiag_parallel(ab: np.ndarray, b: int, tw: int, *, max_steps: int = -1):
    """The reduction of ``band_to_bidiag`` in the cycle schedule of Section
    III-A (lag 2, lag 3 on a stage that ends at bandwidth 1) with the
    row-bulges of each cycle spread over OpenMP threads: the same d and e,
    bit for bit.  The thread count follows ``OMP_NUM_THREADS`` (default: all
    cores).  ``max_steps`` >= 0 stops after the cycle in which that many
    row-bulges were done (a bounded timing sample).  Returns
    (d, e, counts, threads)."""
    lib = _load_parallel()
    ab = np.ascontiguousarray(ab, dtype=np.float64)
    n, ldab = ab.shape
    if n < 1:
        raise ValueError("n must be >= 1")
    d = np.zeros(n)
    e = np.zeros(max(n - 1, 1))
    cnt = _Counts()
    thr = ctypes.c_int(0)
    rc = lib.oracle_band_to_bidiag_omp(n, b, tw, _ptr(ab), ldab, _ptr(d), _ptr(e),
                                       ctypes.byref(cnt), max_steps, ctypes.byref(thr))
    if rc != 0:
        raise ValueError(f"oracle_band_to_bidiag_omp failed: {rc}")
    counts = {k: getattr(cnt, k) for k, _ in _Counts._fields_}
    return d, e[: n - 1], counts, thr.value


def bidiag_sigma(d: np.ndarray, e: np.ndarray, method: str = "auto") -> np.ndarray:
    """Singular values (descending) of the upper bidiagonal with diagonal d
    and superdiagonal e.

    "bisect": our own Sturm-count bisection on the 2n x 2n Golub-Kahan
    tridiagonal (zero diagonal, off-diagonal d0, e0, d1, ...), whose
    eigenvalues are +-sigma.  "lapack": the same Golub-Kahan matrix through
    scipy's tridiagonal eigensolver (LAPACK sterf, root-free QR), used as a
    library step for large n.  "auto" picks bisection up to n = 2048.
    """
    d = np.ascontiguousarray(d, dtype=np.float64)
    e = np.ascontiguousarray(e, dtype=np.float64)
    n = d.shape[0]
    if method == "auto":
        method = "bisect" if n <= 2048 else "lapack"
    if method == "bisect":
        lib = _load()
        out = np.zeros(n)
        ee = e if n > 1 else np.zeros(1)
        rc = lib.oracle_bidiag_sigma(n, _ptr(d), _ptr(ee), _ptr(out))
        if rc != 0:
            raise ValueError("oracle_bidiag_sigma failed")
        return out
    if method == "lapack":
        from scipy.linalg import eigvalsh_tridiagonal
        if n == 1:
            return np.abs(d).copy()
        off = np.zeros(2 * n - 1)
        off[0::2] = d
        off[1::2] = e
        w = eigvalsh_tridiagonal(np.zeros(2 * n), off, lapack_driver="sterf")
        return np.sort(np.abs(w[n:]))[::-1]
    raise ValueError(method)


def bidiag_count_below(d: np.ndarray, e: np.ndarray, x: float, pivmin: float) -> int:
    """#{sigma < x} (x > 0) of the bidiagonal (d, e): the oracle's Sturm count
    in pivot form on the Golub-Kahan matrix (tiny pivots replaced by -pivmin)."""
    lib = _load()
    d = np.ascontiguousarray(d, dtype=np.float64)
    e = np.ascontiguousarray(e if len(e) else np.zeros(1), dtype=np.float64)
    return int(lib.oracle_gk_count(len(d), _ptr(d), _ptr(e), float(x), float(pivmin)))


def jacobi_sigma(a: np.ndarray) -> np.ndarray:
    """Singular values (descending) of a dense square matrix by one-sided
    Jacobi rotations (brute force, small n)."""
    lib = _load()
    a = np.asarray(a, dtype=np.float64)
    n = a.shape[0]
    colmajor = np.array(a.T, dtype=np.float64, order="C")   # column p contiguous
    out = np.zeros(n)
    if lib.oracle_jacobi_sigma(n, _ptr(colmajor), _ptr(out)) != 0:
        raise ValueError("oracle_jacobi_sigma failed")
    return out


def band_gram(ab: np.ndarray, b: int) -> np.ndarray:
    """C = A^T A for the banded A, returned as (n, b+1) with
    C[j, k] = (A^T A)[j, j+k] (symmetric, bandwidth b).  O(n b^2)."""
    ab = np.asarray(ab, dtype=np.float64)
    n = ab.shape[0]
    c = np.zeros((n, b + 1))
    # (A^T A)[j, j+k] = sum_i A[i, j] A[i, j+k]; A[i, j] = ab[j, b + i - j]
    for k in range(b + 1):
        jj = np.arange(0, n - k)
        for t in range(b - k + 1):      # i = j - t, needs j - i = t <= b and j + k - i <= b
            i = jj - t
            ok = i >= 0
            c[jj[ok], k] += ab[jj[ok], b - t] * ab[jj[ok] + k, b - t - k]
    return c


def band_power_sums(ab: np.ndarray, b: int) -> tuple[float, float]:
    """(sum sigma^2, sum sigma^4) of the banded A: ||A||_F^2 and ||A^T A||_F^2."""
    ab = np.asarray(ab, dtype=np.float64)
    p1 = float(np.sum(ab[:, : b + 1] ** 2))
    c = band_gram(ab, b)
    p2 = float(np.sum(c[:, 0] ** 2) + 2.0 * np.sum(c[:, 1:] ** 2))
    return p1, p2


def bidiag_power_sums(d: np.ndarray, e: np.ndarray) -> tuple[float, float]:
    """(sum sigma^2, sum sigma^4) of the bidiagonal B(d, e), via B^T B."""
    d = np.asarray(d, dtype=np.float64)
    e = np.asarray(e, dtype=np.float64)
    p1 = float(np.sum(d * d) + np.sum(e * e))
    diag = d * d
    diag[1:] += e * e
    off = d[:-1] * e
    p2 = float(np.sum(diag * diag) + 2.0 * np.sum(off * off))
    return p1, p2

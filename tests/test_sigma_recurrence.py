"""Host model of the GPU singular-value count (division-free three-term Sturm
recurrence on the Golub-Kahan matrix, restarted at splits, power-of-two
rescaling, bisection started from a shared grid of counts), replayed in Python with the kernel's rules and compared with the
oracle's bisection on the inputs that stress it: exact zeros (splits), tiny
and huge entries, the all-ones closed form."""
import math

import numpy as np
import pytest

import oracle

EPS = 2.220446049250313e-16
DBL_MIN = 2.2250738585072014e-308


def _count(d, e, x, pivmin, sc):
    n = len(d)
    pm1, p = 1.0, -x
    if abs(p) < pivmin:
        p = -pivmin
    neg = 1

    def step(pm1, p, f2, neg):
        if f2 == 0.0:                      # split: q = -x < 0, fresh sequence
            return 1.0, -x, neg + 1
        pn = -x * p - f2 * pm1
        if pn == 0.0:
            pn = -pivmin * p if p != 0.0 else -pivmin
        neg += math.copysign(1.0, pn) != math.copysign(1.0, p)
        return p, pn, neg

    for k in range(n):
        pm1, p, neg = step(pm1, p, (d[k] * sc) ** 2, neg)
        if k + 1 < n:
            pm1, p, neg = step(pm1, p, (e[k] * sc) ** 2, neg)
        if k & 1:
            m = max(abs(pm1), abs(p))
            ex = max(math.frexp(m)[1] - 1, -1023) if m > 0 else -1023
            if ex > 400 or ex < -400:
                s = math.ldexp(1.0, -ex)
                pm1, p = pm1 * s, p * s
    return neg - n


def kernel_sigma(d, e):
    """Descending singular values by the kernel's bisection and count."""
    d = np.asarray(d, np.float64)
    e = np.asarray(e, np.float64)
    n = len(d)
    f = np.empty(2 * n - 1)
    f[0::2] = d
    f[1::2] = e
    fm = float(np.max(np.abs(f)))
    k = min(max(1 - math.frexp(fm)[1], -1022), 1023) if fm > 0 else 0
    sc = math.ldexp(1.0, k)
    fp = np.concatenate([[0.0], f[:-1]])
    ub = 2 * float(np.max(0.5 * np.abs(f) + 0.5 * np.abs(fp))) * sc * (1 + 4 * EPS) + DBL_MIN
    pivmin = max((fm * sc) ** 2 * DBL_MIN, DBL_MIN)
    # shared first cut: counts at ub k / G, G a power of two with 4 G <= n
    # (at most 2^14); each value starts from the cell that brackets it
    G = 1
    while G < 16384 and 4 * G <= n:
        G *= 2
    cnt = [0] + [_count(d, e, ub * (k / G), pivmin, sc) for k in range(1, G)] + [n]
    out = np.empty(n)
    for j in range(n):
        klo, khi = 0, G
        while khi - klo > 1:
            km = (klo + khi) // 2
            if cnt[km] <= j:
                klo = km
            else:
                khi = km
        lo = 0.0 if klo == 0 else ub * (klo / G)
        hi = ub if khi == G else ub * (khi / G)
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            if mid <= lo or mid >= hi:
                break
            if hi - lo <= max(2 * EPS * max(abs(lo), abs(hi)), 0.5 * EPS * ub) + 2 * pivmin:
                break
            if _count(d, e, mid, pivmin, sc) > j:
                hi = mid
            else:
                lo = mid
        out[n - 1 - j] = 0.5 * (lo + hi) / sc
    return out


def _cases():
    rng = np.random.default_rng(5)
    out = []
    for n in (1, 2, 5, 17, 40):
        d, e = rng.standard_normal(n), rng.standard_normal(n - 1)
        out.append((f"random{n}", d, e))
        if n > 3:
            d2, e2 = d.copy(), e.copy()
            d2[n // 2] = 0.0
            e2[n // 3] = 0.0
            out.append((f"zeros{n}", d2, e2))
            d3, e3 = d.copy(), e.copy()
            d3[::3] *= 1e-200
            e3[1::4] = 0.0
            out.append((f"tiny{n}", d3, e3))
    return out


@pytest.mark.parametrize("name,d,e", _cases(), ids=[c[0] for c in _cases()])
def test_kernel_count_matches_oracle(name, d, e):
    ref = oracle.bidiag_sigma(d, e, method="bisect")
    assert np.max(np.abs(kernel_sigma(d, e) - ref)) <= 1e-15 * ref[0]


@pytest.mark.parametrize("scale", [1e250, 1e-250])
def test_extreme_scales(scale):
    d = np.array([1.0, 0.0, 3.0, 2.0, 1e-200, 5.0])
    e = np.array([0.0, 2.0, 0.0, 1e-150, 1.0])
    ref = oracle.bidiag_sigma(d, e, method="bisect")
    s = kernel_sigma(d * scale, e * scale)
    assert np.max(np.abs(s - ref * scale)) <= 1e-15 * ref[0] * scale


def test_closed_form_all_ones():
    n = 200
    k = np.arange(1, n + 1)
    assert np.max(np.abs(kernel_sigma(np.ones(n), np.ones(n - 1)) - 2 * np.cos(k * np.pi / (2 * n + 1)))) < 1e-14


def _exact_count(d, e, x):
    """#{sigma < x}: negative pivots of the shifted Golub-Kahan LDL^T in exact
    rational arithmetic, minus n (brute force, independent of rounding)."""
    from fractions import Fraction
    f = []
    for k in range(len(d)):
        f.append(Fraction(float(d[k])))
        if k + 1 < len(d):
            f.append(Fraction(float(e[k])))
    X = Fraction(x)
    q = -X
    neg = 1
    for fi in f:
        q = -X - fi * fi / q if q != 0 else -X
        neg += q < 0
    return neg - len(d)


@pytest.mark.parametrize("seed", range(12))
def test_count_on_runs_of_tiny_couplings(seed):
    # a run of entries 1e-100 .. 1e-150 of the largest (squares still normal)
    # and shifts over the whole range the bisection evaluates (down to about
    # 2^-55 ub): the kernel's count equals the oracle's and the exact one
    rng = np.random.default_rng(seed)
    n = 30
    d, e = rng.standard_normal(n), rng.standard_normal(n - 1)
    lo = int(rng.integers(2, n - 10))
    d[lo:lo + 8] *= 10.0 ** -rng.uniform(100, 150)
    e[lo:lo + 8] *= 10.0 ** -rng.uniform(100, 150)
    fm = max(np.max(np.abs(d)), np.max(np.abs(e)))
    sc = math.ldexp(1.0, min(max(1 - math.frexp(fm)[1], -1022), 1023))
    pivmin = max((fm * sc) ** 2 * DBL_MIN, DBL_MIN)
    for u in np.linspace(0.0, 16.5, 12):
        x = 10.0 ** -u * sc
        k = _count(d, e, x, pivmin, sc)
        assert k == oracle.bidiag_count_below(d * sc, e * sc, x, pivmin), (u, k)
        assert k == _exact_count(d * sc, e * sc, x), (u, k)


def test_oracle_count_is_exact():
    # the oracle's pivot-form count against the rational count, random inputs
    rng = np.random.default_rng(9)
    for _ in range(20):
        n = int(rng.integers(1, 25))
        d, e = rng.standard_normal(n), rng.standard_normal(max(n - 1, 0))
        for x in 10.0 ** -rng.uniform(-0.5, 12, 5):
            assert oracle.bidiag_count_below(d, e, x, DBL_MIN) == _exact_count(d, e, x)

"""Host replica of the fixed-point sum of squares that the GPU reflector
generation uses for FP32 data (bb_device.cuh, fast_reflector): each FP32
value is mantissa x 2^(exponent - 150), its square a 48-bit integer; the
squares are aligned to the largest exponent with 9 bits of headroom, summed in
64-bit integers and converted to FP64 once.  Checked against the exact
rational sum: the relative error must stay below 2^-51 for any FP32 vector
of up to 33 entries, subnormals and the extremes of the range included."""
from fractions import Fraction

import numpy as np
import pytest


def fixed_point_sumsq(x32):
    bits = np.asarray(x32, dtype=np.float32).view(np.uint32).astype(np.int64)
    e = (bits >> 23) & 0xFF
    mant = bits & 0x7FFFFF
    mant = np.where(e != 0, mant | 0x800000, mant)
    e = np.where(e != 0, e, 1)
    e = np.where(mant == 0, 0, e)
    E = int(e.max())
    acc = 0
    for ei, mi in zip(e.tolist(), mant.tolist()):
        if ei == 0:
            continue
        sh = 2 * (E - ei)
        if sh < 64:
            acc += ((mi * mi) << 9) >> sh
    assert acc < 2 ** 64
    p = 2 * E - 309
    return float(acc) * 2.0 ** (p // 2 if p >= 0 else -((-p) // 2)) * 2.0 ** (p - (p // 2 if p >= 0 else -((-p) // 2)))


def exact_sumsq(x32):
    return sum(Fraction(float(v)) ** 2 for v in np.asarray(x32, dtype=np.float32))


@pytest.mark.parametrize("seed", range(40))
def test_fixed_point_sum_of_squares(seed):
    rng = np.random.default_rng(seed)
    m = int(rng.integers(2, 34))
    kind = seed % 5
    if kind == 0:
        x = rng.standard_normal(m)
    elif kind == 1:                         # wide dynamic range
        x = rng.standard_normal(m) * 10.0 ** rng.uniform(-30, 30, m)
    elif kind == 2:                         # near the top of the FP32 range
        x = rng.uniform(-1, 1, m) * 3e38
    elif kind == 3:                         # subnormals and tiny normals
        x = rng.standard_normal(m) * 1e-41
        x[0] = 1.2e-38
    else:                                   # one large entry, the rest tiny
        x = rng.standard_normal(m) * 1e-20
        x[int(rng.integers(0, m))] = 7.0
    x32 = x.astype(np.float32)
    if not np.any(x32[1:] != 0):
        x32[1] = np.float32(1.0)
    got = fixed_point_sumsq(x32)
    ref = exact_sumsq(x32)
    rel = abs(Fraction(got) - ref) / ref
    assert rel <= Fraction(1, 2 ** 51), float(rel)


def test_fixed_point_exact_on_small_integers():
    x = np.arange(1, 34, dtype=np.float32)
    assert fixed_point_sumsq(x) == float(sum(i * i for i in range(1, 34)))

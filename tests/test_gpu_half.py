"""Half-precision storage forms (BB_F16, BB_BF16): the working band, the input
and d, e in 16 bits, panels and arithmetic in FP32, reflectors generated in
FP64.  Compared with the FP64 oracle run on the same rounded input.

Tolerance: the FP32 form's measured error is about 2 u_32 ||A||_2 (graded
n = 32768 study), i.e. a small multiple of the storage unit roundoff; every
element is rounded to the storage type after each row-bulge, so the half
forms are held to 8 u ||A||_2 with u = 2^-11 (FP16: 3.9e-3) and
u = 2^-8 (BF16: 3.1e-2)."""
import numpy as np
import pytest
import torch

import bandgen
import oracle

pytestmark = pytest.mark.gpu

U = {torch.float16: 2.0 ** -11, torch.bfloat16: 2.0 ** -8}


@pytest.fixture(scope="module")
def bb():
    import paper_2510_12705_gb300 as bb
    from paper_2510_12705_gb300 import build
    build.build()
    return bb


@pytest.mark.parametrize("dt", [torch.float16, torch.bfloat16])
@pytest.mark.parametrize("n,b,tw", [(512, 16, 0), (1000, 40, 0), (777, 9, 4), (300, 33, 16)])
def test_half_storage_sigma(bb, dt, n, b, tw):
    ab = bandgen.random_band(n, b, seed=n + b)
    band = torch.from_numpy(ab).to("cuda", dt)
    ab_r = band.double().cpu().numpy()                       # the rounded input
    d = torch.empty(n, device="cuda", dtype=dt)
    e = torch.empty(n - 1, device="cuda", dtype=dt)
    tun = bb.Tuning(tw=tw) if tw else None
    bb.band_to_bidiag_ex(band, b, d, e, tuning=tun)
    assert bb.bb_device_status(reset=True) == 0
    do, eo, _ = oracle.band_to_bidiag(ab_r, b, 16)
    ref = oracle.bidiag_sigma(do, eo)
    s = oracle.bidiag_sigma(d.double().cpu().numpy(), e.double().cpu().numpy())
    assert np.max(np.abs(s - ref)) <= 8 * U[dt] * ref[0]
    # d[0] is A[0, 0] untouched
    assert float(d[0]) == float(band[0, b])


@pytest.mark.parametrize("dt", [torch.float16, torch.bfloat16])
def test_half_storage_batched_and_repeatable(bb, dt):
    probs = [(200, 8, 1), (333, 17, 2), (64, 63, 3)]
    items = []
    for n, b, s in probs:
        band = torch.from_numpy(bandgen.random_band(n, b, seed=s)).to("cuda", dt)
        items.append((band, b, torch.empty(n, device="cuda", dtype=dt),
                      torch.empty(n - 1, device="cuda", dtype=dt)))
    plan = bb.BatchPlan(items)
    ws = torch.empty(plan.workspace_bytes, dtype=torch.uint8, device="cuda")
    plan.execute(ws)
    torch.cuda.synchronize()
    for band, b, d, e in items:
        d2, e2 = torch.empty_like(d), torch.empty_like(e)
        bb.band_to_bidiag(band, b, d2, e2)
        torch.cuda.synchronize()
        assert torch.equal(d, d2) and torch.equal(e, e2)
    assert bb.bb_device_status(reset=True) == 0


def test_half_storage_nonfinite_reported(bb):
    ab = bandgen.random_band(100, 8, seed=4)
    ab[50, 3] = 1e6            # beyond FP16's range: rounds to inf
    band = torch.from_numpy(ab).to("cuda", torch.float16)
    d = torch.empty(100, device="cuda", dtype=torch.float16)
    e = torch.empty(99, device="cuda", dtype=torch.float16)
    bb.band_to_bidiag(band, 8, d, e)
    assert bb.BB_ERR_NONFINITE in bb.status_bits(bb.bb_device_status(reset=True))

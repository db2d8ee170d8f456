"""Batched reduction of many band matrices of uneven n and b in one
persistent launch per stage (bb_batch_plan / bb_batch_execute), including
capture into a CUDA graph and replay."""
import numpy as np
import pytest

import bandgen
import oracle
from gpu_util import TOL_F32, TOL_F64

pytestmark = pytest.mark.gpu


def _make(problems, dtype):
    import torch
    out = []
    for (n, b, seed) in problems:
        ab = bandgen.random_band(n, b, seed=seed)
        band = torch.from_numpy(ab).to("cuda", dtype)
        d = torch.full((n,), float("nan"), device="cuda", dtype=dtype)
        e = torch.full((max(n - 1, 1),), float("nan"), device="cuda", dtype=dtype)
        out.append((band, b, d, e, ab))
    return out


def _single(band, b, dtype):
    import torch
    import paper_2510_12705_gb300 as bb
    n = band.shape[0]
    d = torch.empty(n, device="cuda", dtype=dtype)
    e = torch.empty(max(n - 1, 1), device="cuda", dtype=dtype)
    bb.band_to_bidiag(band, b, d, e)
    return d.cpu().numpy(), e[: n - 1].cpu().numpy()


@pytest.mark.parametrize("dtype_name", ["f64", "f32"])
def test_batch_matches_single_and_oracle(dtype_name):
    import torch
    import paper_2510_12705_gb300 as bb
    dtype = torch.float64 if dtype_name == "f64" else torch.float32
    tol = TOL_F64 if dtype_name == "f64" else TOL_F32
    probs = bandgen.batch_problems(24, seed=3, n_lo=40, n_hi=700, bands=(1, 8, 16, 32, 64)) + \
        [(1, 0, 5), (2, 1, 6), (3, 2, 7), (50, 80, 8)]          # tiny and b >= n
    items = _make(probs, dtype)
    plan = bb.BatchPlan([(band, b, d, e) for band, b, d, e, _ in items])
    ws = torch.empty(plan.workspace_bytes, dtype=torch.uint8, device="cuda")
    plan.execute(ws)
    torch.cuda.synchronize()
    assert bb.bb_device_status(reset=True) == 0
    for (band, b, d, e, ab) in items:
        n = band.shape[0]
        dg, eg = d.cpu().numpy(), e[: n - 1].cpu().numpy()
        ds, es = _single(band, b, dtype)
        # same kernels and reflector sequence: bitwise equal to the single call
        assert np.array_equal(dg, ds) and np.array_equal(eg, es), (n, b)
        d0, e0, _ = oracle.band_to_bidiag(ab, b, 16)
        s0 = oracle.bidiag_sigma(d0, e0)
        s = oracle.bidiag_sigma(dg.astype(np.float64), eg.astype(np.float64))
        assert np.max(np.abs(s - s0)) <= tol * max(s0[0], 1e-300), (n, b)


def test_batch_graph_capture_and_replay():
    import torch
    import paper_2510_12705_gb300 as bb
    dtype = torch.float32
    probs = bandgen.batch_problems(16, seed=9, n_lo=100, n_hi=900, bands=(8, 16, 32, 64))
    items = _make(probs, dtype)
    plan = bb.BatchPlan([(band, b, d, e) for band, b, d, e, _ in items])
    ws = torch.empty(plan.workspace_bytes, dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):          # warm-up outside the capture (module loading)
        plan.execute(ws, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        plan.execute(ws)
    for rep in range(2):
        # new inputs in the captured buffers, then replay
        refs = []
        for j, (band, b, d, e, _) in enumerate(items):
            n = band.shape[0]
            ab = bandgen.random_band(n, b, seed=1000 * rep + j)
            band.copy_(torch.from_numpy(ab).to(dtype))
            refs.append(ab)
        g.replay()
        torch.cuda.synchronize()
        assert bb.bb_device_status(reset=True) == 0
        for (band, b, d, e, _), ab in zip(items, refs):
            n = band.shape[0]
            ds, es = _single(band, b, dtype)
            assert np.array_equal(d.cpu().numpy(), ds)
            assert np.array_equal(e[: n - 1].cpu().numpy(), es)


def test_batch_plan_rejects_bad_problem():
    import torch
    import paper_2510_12705_gb300 as bb
    band = torch.zeros((10, 3), device="cuda", dtype=torch.float64)
    d = torch.empty(10, device="cuda", dtype=torch.float64)
    e = torch.empty(9, device="cuda", dtype=torch.float64)
    with pytest.raises(bb.BBError):
        bb.BatchPlan([(band, 5, d, e)])        # ldab = 3 < b + 1


def test_shard_run_local_matches_single_calls():
    """One rank's share of a partitioned batch (shard.run_local) gives the same
    bits as reducing each of its problems alone."""
    import torch

    import paper_2510_12705_gb300 as bb
    from paper_2510_12705_gb300 import shard
    specs = [(300, 8, 1), (513, 16, 2), (128, 32, 3), (777, 5, 4), (64, 63, 5), (1000, 12, 6)]
    problems = [(bandgen.random_band(n, b, seed=s), b) for n, b, s in specs]
    parts = shard.partition([(ab.shape[0], b) for ab, b in problems], 2)
    for rank in range(2):
        got = shard.run_local(problems, parts[rank], dtype="f64")
        assert sorted(got) == parts[rank]
        for i in parts[rank]:
            ab, b = problems[i]
            band = torch.from_numpy(ab).cuda()
            n = ab.shape[0]
            d = torch.empty(n, device="cuda", dtype=torch.float64)
            e = torch.empty(n - 1, device="cuda", dtype=torch.float64)
            bb.band_to_bidiag(band, b, d, e)
            assert np.array_equal(got[i][0], d.cpu().numpy())
            assert np.array_equal(got[i][1], e.cpu().numpy())


def test_one_call_batched_equals_plan():
    """band_to_bidiag_batched (one call) gives the same bits as the plan API."""
    import torch
    import paper_2510_12705_gb300 as bb
    dtype = torch.float64
    probs = bandgen.batch_problems(12, seed=5, n_lo=50, n_hi=600, bands=(4, 16, 40, 64))
    a = _make(probs, dtype)
    b_ = _make(probs, dtype)
    plan = bb.BatchPlan([(band, b, d, e) for band, b, d, e, _ in a])
    ws = torch.empty(plan.workspace_bytes, dtype=torch.uint8, device="cuda")
    plan.execute(ws)
    bb.band_to_bidiag_batched([(band, b, d, e) for band, b, d, e, _ in b_])
    assert bb.bb_last_device_status() == 0
    for (_, _, d1, e1, _), (_, _, d2, e2, _) in zip(a, b_):
        n = d1.numel()
        assert torch.equal(d1, d2) and torch.equal(e1[: n - 1], e2[: n - 1])


def test_cfg4_sample_sigma_vs_oracle():
    """The 512-matrix batch of the batched workload (n ~ U[256, 4096],
    b in {8, 16, 32, 64}, FP32, seed 3), reduced in one plan: the four
    largest matrices and four others of the batch against the FP64 oracle's
    singular values at the FP32 tolerance."""
    import torch
    import paper_2510_12705_gb300 as bb
    probs = bandgen.batch_problems(512, seed=3)
    items = _make(probs, torch.float32)
    plan = bb.BatchPlan([(band, b, d, e) for band, b, d, e, _ in items])
    ws = torch.empty(plan.workspace_bytes, dtype=torch.uint8, device="cuda")
    plan.execute(ws)
    torch.cuda.synchronize()
    assert bb.bb_device_status(reset=True) == 0
    order = sorted(range(len(probs)), key=lambda i: -probs[i][0])
    sample = order[:4] + [order[len(order) // 4], order[len(order) // 2], order[-2], order[-1]]
    assert max(probs[i][0] for i in sample) > 3500
    for i in sample:
        band, b, d, e, ab = items[i]
        n = band.shape[0]
        d0, e0, _ = oracle.band_to_bidiag(ab, b, 32)
        s0 = oracle.bidiag_sigma(d0, e0)
        s = oracle.bidiag_sigma(d.cpu().numpy().astype(np.float64), e[: n - 1].cpu().numpy().astype(np.float64))
        assert np.max(np.abs(s - s0)) <= TOL_F32 * s0[0], (n, b)

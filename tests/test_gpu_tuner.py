"""GPU tests of the tuning layer: the MLP's forward, backward and Adam kernels
against the FP64 oracle (oracle/mlp.py), training on the GPU kernels, the
exhaustive autotuner, and the trained tuner's regret and gain on problems
outside its training grid."""
import json
import os

import numpy as np
import pytest
import torch

from oracle import mlp

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bb():
    import paper_2510_12705_gb300 as bb
    from paper_2510_12705_gb300 import build
    build.build()
    return bb


def _case(D, H, N, seed):
    rng = np.random.default_rng(seed)
    p = rng.standard_normal(mlp.param_count(D, H)) * 0.5
    X = rng.standard_normal((N, D))
    T = rng.standard_normal(N)
    return p.astype(np.float32), X.astype(np.float32), T.astype(np.float32)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


@pytest.mark.parametrize("D,H,N", [(8, 32, 1), (8, 32, 97), (5, 64, 300), (32, 128, 33)])
def test_mlp_forward_backward_match_oracle(bb, D, H, N):
    p, X, T = _case(D, H, N, seed=D * 1000 + N)
    P, Xd, Td = _dev(p), _dev(X), _dev(T)
    Y = torch.empty(N, device="cuda")
    H1 = torch.empty(N, H, device="cuda")
    H2 = torch.empty(N, H, device="cuda")
    G = torch.empty_like(P)
    S = torch.empty(bb.bb_mlp_backward_scratch(H, N), device="cuda")
    bb.bb_mlp_forward(D, H, P, Xd, Y, H1, H2)
    bb.bb_mlp_backward(D, H, P, Xd, H1, H2, Y, Td, G, S)
    torch.cuda.synchronize()
    # the oracle runs in FP64 on the same FP32 inputs
    Yr, H1r, H2r = mlp.forward(p.astype(np.float64), X.astype(np.float64), D, H)
    Gr = mlp.backward(p.astype(np.float64), X.astype(np.float64), T.astype(np.float64), D, H)
    # FP32 sums of at most max(D, H, N) terms: a few hundred ulps of the scale
    tol = 2e-5 * max(D, H, N) ** 0.5
    scale = max(1.0, float(np.abs(Yr).max()))
    np.testing.assert_allclose(Y.cpu().numpy(), Yr, rtol=0, atol=tol * scale)
    np.testing.assert_allclose(H1.cpu().numpy(), H1r, rtol=0, atol=tol * max(1.0, np.abs(H1r).max()))
    np.testing.assert_allclose(H2.cpu().numpy(), H2r, rtol=0, atol=tol * max(1.0, np.abs(H2r).max()))
    g = G.cpu().numpy()
    gs = max(1e-3, float(np.abs(Gr).max()))
    assert np.max(np.abs(g - Gr)) <= 5 * tol * gs, np.max(np.abs(g - Gr)) / gs


def test_adam_kernel_matches_oracle(bb):
    rng = np.random.default_rng(11)
    n = 1000
    p = rng.standard_normal(n)
    m = np.zeros(n)
    v = np.zeros(n)
    mabs = np.zeros(n)          # the same moment over |g|: the scale of the rounding
    P, M, V = _dev(p), _dev(m), _dev(v)
    for step in range(1, 6):
        g = rng.standard_normal(n) * 10.0 ** rng.uniform(-4, 1, n)
        bb.bb_mlp_adam(P, _dev(g), M, V, step, 1e-2)
        g = g.astype(np.float32).astype(np.float64)
        p, m, v = mlp.adam(p, g, m, v, step, 1e-2)
        mabs = 0.9 * mabs + 0.1 * np.abs(g)
    torch.cuda.synchronize()
    np.testing.assert_allclose(P.cpu().numpy(), p, rtol=0, atol=1e-5)
    # a few FP32 roundings per step of terms no larger than mabs
    assert np.all(np.abs(M.cpu().numpy() - m) <= 16 * 2.0 ** -24 * 5 * mabs)


def test_gpu_training_follows_oracle_training(bb):
    """Thirty full-batch Adam steps with the GPU kernels track the same steps
    taken by the FP64 oracle, and the loss falls."""
    D, H, N = 8, 32, 200
    p, X, _ = _case(D, H, N, seed=4)
    T = (np.sin(X[:, 0]) + X[:, 1] * X[:, 2]).astype(np.float32)
    P, Xd, Td = _dev(p), _dev(X), _dev(T)
    G, M, V = torch.zeros_like(P), torch.zeros_like(P), torch.zeros_like(P)
    Y = torch.empty(N, device="cuda")
    H1 = torch.empty(N, H, device="cuda")
    H2 = torch.empty(N, H, device="cuda")
    S = torch.empty(bb.bb_mlp_backward_scratch(H, N), device="cuda")
    pr = p.astype(np.float64)
    mr = np.zeros_like(pr)
    vr = np.zeros_like(pr)
    Xr, Tr = X.astype(np.float64), T.astype(np.float64)
    l0 = mlp.loss(pr, Xr, Tr, D, H)
    for step in range(1, 31):
        bb.bb_mlp_forward(D, H, P, Xd, Y, H1, H2)
        bb.bb_mlp_backward(D, H, P, Xd, H1, H2, Y, Td, G, S)
        bb.bb_mlp_adam(P, G, M, V, step, 3e-3)
        pr, mr, vr = mlp.adam(pr, mlp.backward(pr, Xr, Tr, D, H), mr, vr, step, 3e-3)
    torch.cuda.synchronize()
    # Adam's normalised steps amplify rounding only where a gradient is at the
    # rounding level; those parameters can drift by at most 2 lr per step
    diff = np.abs(P.cpu().numpy() - pr)
    assert np.quantile(diff, 0.99) <= 1e-3 and diff.max() <= 2 * 3e-3 * 30
    l_gpu = mlp.loss(P.cpu().numpy().astype(np.float64), Xr, Tr, D, H)
    l_ref = mlp.loss(pr, Xr, Tr, D, H)
    assert l_gpu < 0.8 * l0 and abs(l_gpu - l_ref) <= 1e-3 * l0


def test_autotune_times_every_candidate(bb):
    import bandgen
    n, b = 1024, 32
    band = torch.from_numpy(bandgen.random_band(n, b, seed=1)).cuda().float()
    d = torch.empty(n, device="cuda")
    e = torch.empty(n - 1, device="cuda")
    cands = [bb.Tuning(tw=32), bb.Tuning(tw=16, tpb=256), bb.Tuning(tw=8, sweeps_in_flight=152)]
    times, best = bb.bb_autotune(band, b, d, e, cands, reps=3)
    assert len(times) == 3 and all(t > 0 for t in times)
    assert best == int(np.argmin(times))
    assert bb.bb_device_status(reset=True) == 0
    # the outputs are those of the last candidate's run
    d2, e2 = torch.empty_like(d), torch.empty_like(e)
    bb.band_to_bidiag_ex(band, b, d2, e2, tuning=cands[-1])
    torch.cuda.synchronize()
    assert torch.equal(d, d2) and torch.equal(e, e2)


def test_autotune_rejects_bad_arguments(bb):
    import bandgen
    band = torch.from_numpy(bandgen.random_band(64, 4, seed=1)).cuda()
    d = torch.empty(64, device="cuda", dtype=torch.float64)
    e = torch.empty(63, device="cuda", dtype=torch.float64)
    with pytest.raises(bb.BBError):
        bb.bb_autotune(band, 4, d, e, [], reps=1)
    with pytest.raises(bb.BBError):
        bb.bb_autotune(band, 4, d, e, [bb.Tuning(tw=64)], reps=1)


MODEL = os.path.join(ROOT, "paper_2510_12705_gb300", "tuner_model.json")


@pytest.mark.skipif(not os.path.exists(MODEL), reason="no trained tuner model committed")
@pytest.mark.parametrize("n,b,dtype", [(3072, 96, "f32"), (6144, 48, "f64"), (65536, 256, "f32")])
def test_trained_tuner_regret_and_gain(bb, n, b, dtype):
    """On problems outside the training grid (n and b not powers of two, and
    the held-out n = 65536, b = 256, FP32, which lies beyond the grid's
    largest n and n*b), the MLP's pick is within 10% of the exhaustive
    search's best time, needs no timed runs where the search needs one per
    candidate, and is no slower than the library's fixed default tuning (the
    method without the tuner)."""
    from paper_2510_12705_gb300 import tuner
    tun = tuner.MlpTuner.load(MODEL)
    r = tuner.evaluate(tun, n, b, dtype, reps=1 if n >= 65536 else 3)
    print(json.dumps({k: v for k, v in r.items() if k != "all_ms"}))
    assert r["mlp_regret"] <= 0.10, r
    assert r["mlp_ms"] <= 1.05 * r["default_ms"], r
    assert r["mlp_ms"] < r["mean_candidate_ms"], r


@pytest.mark.skipif(not os.path.exists(MODEL), reason="no trained tuner model committed")
def test_trained_tuner_beats_the_default_where_the_default_is_not_best(bb):
    """What the network gains over the method without it: on an FP64 shape
    outside the training grid the library default (TW = 16, the paper's FP64
    tilewidth) is not the fastest candidate, and the MLP's pick is measurably
    faster than it."""
    from paper_2510_12705_gb300 import tuner
    tun = tuner.MlpTuner.load(MODEL)
    r = tuner.evaluate(tun, 6144, 48, "f64", reps=3)
    print(json.dumps({k: v for k, v in r.items() if k != "all_ms"}))
    assert r["exhaustive_ms"] < 0.97 * r["default_ms"], r
    assert r["mlp_ms"] < 0.97 * r["default_ms"], r

"""The C-ABI library builds, loads without a GPU, exports every symbol the
header declares, and its host-only parts (work model, argument checks) agree
with the oracle.  No compute call reaches the GPU here."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import bandgen
import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bb():
    from paper_2510_12705_gb300 import build
    build.build()
    import paper_2510_12705_gb300 as m
    m.lib()
    return m


def _declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(\w+)\s*\(", src, flags=re.M):
            name = m.group(1)
            if name not in ("if", "while", "for", "return", "sizeof", "defined"):
                names.append(name)
    return sorted(set(names))


def test_header_symbols_exported(bb):
    names = _declared_functions()
    assert "band_to_bidiag" in names and "bb_batch_execute" in names
    lib = ctypes.CDLL(bb.LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


@pytest.mark.parametrize("n,b,tw", [(512, 16, 16), (300, 40, 16), (257, 33, 8), (400, 64, 32),
                                    (100, 7, 3), (64, 63, 16), (30, 50, 4), (5, 1, 4), (1, 0, 16)])
def test_work_model_matches_oracle_counts(bb, n, b, tw):
    ab = bandgen.random_band(n, b, seed=n + b)
    _, _, cnt = oracle.band_to_bidiag(ab, b, tw)
    wm = bb.bb_schedule_counts(n, b, tw)
    assert wm.steps == cnt["steps"]
    assert wm.stages == cnt["stages"]
    assert wm.flops == pytest.approx(cnt["flops"], rel=1e-12, abs=0)
    assert wm.elements == pytest.approx(cnt["elements"], rel=1e-12, abs=0)


def test_work_model_large_is_fast_and_consistent(bb):
    # headline configuration: the per-sweep closed form must agree with a
    # direct per-step sum on a smaller case and scale smoothly
    wm = bb.bb_schedule_counts(32768, 128, 16)
    assert wm.stages == 8
    # leading term 4 n^2 b (1 + 1/d) ~ the executed flops within a factor of 2
    assert 0.5 < wm.flops / (4 * 32768**2 * 128 * (1 + 1 / 16)) < 2.0


def test_default_tuning(bb):
    t64 = bb.bb_default_tuning(32768, 128, bb.BB_F64)
    t32 = bb.bb_default_tuning(32768, 128, bb.BB_F32)
    # one 128-byte line per tile row: 16 doubles, 32 floats (Section V-B)
    assert t64.tw == 16 and t32.tw == 32
    assert t64.tpb == 0          # 0: sized per stage (two threads per panel row + a reflector warp)


def test_host_side_argument_errors(bb):
    L = bb.lib()
    # validation happens before any CUDA call
    assert L.band_to_bidiag(0, 4, 1, 16, 5, 16, 16, None) == bb.BB_ERR_ARG
    assert L.band_to_bidiag(10, -1, 1, 16, 5, 16, 16, None) == bb.BB_ERR_ARG
    assert L.band_to_bidiag(10, 4, 1, 16, 4, 16, 16, None) == bb.BB_ERR_ARG     # ldab < b+1
    assert L.band_to_bidiag(10, 4, 1, None, 5, 16, 16, None) == bb.BB_ERR_ARG
    assert L.band_to_bidiag(10, 4, 7, 16, 5, 16, 16, None) == bb.BB_ERR_ARG     # dtype
    assert L.band_to_bidiag(10, 4, 1, 16, 5, 16, None, None) == bb.BB_ERR_ARG   # e_out
    assert L.band_to_bidiag(1 << 20, 4, 1, 16, 5, 16, 16, None) == bb.BB_ERR_UNSUPPORTED
    t = bb.Tuning(tw=40)
    assert L.band_to_bidiag_ex(10, 4, 1, 16, 5, 16, 16, ctypes.byref(t), None, 0, None) == bb.BB_ERR_ARG
    t = bb.Tuning(tpb=100)     # not a multiple of 32
    assert L.band_to_bidiag_ex(10, 4, 1, 16, 5, 16, 16, ctypes.byref(t), None, 0, None) == bb.BB_ERR_ARG
    # caller workspace too small / misaligned
    ws = bb.band_to_bidiag_workspace_size(100, 8, bb.BB_F64)
    assert ws > 0 and ws % 256 == 0
    assert L.band_to_bidiag_ex(100, 8, 1, 16, 9, 16, 16, None, 256, 1024, None) == bb.BB_ERR_WORKSPACE
    assert L.band_to_bidiag_ex(100, 8, 1, 16, 9, 16, 16, None, 257, ws, None) == bb.BB_ERR_WORKSPACE
    assert bb.status_string(bb.BB_ERR_TIMEOUT) == "device wait timed out"


def test_tuning_entry_points_host_checks(bb):
    L = bb.lib()
    D, H = 8, 32
    assert bb.bb_mlp_param_count(D, H) == H * D + H + H * H + H + H + 1
    assert bb.bb_mlp_param_count(8, 48) == 0          # hidden must be a multiple of 32
    assert bb.bb_mlp_param_count(33, 64) == 0         # in_dim <= 32
    assert bb.bb_mlp_param_count(0, 32) == 0
    assert bb.bb_mlp_backward_scratch(H, 10) == 10 * (1 + 2 * H)
    # validation happens before any CUDA call
    assert L.bb_mlp_forward(D, H, None, 16, 4, 16, 16, 16, None) == bb.BB_ERR_ARG
    assert L.bb_mlp_forward(D, 40, 16, 16, 4, 16, 16, 16, None) == bb.BB_ERR_ARG
    assert L.bb_mlp_backward(D, H, 16, 16, 16, 16, 16, 16, 0, 16, 16, None) == bb.BB_ERR_ARG
    assert L.bb_mlp_adam(0, 16, 16, 16, 16, 1, 1e-3, 0.9, 0.999, 1e-8, None) == bb.BB_ERR_ARG
    assert L.bb_mlp_adam(10, 16, 16, 16, 16, 0, 1e-3, 0.9, 0.999, 1e-8, None) == bb.BB_ERR_ARG
    times = (ctypes.c_float * 1)()
    best = ctypes.c_int()
    assert L.bb_autotune(100, 8, 1, 16, 9, 16, 16, None, 1, 1, times, ctypes.byref(best),
                         None) == bb.BB_ERR_ARG
    cand = (bb.Tuning * 1)(bb.Tuning(tw=16))
    assert L.bb_autotune(100, 8, 1, 16, 9, 16, 16, cand, 0, 1, times, ctypes.byref(best),
                         None) == bb.BB_ERR_ARG
    assert L.bb_autotune(100, 8, 1, 16, 9, 16, 16, cand, 1, 0, times, ctypes.byref(best),
                         None) == bb.BB_ERR_ARG
    bad = (bb.Tuning * 1)(bb.Tuning(tw=64))
    assert L.bb_autotune(100, 8, 1, 16, 9, 16, 16, bad, 1, 1, times, ctypes.byref(best),
                         None) == bb.BB_ERR_ARG


def test_bidiag_sigma_host_checks(bb):
    L = bb.lib()
    ws = bb.lib().bb_bidiag_sigma_workspace_size(100)
    # bounds + grid counts (66048 B) + 2n doubles of squared couplings
    assert ws == 66048 + 16 * 100
    # validation happens before any CUDA call
    assert L.bb_bidiag_sigma(0, 1, 16, 16, 16, 256, ws, None) == bb.BB_ERR_ARG
    assert L.bb_bidiag_sigma(10, 7, 16, 16, 16, 256, ws, None) == bb.BB_ERR_ARG
    assert L.bb_bidiag_sigma(10, 1, 16, None, 16, 256, ws, None) == bb.BB_ERR_ARG
    assert L.bb_bidiag_sigma(10, 1, None, 16, 16, 256, ws, None) == bb.BB_ERR_ARG
    assert L.bb_bidiag_sigma(10, 1, 16, 16, 16, None, ws, None) == bb.BB_ERR_WORKSPACE
    assert L.bb_bidiag_sigma(10, 1, 16, 16, 16, 256, 8, None) == bb.BB_ERR_WORKSPACE
    assert L.bb_bidiag_sigma(10, 1, 16, 16, 16, 257, ws, None) == bb.BB_ERR_WORKSPACE


def test_half_storage_host_model(bb):
    # 16-bit working band, FP32 panels in shared memory
    t = bb.Tuning(tw=32)
    w16 = bb.band_to_bidiag_workspace_size(4096, 128, bb.BB_F16, t)
    w32 = bb.band_to_bidiag_workspace_size(4096, 128, bb.BB_F32, t)
    assert 0 < w16 < w32
    assert bb.bb_shared_bytes(4096, 128, bb.BB_BF16, t) == bb.bb_shared_bytes(4096, 128, bb.BB_F32, t)
    assert bb.bb_default_tuning(4096, 128, bb.BB_F16).tw == 32
    assert bb.band_to_bidiag_workspace_size(4096, 128, 4, t) == 0      # unknown dtype


def test_stage_count_limit(bb):
    # 2047 stages or more would overflow the int progress words: refused on the host
    assert bb.band_to_bidiag_workspace_size(4096, 2047, bb.BB_F64, bb.Tuning(tw=1)) > 0
    assert bb.band_to_bidiag_workspace_size(4096, 2048, bb.BB_F64, bb.Tuning(tw=1)) == 0
    L = bb.lib()
    t = bb.Tuning(tw=1)
    assert L.band_to_bidiag_ex(4096, 2048, 1, 16, 2049, 16, 16, ctypes.byref(t), None, 0,
                               None) == bb.BB_ERR_UNSUPPORTED


def _group_window_bytes(es, b, tw, K, maxm):
    """Largest group-kernel window over the stages: V (K+d) x PV, H (bw-K-d) x
    PH with odd pitches, plus K right and K left reflectors (vectors and
    {tau, beta, vs}) and the staging vector."""
    best, bw = 0, b
    while bw > 1:
        d = min(tw, bw - 1)
        k = min(K, (bw - d) // 3)
        if k >= 1:
            pv, ph = (bw + k + d) | 1, (k + d) | 1
            best = max(best, (k + d) * pv + (bw - k - d) * ph)
        bw -= d
    small = (2 * K * maxm + 8 * K + (maxm + 1) + 64 + 3) & ~3
    return es * (small + best) if best else 0


def test_shared_bytes_model(bb):
    # per-sweep kernel: both panels of a row-bulge, (MAXM + 1) x (b + TW + 2) elements each
    t = bb.Tuning(tw=16, group=-1, teams=-1)
    assert bb.bb_shared_bytes(4096, 128, bb.BB_F64, t) == 8 * 18 * 2 * (128 + 16 + 2)
    t = bb.Tuning(tw=32, group=-1, teams=-1)
    assert bb.bb_shared_bytes(4096, 512, bb.BB_F32, t) == 4 * 34 * 2 * (512 + 32 + 2)
    assert bb.bb_shared_bytes(4096, 512, bb.BB_F64, bb.Tuning(tw=32, group=-1, teams=-1)) > 227 * 1024
    assert bb.bb_shared_bytes(0, 4, bb.BB_F64) == 0
    # with the group kernel: the larger of the two
    for (b, tw, es, dt, K, maxm) in [(128, 16, 8, bb.BB_F64, 8, 17), (128, 32, 4, bb.BB_F32, 16, 33),
                                     (64, 32, 8, bb.BB_F64, 4, 33), (40, 8, 4, bb.BB_F32, 8, 9)]:
        per_sweep = es * (maxm + 1) * 2 * (b + tw + 2)
        got = bb.bb_shared_bytes(4096, b, dt, bb.Tuning(tw=tw, group=K, teams=-1))
        assert got == max(per_sweep, _group_window_bytes(es, b, tw, K, maxm)), (b, tw, K)
        # team kernel on the last stage: circular window (2W + 3) bw columns of
        # 3 bw - 1 band offsets (even pitch) plus per-team scratch
        bwl = b
        while bwl - min(tw, bwl - 1) > 1:
            bwl -= min(tw, bwl - 1)
        for W in (2, 4):
            pitch = 3 * bwl - 1 + ((3 * bwl - 1) & 1)
            team = es * ((2 * W + 3) * bwl * pitch + W * ((5 * maxm + 73 + 3) & ~3))
            got = bb.bb_shared_bytes(4096, b, dt, bb.Tuning(tw=tw, group=-1, teams=W))
            assert got == max(per_sweep, team), (b, tw, W)


def test_tuner_features_and_grid():
    from paper_2510_12705_gb300 import tuner
    c = tuner.candidates()
    assert len(c) == len(set(c)) == len(tuner.TWS) * len(tuner.GROUPS) * len(tuner.SIFS)
    f = tuner.features(65536, 256, "f32", c[0])
    assert len(f) == tuner.IN_DIM and all(abs(x) < 4 for x in f)
    g = tuner.default_grid()
    assert all(b <= n // 4 and n * b <= (1 << 22) for n, b, _ in g)
    assert (65536, 256, "f32") not in g
    assert {dt for _, _, dt in g} == {"f32", "f64"} and len(set(g)) == len(g)


def test_workspace_size_model(bb):
    # working band of height b + 2 TW + 1 (Section IV storage format), padded
    n, b = 32768, 128
    ws = bb.band_to_bidiag_workspace_size(n, b, bb.BB_F64)
    ldw = -(-(b + 2 * 16) // 4) * 4 + 1          # ldw - 1 a multiple of 4 (16-byte phase)
    assert ldw >= b + 2 * 16 + 1
    assert ldw * n * 8 <= ws <= ldw * n * 8 + 128 * n + 4096


def test_committed_tuner_artifacts_consistent():
    """The packaged model matches the tuner's feature set and candidates, its
    timings file covers the training grid (held-out problem excluded), and the
    FP64 MLP oracle evaluates the weights to the pick the bench's reference arm
    uses."""
    import json
    import os

    import bench
    from paper_2510_12705_gb300 import tuner
    if not os.path.exists(tuner.MODEL_PATH):
        import pytest
        pytest.skip("no trained tuner model")
    with open(tuner.MODEL_PATH) as f:
        m = json.load(f)
    assert m["in_dim"] == tuner.IN_DIM and [tuple(c) for c in m["candidates"]] == tuner.candidates()
    D, H = m["in_dim"], m["hidden"]
    assert len(m["params"]) == H * D + H + H * H + H + H + 1
    timings = os.path.join(os.path.dirname(tuner.MODEL_PATH), "tuner_timings.json")
    with open(timings) as f:
        rows = json.load(f)
    probs = {(r["n"], r["b"], r["dtype"]) for r in rows}
    assert tuner.HELD_OUT not in probs
    assert probs <= set(tuner.default_grid())
    assert all(r["ms"] > 0 for r in rows)
    assert bench.reference_tw(32768, 128) in tuner.TWS


@pytest.mark.parametrize("n,b,tw", [(32768, 128, 32), (32768, 128, 16), (300, 40, 16), (100, 7, 3)])
def test_stage_counts_sum_to_schedule(bb, n, b, tw):
    tot = bb.bb_schedule_counts(n, b, tw)
    parts = [bb.bb_stage_counts(n, b, tw, s) for s in range(tot.stages)]
    assert all(p.stages == tot.stages for p in parts)
    assert sum(p.steps for p in parts) == tot.steps
    assert sum(p.flops for p in parts) == pytest.approx(tot.flops, rel=1e-12)
    assert sum(p.elements for p in parts) == pytest.approx(tot.elements, rel=1e-12)


def test_dense_to_band_argument_checks(bb):
    """dense_to_band rejects bad arguments before any GPU work (Section V-A's
    stage 1 entry point)."""
    L = bb.lib()
    fake = 0x1000
    n, b = 64, 8
    assert L.dense_to_band(0, b, bb.BB_F64, fake, 64, fake, 9, None, 0, None) == bb.BB_ERR_ARG
    assert L.dense_to_band(n, 0, bb.BB_F64, fake, 64, fake, 9, None, 0, None) == bb.BB_ERR_ARG
    assert L.dense_to_band(n, b, bb.BB_F64, fake, 63, fake, 9, None, 0, None) == bb.BB_ERR_ARG
    assert L.dense_to_band(n, b, bb.BB_F64, fake, 64, fake, 8, None, 0, None) == bb.BB_ERR_ARG
    assert L.dense_to_band(n, b, bb.BB_F64, None, 64, fake, 9, None, 0, None) == bb.BB_ERR_ARG
    assert L.dense_to_band(n, b, bb.BB_F16, fake, 64, fake, 9, None, 0, None) == bb.BB_ERR_UNSUPPORTED
    assert L.dense_to_band(n, b, 9, fake, 64, fake, 9, None, 0, None) == bb.BB_ERR_ARG
    assert L.dense_to_band(n, b, bb.BB_F64, fake, 64, fake, 9, fake, 16, None) == bb.BB_ERR_WORKSPACE
    assert bb.dense_to_band_workspace_size(0, b, bb.BB_F64) == 0
    assert bb.dense_to_band_workspace_size(n, b, bb.BB_F16) == 0
    ws64 = bb.dense_to_band_workspace_size(n, b, bb.BB_F64)
    assert 8 * n * n <= ws64 <= 8 * n * n + 8 * (6 * n * b + 2 * b * b) + 4096
    assert bb.dense_to_band_workspace_size(n, b, bb.BB_F32) < ws64
    big = 1 << 31
    assert L.dense_to_band_qp(n, b, bb.BB_F64, fake, 64, fake, 9, fake, big, fake, 64, None, 0,
                              None) == bb.BB_ERR_UNSUPPORTED
    assert L.dense_to_band_qp(n, b, bb.BB_F64, fake, 64, fake, 9, fake, 64, fake, big, None, 0,
                              None) == bb.BB_ERR_UNSUPPORTED
    assert L.dense_to_band_qp(n, b, bb.BB_F64, fake, 64, fake, 9, fake, 63, fake, 64, None, 0,
                              None) == bb.BB_ERR_ARG


def test_vectors_entry_point_checks_and_store_size(bb):
    """band_to_bidiag_vectors: argument checks before any GPU work, and the
    reflector store is two slots of (MAXM + 1, rounded to 4) values per
    row-bulge on top of the reduction's workspace."""
    L = bb.lib()
    fake = 0x1000
    n, b = 300, 40
    t = bb.Tuning(tw=16)
    assert L.band_to_bidiag_vectors(n, b, bb.BB_F64, fake, b + 1, fake, fake, None, n, fake, n, t, None, 0,
                                    None) == bb.BB_ERR_ARG
    assert L.band_to_bidiag_vectors(n, b, bb.BB_F64, fake, b + 1, fake, fake, fake, n - 1, fake, n, t, None, 0,
                                    None) == bb.BB_ERR_ARG
    assert L.band_to_bidiag_vectors(n, b, bb.BB_F16, fake, b + 1, fake, fake, fake, n, fake, n, t, None, 0,
                                    None) == bb.BB_ERR_UNSUPPORTED
    assert L.band_to_bidiag_vectors_workspace_size(n, b, bb.BB_F16, t) == 0
    base = bb.band_to_bidiag_workspace_size(n, b, bb.BB_F64, bb.Tuning(tw=16, teams=-1))
    got = L.band_to_bidiag_vectors_workspace_size(n, b, bb.BB_F64, t)
    steps = bb.bb_schedule_counts(n, b, 16).steps
    store = 2 * steps * ((17 + 1 + 3) & ~3) * 8
    assert got >= base + store and got <= base + store + 512


@pytest.mark.parametrize("n,b,tw", [(1, 0, 16), (2, 1, 4), (50, 3, 2), (200, 16, 8), (300, 40, 16),
                                    (257, 33, 32), (129, 128, 32), (97, 200, 16), (400, 64, 5)])
def test_reflector_index_matches_generation_order(bb, n, b, tw):
    """The slot a kernel stores a row-bulge's reflectors in (closed form:
    earlier stages' row-bulges + earlier sweeps' + s) equals the running count
    of the back-transformation, which walks stage by stage, sweep by sweep,
    step by step.  A row-bulge exists while its block's first column
    c = R + (bw - d) + s*bw has a column to its right (Section III's chase)."""
    k = 0
    bw, stage = min(b, n - 1), 0
    while bw > 1:
        d = min(tw, bw - 1)
        for R in range(n - 1):
            s = 0
            while R + (bw - d) + s * bw < n - 1:
                assert bb.bb_reflector_index(n, b, tw, stage, R, s) == k
                k += 1
                s += 1
            with pytest.raises(bb.BBError):        # one past the sweep's last row-bulge
                bb.bb_reflector_index(n, b, tw, stage, R, s)
        bw -= d
        stage += 1
    assert k == bb.bb_schedule_counts(n, b, tw).steps
    with pytest.raises(bb.BBError):                # no such stage
        bb.bb_reflector_index(n, b, tw, stage, 0, 0)


def test_reflector_index_at_the_bench_size(bb):
    """n = 32768, b = 128, TW = 32: sampled sweeps against prefix sums of the
    per-sweep row-bulge counts (same definition as above)."""
    n, b, tw = 32768, 128, 32
    base, bw, stage = 0, b, 0
    rng = np.random.default_rng(0)
    while bw > 1:
        d = min(tw, bw - 1)
        R = np.arange(n - 1)
        c0 = R + (bw - d)
        ns = np.where(c0 < n - 1, (n - 2 - c0) // bw + 1, 0)
        before = np.concatenate([[0], np.cumsum(ns)])
        for r in list(rng.integers(0, n - 1, 40)) + [0, n - 2 - (bw - d)]:
            r = int(r)
            if ns[r] == 0:
                continue
            for s in {0, int(ns[r]) - 1, int(ns[r]) // 2}:
                assert bb.bb_reflector_index(n, b, tw, stage, r, s) == base + before[r] + s
        base += int(before[-1])
        bw -= d
        stage += 1
    assert base == bb.bb_schedule_counts(n, b, tw).steps


def test_binding_refuses_host_tensors(bb):
    """The Python binding passes raw pointers to the kernels, so every tensor
    they read or write must be a CUDA tensor: host tensors (whose pointers
    would reach a kernel as device addresses) raise ValueError before any
    library call."""
    import torch
    h = torch.zeros(64, dtype=torch.float32)
    with pytest.raises(ValueError):
        bb._device_buffer(h, "x")
    with pytest.raises(ValueError):
        bb._workspace_args(torch.zeros(16, dtype=torch.uint8), h)
    assert bb._workspace_args(None, h) == (None, 0)
    with pytest.raises(ValueError):
        bb.bb_bidiag_sigma(torch.zeros(8, dtype=torch.float64), torch.zeros(7, dtype=torch.float64))
    with pytest.raises(ValueError):
        bb.bb_mlp_adam(h, h, h, h, 1, 1e-3)
    X = torch.zeros(4, 8, dtype=torch.float32)
    with pytest.raises(ValueError):
        bb.bb_mlp_forward(8, 32, h, X, h, h, h)
    with pytest.raises(ValueError):                     # X's width is not in_dim
        bb.bb_mlp_forward(8, 32, h, torch.zeros(4, 5), h, h, h)
    band = torch.zeros(10, 3, dtype=torch.float64)
    d = torch.zeros(10, dtype=torch.float64)
    e = torch.zeros(9, dtype=torch.float64)
    for call in (lambda: bb.band_to_bidiag(band, 2, d, e),
                 lambda: bb.band_to_bidiag_ex(band, 2, d, e),
                 lambda: bb.band_to_bidiag_noalloc(band, 2, d, e),
                 lambda: bb.band_to_bidiag_vectors(band, 2, d, e, torch.zeros(10, 10, dtype=torch.float64),
                                                   torch.zeros(10, 10, dtype=torch.float64)),
                 lambda: bb.dense_to_band(torch.zeros(10, 10, dtype=torch.float64), 2, band)):
        with pytest.raises(ValueError):
            call()


_C_PROGRAM = r"""
#include <stdio.h>
#include "band_bidiag.h"
int main(void) {
    int64_t st = 0, sp = 0, k = -1;
    double fl = 0, el = 0;
    if (bb_schedule_counts(32768, 128, 32, &st, &sp, &fl, &el) != BB_OK) return 1;
    if (bb_reflector_index(32768, 128, 32, 1, 5, 3, &k) != BB_OK) return 2;
    if (band_to_bidiag(0, 4, BB_F64, 0, 5, 0, 0, 0) != BB_ERR_ARG) return 3;
    printf("%lld %lld %.17g %.17g %lld %s\n", (long long)st, (long long)sp, fl, el, (long long)k,
           bb_status_string(BB_ERR_ARG));
    return 0;
}
"""


def test_header_is_plain_c_and_links_from_c(bb, tmp_path):
    """The boundary is a C ABI: the header compiles on its own as C99 and as
    C++, and a plain C program links against the library and gets the same
    host-side answers as the Python binding (no GPU call is made)."""
    import shutil
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    inc = os.path.join(ROOT, "include")
    hdr = os.path.join(inc, "band_bidiag.h")
    subprocess.check_call([gcc, "-fsyntax-only", "-x", "c", "-std=c99", "-Wall", "-Wextra", "-Werror", hdr])
    gxx = shutil.which("g++")
    if gxx:
        subprocess.check_call([gxx, "-fsyntax-only", "-x", "c++", "-Wall", "-Werror", hdr])
    src = tmp_path / "prog.c"
    src.write_text(_C_PROGRAM)
    libdir = os.path.dirname(bb.LIB_PATH)
    exe = tmp_path / "prog"
    subprocess.check_call([gcc, "-std=c99", "-Wall", "-Werror", "-I", inc, str(src), "-L", libdir,
                           "-lbandbidiag", f"-Wl,-rpath,{libdir}", "-o", str(exe)])
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stderr
    st, sp, fl, el, k, *msg = out.stdout.split()
    ref = bb.bb_schedule_counts(32768, 128, 32)
    assert (int(st), int(sp)) == (ref.stages, ref.steps)
    assert float(fl) == ref.flops and float(el) == ref.elements
    assert int(k) == bb.bb_reflector_index(32768, 128, 32, 1, 5, 3)
    assert " ".join(msg) == bb.lib().bb_status_string(bb.BB_ERR_ARG).decode()


@pytest.mark.parametrize("n,b,tw", [(1, 0, 16), (2, 1, 4), (100, 3, 2), (300, 40, 16), (257, 33, 32),
                                    (2048, 128, 32)])
def test_back_transformation_flop_count(bb, n, b, tw):
    """bench_vectors reports the back-transformation's rate against
    8 n * sum(m); its closed sum over the schedule equals a walk over every
    row-bulge, and the walk's count is the schedule's row-bulge count."""
    from paper_2510_12705_gb300.bench_vectors import reflector_length_sum
    total, count, bw = 0, 0, min(b, n - 1)
    while bw > 1:
        d = min(tw, bw - 1)
        for R in range(n - 1):
            c = R + (bw - d)
            while c < n - 1:
                total += min(d + 1, n - c)
                count += 1
                c += bw
        bw -= d
    assert reflector_length_sum(n, b, tw) == total
    assert count == bb.bb_schedule_counts(n, b, tw).steps

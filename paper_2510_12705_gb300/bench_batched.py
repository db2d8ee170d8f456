"""Batched workload: many independent band matrices of uneven n and b.

    python -m paper_2510_12705_gb300.bench_batched [--count 512] [--reps 5]

512 matrices, n ~ U[256, 4096], b uniform over {8, 16, 32, 64}, iid N(0, 1)
entries (seed 3), FP32.  Compares one CUDA-graph replay of the batched
reduction (one persistent launch per stage for all matrices) with a loop that
reduces the matrices one by one through band_to_bidiag.  Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--count", type=int, default=512)
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--seed", type=int, default=3)
    ap.add_argument("--dtype", choices=["f32", "f64"], default="f32")
    args = ap.parse_args(argv)

    import numpy as np
    import torch

    import bandgen
    import paper_2510_12705_gb300 as bb
    from paper_2510_12705_gb300 import build

    build.build()
    dt = torch.float32 if args.dtype == "f32" else torch.float64
    probs = bandgen.batch_problems(args.count, seed=args.seed)
    items = []
    flops = 0.0
    tw = bb.bb_default_tuning(4096, 64, bb.BB_F32 if args.dtype == "f32" else bb.BB_F64).tw
    for (n, b, s) in probs:
        band = torch.from_numpy(bandgen.random_band(n, b, seed=s)).to("cuda", dt)
        d = torch.empty(n, device="cuda", dtype=dt)
        e = torch.empty(n - 1, device="cuda", dtype=dt)
        items.append((band, b, d, e))
        flops += bb.bb_schedule_counts(n, b, tw).flops

    plan = bb.BatchPlan(items)
    ws = torch.empty(plan.workspace_bytes, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(stream):
        plan.execute(ws, stream=stream)           # warm-up, module loading
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        plan.execute(ws)
    g.replay()
    torch.cuda.synchronize()
    batched = []
    for _ in range(args.reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        g.replay()
        e1.record()
        torch.cuda.synchronize()
        batched.append(e0.elapsed_time(e1))
    st_b = bb.bb_device_status(reset=True)
    ref = [(d.clone(), e.clone()) for (_, _, d, e) in items]

    # one reduction per matrix, same stream, workspaces preallocated
    wss = [torch.empty(bb.band_to_bidiag_workspace_size(band.shape[0], b, bb._dtype_code(dt)),
                       dtype=torch.uint8, device="cuda") for (band, b, _, _) in items]
    for (band, b, d, e), w in zip(items, wss):
        bb.band_to_bidiag_ex(band, b, d, e, workspace=w)
    torch.cuda.synchronize()
    loop = []
    for _ in range(args.reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for (band, b, d, e), w in zip(items, wss):
            bb.band_to_bidiag_ex(band, b, d, e, workspace=w)
        e1.record()
        torch.cuda.synchronize()
        loop.append(e0.elapsed_time(e1))
    st_l = bb.bb_device_status(reset=True)
    same = all(torch.equal(d, rd) and torch.equal(e, re) for (_, _, d, e), (rd, re) in zip(items, ref))
    tb, tl = float(np.median(batched)), float(np.median(loop))
    print(json.dumps({
        "workload": f"{args.count} band matrices, n~U[256,4096], b in {{8,16,32,64}}, {args.dtype}, seed {args.seed}",
        "flops": flops, "batched_graph_ms": tb, "per_matrix_loop_ms": tl,
        "speedup": tl / tb, "batched_gflops": flops / (tb * 1e-3) / 1e9,
        "loop_gflops": flops / (tl * 1e-3) / 1e9, "bitwise_equal": bool(same),
        "status": [st_b, st_l]}))
    return 0 if (st_b == 0 and st_l == 0 and same) else 1


if __name__ == "__main__":
    sys.exit(main())

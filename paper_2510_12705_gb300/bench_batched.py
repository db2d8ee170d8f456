"""Batched workload: many independent band matrices of uneven n and b.

    python -m paper_2510_12705_gb300.bench_batched [--count 512] [--reps 5] [--tune]

512 matrices, n ~ U[256, 4096], b uniform over {8, 16, 32, 64}, iid N(0, 1)
entries (seed 3), FP32.  Compares one CUDA-graph replay of the batched
reduction (one persistent launch per stage for all matrices) with a loop that
reduces the matrices one by one through band_to_bidiag.  With --tune the
batched plan's hyperparameters (TW, sweeps per CTA, CTAs per SM: the learned
tuner's candidates) are searched exhaustively, each candidate timed as a
graph replay of the whole batch, and the learned tuner's pick for the batch's
widest problem is timed beside it.  Prints one JSON line.
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
    ap.add_argument("--tune", action="store_true", help="search the batch plan's hyperparameters")
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

    def time_plan(tuning, reps):
        """Median graph-replay time of the whole batch under one plan tuning."""
        plan = bb.BatchPlan(items, tuning)
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
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            g.replay()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.median(ts)), ts

    search = None
    if args.tune:
        from paper_2510_12705_gb300 import tuner
        nsm = torch.cuda.get_device_properties(0).multi_processor_count
        cands = tuner.candidates()
        times = [time_plan(tuner._tuning(c, nsm), 1)[0] for c in cands]
        best = int(np.argmin(times))
        nmax = max(n for n, _, _ in probs)
        bmax = max(b for _, b, _ in probs)
        mlp, src = tuner.tuning_for(nmax, bmax, args.dtype)
        search = {"candidates": [list(c) for c in cands], "ms": times, "best": list(cands[best]),
                  "best_ms": times[best], "default_ms": time_plan(None, 1)[0],
                  "mlp_pick": [mlp.tw, mlp.group, int(mlp.sweeps_in_flight > 0)], "mlp_source": src,
                  "mlp_ms": time_plan(mlp, 1)[0]}
        tuned = tuner._tuning(cands[best], nsm)
    else:
        tuned = None
    tb_default, _ = time_plan(None, args.reps)
    tb, batched = time_plan(tuned, args.reps) if tuned is not None else (tb_default, None)
    st_b = bb.bb_device_status(reset=True)
    if tuned is not None:                     # the outputs compared below: the default plan's
        time_plan(None, 1)
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
    tl = float(np.median(loop))
    if tuned is not None and tuned.tw != tw:      # the tuned plan's schedule has its own flop count
        flops_b = sum(bb.bb_schedule_counts(n, b, tuned.tw).flops for (n, b, _) in probs)
    else:
        flops_b = flops
    print(json.dumps({
        "workload": f"{args.count} band matrices, n~U[256,4096], b in {{8,16,32,64}}, {args.dtype}, seed {args.seed}",
        "flops": flops, "batched_graph_ms": tb, "batched_default_plan_ms": tb_default,
        "per_matrix_loop_ms": tl, "speedup": tl / tb, "batched_gflops": flops_b / (tb * 1e-3) / 1e9,
        "tuned_tw": tuned.tw if tuned is not None else tw,
        "loop_gflops": flops / (tl * 1e-3) / 1e9, "bitwise_equal_default_plan_vs_loop": bool(same),
        "plan_search": search, "status": [st_b, st_l]}))
    return 0 if (st_b == 0 and st_l == 0 and same) else 1


if __name__ == "__main__":
    sys.exit(main())

"""Stage 1 timing: dense n x n -> upper band (dense_to_band) on the GPU.

    python -m paper_2510_12705_gb300.bench_dense [--n 2048 4096 8192] [--b 64 128] [--reps 3]

Input: iid N(0, 1) dense matrices (seed 0), FP64 and FP32.  One line of JSON
per configuration: median time (CUDA events around the call, workspace
preallocated) and GFLOP/s against the leading-order flop count 8/3 n^3 of a
two-sided orthogonal reduction (Householder QR and LQ of every panel applied
to the trailing matrix).
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
    ap.add_argument("--n", type=int, nargs="+", default=[2048, 4096, 8192])
    ap.add_argument("--b", type=int, nargs="+", default=[64, 128])
    ap.add_argument("--reps", type=int, default=3)
    args = ap.parse_args(argv)

    import numpy as np
    import torch

    import paper_2510_12705_gb300 as bb
    from paper_2510_12705_gb300 import build

    build.build()
    for n in args.n:
        a64 = torch.randn(n, n, generator=torch.Generator().manual_seed(0), dtype=torch.float64).cuda()
        for dt, name, code in ((torch.float64, "f64", bb.BB_F64), (torch.float32, "f32", bb.BB_F32)):
            a = a64.to(dt)
            for b in args.b:
                band = torch.empty((n, b + 1), device="cuda", dtype=dt)
                ws = torch.empty(bb.dense_to_band_workspace_size(n, b, code), dtype=torch.uint8, device="cuda")
                bb.dense_to_band(a, b, band, workspace=ws)          # warm-up
                torch.cuda.synchronize()
                ts = []
                for _ in range(args.reps):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    bb.dense_to_band(a, b, band, workspace=ws)
                    e1.record()
                    torch.cuda.synchronize()
                    ts.append(e0.elapsed_time(e1))
                ms = float(np.median(ts))
                flops = 8.0 / 3.0 * n ** 3
                print(json.dumps({"n": n, "b": b, "dtype": name, "ms": ms,
                                  "gflops_8n3_over_3": flops / (ms * 1e-3) / 1e9}), flush=True)
                del band, ws
    return 0


if __name__ == "__main__":
    sys.exit(main())

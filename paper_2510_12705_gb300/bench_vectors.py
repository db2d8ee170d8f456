"""Cost of the band stage's singular vectors on the GPU: band_to_bidiag (d and
e only) against band_to_bidiag_vectors (d, e and the orthogonal factors Q and
P, through the reflector store and the back-transformation).

    python -m paper_2510_12705_gb300.bench_vectors [--n 1024 2048] [--b 128] [--tw 32] [--reps 3]

Input: bandgen.random_band(n, b, seed=0), FP64 and FP32.  One line of JSON
per configuration: median times (CUDA events around each call, workspaces
preallocated), the time the vectors add, and that extra time's rate against
the back-transformation's flop count.  Each reflector of length m updates
every one of the n rows of its factor with a dot product and an axpy (4m
flops per row); both sides together give 8 n * sum(m) over the row-bulges.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def reflector_length_sum(n: int, b: int, tw: int) -> int:
    """sum of m = min(d + 1, n - c) over every row-bulge of the schedule
    (block column c = R + (bw - d) + s*bw of step s of sweep R)."""
    import numpy as np
    total = 0
    bw = min(b, n - 1)
    while bw > 1:
        d = min(tw, bw - 1)
        c = np.arange(n - 1) + (bw - d)
        while True:
            live = c < n - 1
            if not live.any():
                break
            total += int(np.minimum(d + 1, n - c[live]).sum())
            c = c + bw
        bw -= d
    return total


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, nargs="+", default=[1024, 2048])
    ap.add_argument("--b", type=int, default=128)
    ap.add_argument("--tw", type=int, default=32)
    ap.add_argument("--reps", type=int, default=3)
    args = ap.parse_args(argv)

    import numpy as np
    import torch

    import bandgen
    import paper_2510_12705_gb300 as bb
    from paper_2510_12705_gb300 import build

    build.build()

    def timed(fn):
        fn()                                     # warm-up, module loading
        torch.cuda.synchronize()
        ts = []
        for _ in range(args.reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.median(ts))

    for n in args.n:
        ab = bandgen.random_band(n, args.b, seed=0)
        flops = 8.0 * n * reflector_length_sum(n, args.b, args.tw)
        for dt, name, code in ((torch.float64, "f64", bb.BB_F64), (torch.float32, "f32", bb.BB_F32)):
            tun = bb.Tuning(tw=args.tw)
            band = torch.from_numpy(ab).to("cuda", dt)
            d = torch.empty(n, device="cuda", dtype=dt)
            e = torch.empty(n - 1, device="cuda", dtype=dt)
            q = torch.empty((n, n), device="cuda", dtype=dt)
            p = torch.empty((n, n), device="cuda", dtype=dt)
            ws1 = torch.empty(bb.band_to_bidiag_workspace_size(n, args.b, code, tun), dtype=torch.uint8,
                              device="cuda")
            ws2 = torch.empty(int(bb.lib().band_to_bidiag_vectors_workspace_size(n, args.b, code,
                                                                                  bb._tuning_ptr(tun))),
                              dtype=torch.uint8, device="cuda")
            ms_red = timed(lambda: bb.band_to_bidiag_ex(band, args.b, d, e, tuning=tun, workspace=ws1))
            ms_vec = timed(lambda: bb.band_to_bidiag_vectors(band, args.b, d, e, q, p, tuning=tun, workspace=ws2))
            status = bb.bb_device_status(reset=True)
            extra = ms_vec - ms_red
            print(json.dumps({
                "n": n, "b": args.b, "tw": args.tw, "dtype": name, "reduction_ms": ms_red, "vectors_ms": ms_vec,
                "extra_ms": extra, "store_bytes": int(ws2.numel()) - int(ws1.numel()),
                "backtransform_flops": flops,
                "extra_gflops": flops / (extra * 1e-3) / 1e9 if extra > 0 else None,
                "device_status": status}), flush=True)
            del band, d, e, q, p, ws1, ws2
    return 0


if __name__ == "__main__":
    sys.exit(main())

"""Run the reduction on one synthetic band matrix (for profiling and timing).

    python -m paper_2510_12705_gb300.run_case --n 8192 --b 64 --dtype f64 --reps 2

Prints one JSON line with the CUDA-event time of the persistent bulge-chasing
kernel and of the whole call for each repetition.
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
    ap.add_argument("--n", type=int, default=8192)
    ap.add_argument("--b", type=int, default=64)
    ap.add_argument("--dtype", choices=["f64", "f32"], default="f64")
    ap.add_argument("--reps", type=int, default=1)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--tw", type=int, default=0)
    ap.add_argument("--tpb", type=int, default=0)
    ap.add_argument("--sif", type=int, default=0)
    ap.add_argument("--sigma", action="store_true",
                    help="also time the singular values of the result on the GPU (bb_bidiag_sigma)")
    ap.add_argument("--tuned", action="store_true",
                    help="hyperparameters from the trained tuner (as bench.py uses them)")
    args = ap.parse_args(argv)

    import torch

    import bandgen
    import paper_2510_12705_gb300 as bb
    from paper_2510_12705_gb300 import build

    build.build()
    dt = torch.float64 if args.dtype == "f64" else torch.float32
    code = bb.BB_F64 if args.dtype == "f64" else bb.BB_F32
    band = torch.from_numpy(bandgen.random_band(args.n, args.b, seed=args.seed)).to("cuda", dt)
    d = torch.empty(args.n, device="cuda", dtype=dt)
    e = torch.empty(max(args.n - 1, 1), device="cuda", dtype=dt)
    if args.tuned:
        from paper_2510_12705_gb300 import tuner
        tun, _ = tuner.tuning_for(args.n, args.b, args.dtype)
    else:
        tun = bb.bb_default_tuning(args.n, args.b, code)
    if args.tw:
        tun.tw = args.tw
    if args.tpb:
        tun.tpb = args.tpb
    if args.sif:
        tun.sweeps_in_flight = args.sif
    ws = torch.empty(bb.band_to_bidiag_workspace_size(args.n, args.b, code, tun),
                     dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    out = []
    for _ in range(args.reps):
        k0, k1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for ev in (k0, k1):
            ev.record(stream)
        tun.ev_start, tun.ev_stop = k0.cuda_event, k1.cuda_event
        e0.record(stream)
        bb.band_to_bidiag_ex(band, args.b, d, e, tuning=tun, workspace=ws, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        out.append({"kernel_ms": k0.elapsed_time(k1), "call_ms": e0.elapsed_time(e1)})
    sig = None
    if args.sigma:
        s_out = torch.empty(args.n, device="cuda", dtype=torch.float64)
        sws = torch.empty(int(bb.lib().bb_bidiag_sigma_workspace_size(args.n)), dtype=torch.uint8,
                          device="cuda")
        bb.bb_bidiag_sigma(d, e, s_out, sws, stream=stream)          # warm-up
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        bb.bb_bidiag_sigma(d, e, s_out, sws, stream=stream)
        s1.record(stream)
        torch.cuda.synchronize()
        sig = {"sigma_ms": s0.elapsed_time(s1), "sigma_max": float(s_out[0]), "sigma_min": float(s_out[-1])}
    status = bb.bb_device_status(stream, reset=True)
    w = bb.bb_schedule_counts(args.n, args.b, tun.tw)
    print(json.dumps({"n": args.n, "b": args.b, "dtype": args.dtype, "tw": tun.tw, "tpb": tun.tpb,
                      "sweeps_in_flight": tun.sweeps_in_flight,
                      "status": status, "flops": w.flops, "row_bulges": w.steps, "runs": out,
                      "sigma": sig}))
    return 0 if status == 0 else 1


if __name__ == "__main__":
    sys.exit(main())

#!/usr/bin/env python3
"""Benchmark: band -> bidiagonal reduction at n = 32768, b = 128 on GB300.

One step = one full reduction of one synthetic band matrix (pack, every
bandwidth-reduction stage, extract) through the library's C ABI, with the band
already resident in HBM.  The plain FP64 form is the headline; the FP32 form
(FP32 storage and arithmetic, FP64 reflector generation) is timed beside it.
Between timed steps the L2 is flushed by writing a 256 MiB buffer, so every
step starts from HBM.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs one independent replica per GPU (the reduction of one matrix does
not shard); the JSON value is the aggregate over ranks.  --impl reference times
the CPU oracle on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N, B, SEED = 32768, 128, 2
METRIC = "band->bidiag effective GFLOP/s at n=32768, b=128 (FP64; FP32 form alongside)"
L2_FLUSH_BYTES = 256 << 20
ORACLE_SAMPLE_STEPS = 600_000        # row-bulges of the first stage (~10-30 s of CPU work)
REF_STEP_SAMPLE = 150_000            # per --impl reference step


def _peaks_file():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f)
    return None


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", f"bb_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def oracle_sample(n, b, tw, max_steps, seed=SEED):
    """Time the CPU oracle (as it stands) on the first `max_steps` row-bulges."""
    import bandgen
    import oracle
    ab = bandgen.random_band(n, b, seed=seed)
    oracle.build()
    t0 = time.perf_counter()
    _, _, cnt = oracle.band_to_bidiag(ab, b, tw, max_steps=max_steps)
    dt = time.perf_counter() - t0
    return cnt["flops"], dt, cnt["steps"]


def reference_tw(n: int, b: int) -> int:
    """TW of our arm's FP64 configuration without touching the GPU path: the
    committed tuner weights evaluated by the FP64 MLP oracle (the library's own
    pick runs the same network with its GPU kernels); 16 without a model."""
    from paper_2510_12705_gb300 import tuner
    if not os.path.exists(tuner.MODEL_PATH):
        return 16
    import oracle.mlp as omlp
    with open(tuner.MODEL_PATH) as f:
        m = json.load(f)
    cands = [tuple(c) for c in m["candidates"]]
    X = np.array([tuner.features(n, b, "f64", c) for c in cands])
    y, _, _ = omlp.forward(np.array(m["params"], np.float64), X, m["in_dim"], m["hidden"])
    return cands[int(np.argmin(y))][0]


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    n, b = args.n, args.b
    tw = reference_tw(n, b)
    ms, gf = [], []
    for i in range(args.warmup + args.steps):
        flops, dt, steps = oracle_sample(n, b, tw, REF_STEP_SAMPLE)
        if i >= args.warmup:
            ms.append(dt * 1e3)
            gf.append(flops / dt / 1e9)
    value = float(np.median(gf))
    sample = (f"first {REF_STEP_SAMPLE} row-bulges (stage 1, sweeps 0..~{REF_STEP_SAMPLE // (n // b)}) "
              f"of the n={n}, b={b}, TW={tw} FP64 reduction, single thread")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GFLOP/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": float(np.mean(ms)), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"band->bidiag n={n} b={b} FP64 TW={tw}, N(0,1) seed {SEED}",
                   "n": n, "b": b, "tw": tw, "sample": sample},
        "cpu_baseline": {"value": value, "unit": "GFLOP/s", "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# DRAM bytes (read + write) per launch of the bulge kernel, from one ncu capture
# of this workload (profiles/bulge_kernel_dram_n32768_b128.md), keyed by the
# launch configuration; None (reported as null) for any other configuration.
MEASURED_DRAM_BYTES_PER_LAUNCH = {
    ("bulge_kernel<double,33>", 32768, 128, 32, 0, 0): 440363008.0,
}


def maxm_for(tw: int) -> int:
    """Template size of the bulge kernel the library launches for this TW."""
    return 5 if tw <= 4 else 9 if tw <= 8 else 17 if tw <= 16 else 33


def pick_tuning(bb, torch, dev, n, b, dtype_code):
    """Hyperparameters for the timed reduction: the learned tuner's pick (one
    forward pass of the trained MLP on this GPU, outside the timed region), or
    the library default when no trained model is present."""
    from paper_2510_12705_gb300 import tuner
    return tuner.tuning_for(n, b, "f64" if dtype_code == bb.BB_F64 else "f32", dev)


def run_ours(args, rank, world):
    import torch
    import bandgen
    import paper_2510_12705_gb300 as bb
    from paper_2510_12705_gb300 import build as bbuild

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    bbuild.build()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", dev))

    n, b = args.n, args.b
    stream = torch.cuda.current_stream()
    ab = bandgen.random_band(n, b, seed=SEED)
    band64 = torch.from_numpy(ab).cuda()
    band32 = band64.float()
    d64 = torch.empty(n, dtype=torch.float64, device="cuda")
    e64 = torch.empty(n - 1, dtype=torch.float64, device="cuda")
    d32 = torch.empty(n, dtype=torch.float32, device="cuda")
    e32 = torch.empty(n - 1, dtype=torch.float32, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    t64, src64 = pick_tuning(bb, torch, dev, n, b, bb.BB_F64)
    t32, src32 = pick_tuning(bb, torch, dev, n, b, bb.BB_F32)
    work64 = bb.bb_schedule_counts(n, b, t64.tw)
    work32 = bb.bb_schedule_counts(n, b, t32.tw)

    def timed(band, d, e, tun, steps, warmup, work, bracket=False):
        """warmup untimed steps, then `steps` timed ones; every step starts
        after an L2 flush; per-step CUDA events around the call and around
        the bulge-chasing kernels (library-recorded)."""
        ws = torch.empty(bb.band_to_bidiag_workspace_size(n, b, bb._dtype_code(band.dtype), tun),
                         dtype=torch.uint8, device="cuda")
        for i in range(warmup):
            flush.fill_(i & 0xFF)
            bb.band_to_bidiag_ex(band, b, d, e, tuning=tun, workspace=ws, stream=stream)
        torch.cuda.synchronize()
        if bracket:
            if dist:
                dist.barrier()
            torch.cuda.synchronize()
            clocks.start()
        t0 = time.perf_counter()
        evs = []
        for i in range(steps):
            flush.fill_(i & 0xFF)              # evict the band and workspace from L2
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            k0 = torch.cuda.Event(enable_timing=True)
            k1 = torch.cuda.Event(enable_timing=True)
            for ev in (k0, k1):                 # materialise the raw handles
                ev.record(stream)
            tun.ev_start = k0.cuda_event
            tun.ev_stop = k1.cuda_event
            e0.record(stream)
            bb.band_to_bidiag_ex(band, b, d, e, tuning=tun, workspace=ws, stream=stream)
            e1.record(stream)
            evs.append((e0, e1, k0, k1))
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        clk = None
        if bracket:
            clk = clocks.stop()
            if dist:
                dist.barrier()
        tun.ev_start = None
        tun.ev_stop = None
        step_ms = [a.elapsed_time(z) for a, z, _, _ in evs]
        kern_ms = [a.elapsed_time(z) for _, _, a, z in evs]
        return step_ms, kern_ms, wall, clk

    # roofline denominators measured on this GPU
    peaks = _peaks_file() or {}
    fp64_peak = bb.bb_measure_fma_peak(bb.BB_F64)
    fp32_peak = bb.bb_measure_fma_peak(bb.BB_F32)
    l2_gbs = bb.bb_measure_l2_bandwidth(32 << 20, 200)

    # ---- timed region: K FP64 reductions (the headline), warm-up outside it
    clocks = ClockSampler(dev)
    step_ms, kern_ms, wall, clk = timed(band64, d64, e64, t64, args.steps, args.warmup, work64,
                                        bracket=True)
    status = bb.bb_device_status(stream, reset=True)

    ms_step = float(np.mean(step_ms))
    ms_kern = float(np.mean(kern_ms))
    if dist:
        t = torch.tensor([ms_step], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_step = float(t.item())
    gflops = world * work64.flops / (ms_step * 1e-3) / 1e9

    # ---- FP32 form (same workload)
    step32, kern32, _, _ = timed(band32, d32, e32, t32, args.steps, args.warmup, work32)
    ms32 = float(np.mean(step32))
    ms32_kern = float(np.mean(kern32))

    # ---- end to end through the host-buffer entry point (pinned host memory)
    hband = torch.from_numpy(ab).pin_memory()
    hd = torch.empty(n, dtype=torch.float64).pin_memory()
    he = torch.empty(n - 1, dtype=torch.float64).pin_memory()
    e2e_ms = []
    for i in range(max(1, args.warmup // 2) + args.steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rc = bb.band_to_bidiag_host_ptr(n, b, bb.BB_F64, hband.data_ptr(), hband.shape[1],
                                        hd.data_ptr(), he.data_ptr(), t64, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        if rc != 0:
            raise RuntimeError(f"band_to_bidiag_host failed: {bb.status_string(rc)}")
        if i >= max(1, args.warmup // 2):
            e2e_ms.append(e0.elapsed_time(e1))
    e2e = {"value": world * work64.flops / (float(np.mean(e2e_ms)) * 1e-3) / 1e9,
           "unit": "GFLOP/s", "ms_per_step": float(np.mean(e2e_ms)),
           "h2d_bytes_per_step": int(hband.numel() * 8),
           "d2h_bytes_per_step": int((hd.numel() + he.numel()) * 8)}

    # correctness guard on the timed output (cheap properties)
    dd = d64.cpu().numpy()
    ok = bool(dd[0] == ab[0, b]) and status == 0

    bytes64 = work64.bytes(8)
    bytes32 = work32.bytes(4)
    achieved_fp64 = work64.flops / (ms_kern * 1e-3) / 1e9          # GFLOP/s
    achieved_l2_64 = bytes64 / (ms_kern * 1e-3) / 1e9              # GB/s
    achieved_l2_32 = bytes32 / (ms32_kern * 1e-3) / 1e9
    roofline = {
        "bound": "alu", "kernel": f"bulge_kernel<double,{maxm_for(t64.tw)}>",
        "achieved": achieved_fp64 / 1e3, "peak": fp64_peak / 1e3, "unit": "TFLOP/s",
        "frac": achieved_fp64 / fp64_peak if fp64_peak > 0 else None,
        "peak_source": "measured FP64 FMA rate on this GPU (bb_measure_fma_peak)",
        "traffic": MEASURED_DRAM_BYTES_PER_LAUNCH.get(
            (f"bulge_kernel<double,{maxm_for(t64.tw)}>", n, b, t64.tw, t64.tpb, t64.sweeps_in_flight)),
        "traffic_unit": "DRAM bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)",
        "algorithmic_bytes_per_launch": bytes64 / max(work64.stages, 1),
        "l2": {"achieved": achieved_l2_64, "peak": l2_gbs, "unit": "GB/s",
               "frac": achieved_l2_64 / l2_gbs if l2_gbs > 0 else None,
               "peak_source": "measured L2-resident copy bandwidth (bb_measure_l2_bandwidth)"},
        "hbm_peak_gbs": peaks.get("hbm_gbs"),
    }
    fp32 = {
        "ms_per_step": ms32, "kernel_ms": ms32_kern,
        "gflops": work32.flops / (ms32 * 1e-3) / 1e9,
        "speedup_vs_fp64": ms_step / ms32,
        "tw": t32.tw, "tpb": t32.tpb, "sweeps_in_flight": t32.sweeps_in_flight, "tuning": src32,
        "roofline": {"bound": "l2", "achieved": achieved_l2_32, "peak": l2_gbs, "unit": "GB/s",
                     "frac": achieved_l2_32 / l2_gbs if l2_gbs > 0 else None,
                     "alu_frac": (work32.flops / (ms32_kern * 1e-3) / 1e9) / fp32_peak
                     if fp32_peak > 0 else None},
    }

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        flops, dt, steps = oracle_sample(n, b, t64.tw, ORACLE_SAMPLE_STEPS)
        cpu = {"value": flops / dt / 1e9, "unit": "GFLOP/s", "cores": 1, "kind": "oracle",
               "seconds": dt,
               "sample": f"first {steps} row-bulges of stage 1 of the same n={n}, b={b}, TW={t64.tw} "
                         "FP64 reduction (sequential sweep order), single-threaded C oracle"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": gflops, "unit": "GFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"band->bidiag n={n} b={b} FP64 TW={t64.tw}, iid N(0,1) band, seed {SEED}",
                       "n": n, "b": b, "tw": t64.tw, "tpb": t64.tpb,
                       "sweeps_in_flight": t64.sweeps_in_flight, "tuning": src64,
                       "stages": work64.stages, "row_bulges": work64.steps,
                       "flops_per_step": work64.flops, "algorithmic_bytes_per_step": bytes64,
                       "l2": "flushed between steps (256 MiB write)", "parallelism": "replicas"},
            "kernel_ms": ms_kern,
            "roofline": roofline,
            "fp32": fp32,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": clk,
            # pack + one persistent launch per stage + extract, per timed step
            "gpu_launches": (2 + work64.stages) * args.steps,
            "wall_s_timed_region": wall,
            "checks": {"device_status": status, "d0_exact": ok},
            "peaks_measured": {"fp64_gflops": fp64_peak, "fp32_gflops": fp32_peak, "l2_gbs": l2_gbs},
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=N)
    ap.add_argument("--b", type=int, default=B)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    return run_ours(args, rank, world)


if __name__ == "__main__":
    sys.exit(main())

#!/usr/bin/env python3
"""Benchmark: band -> bidiagonal reduction at n = 32768, b = 128 on GB300.

One step = one full reduction of one synthetic band matrix (pack, every
bandwidth-reduction stage, extract) through the library's C ABI, with the band
already resident in HBM.  The plain FP64 form is the headline; the FP32 form
(FP32 storage and arithmetic, FP64 reflector generation) is timed beside it.
Between timed steps the L2 is flushed by writing a 256 MiB buffer, so every
step starts from HBM.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
    python bench.py --profile-case --n 8192 --b 128 --dtype f64 [--tw 32 --group 8 --reps 2]

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


def oracle_sample_parallel(n, b, tw, max_steps, seed=SEED):
    """Time the OpenMP form of the oracle (the cycle schedule of Section III-A,
    the row-bulges of each cycle on all host cores) on the first cycles that
    hold `max_steps` row-bulges.  Returns (flops, seconds, steps, threads)."""
    import bandgen
    import oracle
    ab = bandgen.random_band(n, b, seed=seed)
    oracle.build_parallel()
    t0 = time.perf_counter()
    _, _, cnt, thr = oracle.band_to_bidiag_parallel(ab, b, tw, max_steps=max_steps)
    dt = time.perf_counter() - t0
    return cnt["flops"], dt, cnt["steps"], thr


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
    # one step of our arm is the whole reduction: the sample's time scaled to
    # the full schedule's flop count (the reduction's work model, host only)
    from paper_2510_12705_gb300 import build as bbuild
    bbuild.build()
    import paper_2510_12705_gb300 as bb
    full_flops = bb.bb_schedule_counts(n, b, tw).flops
    ms_full = full_flops / (value * 1e9) * 1e3
    sample = (f"first {REF_STEP_SAMPLE} row-bulges (stage 1, sweeps 0..~{REF_STEP_SAMPLE // (n // b)}) "
              f"of the n={n}, b={b}, TW={tw} FP64 reduction, single thread")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GFLOP/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_full, "ms_per_step_basis": "extrapolated: full-reduction flops / sampled rate",
        "sample_ms": float(np.mean(ms)), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"band->bidiag n={n} b={b} FP64 TW={tw}, N(0,1) seed {SEED}",
                   "n": n, "b": b, "tw": tw, "sample": sample},
        "cpu_baseline": {"value": value, "unit": "GFLOP/s", "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# DRAM bytes (read + write) per launch of a bulge-chasing kernel, from one ncu
# capture of this workload, keyed by a hash of the kernel sources the capture
# was taken with and by (kernel, n, b, tw, group); a changed kernel source or
# another configuration reports null.  Mean over the launches of that kernel
# in one reduction (ncu dram__bytes_read.sum + dram__bytes_write.sum).
_DRAM_085875e7 = {
    ("group_kernel<double,double,33>", 32768, 128, 32, 24): (51286016 + 14431488 + 47294976 + 23750912
                                                            + 39432192 + 16101888) / 3,
    ("bulge_kernel<double,double,33>", 32768, 128, 32, 24): 34132736 + 409594112,
}
MEASURED_DRAM_BYTES_PER_LAUNCH: dict = {
    "085875e7adeb6037": _DRAM_085875e7,
    # the same capture: this source differs from the one above only in the
    # back-transformation kernel of the singular vectors and its launcher,
    # which the reduction does not run; the captured kernels' code is identical
    "7c2b64bc09d69f4e": _DRAM_085875e7,
}


REDUCTION_SOURCES = ("band_bidiag.cu", "bb_device.cuh", "bb_group.cuh", "bb_team.cuh")


def kernel_source_hash() -> str:
    """Short hash of the CUDA code of the reduction's kernels (the singular
    value, tuning and peak-probe kernels are not part of it), with the
    comments and blank lines left out, so that a change of wording alone keeps
    a stored capture valid."""
    import hashlib
    import re
    h = hashlib.sha256()
    for name in REDUCTION_SOURCES:
        f = os.path.join(ROOT, "paper_2510_12705_gb300", "csrc", name)
        with open(f, encoding="utf-8") as fh:
            text = fh.read()
        code = [ln.rstrip() for ln in (re.sub(r"//.*", "", line) for line in text.splitlines())]
        h.update(os.path.basename(f).encode())
        h.update("\n".join(ln for ln in code if ln.strip()).encode())
    return h.hexdigest()[:16]


KERNEL_NAMES = {0: "group_kernel", 1: "team_kernel", 2: "bulge_kernel"}


class LaunchTimer:
    """CUDA events the library records around every bulge-chasing launch
    (bb_tuning.ev_launch), with the (stage, kernel) of each launch."""

    def __init__(self, torch, max_launches: int):
        import ctypes
        self.ctypes = ctypes
        self.evs = [torch.cuda.Event(enable_timing=True) for _ in range(2 * max_launches)]
        self.arr = (ctypes.c_void_p * len(self.evs))()
        self.log = (ctypes.c_int * max_launches)()

    def arm(self, tun, stream):
        for i, ev in enumerate(self.evs):
            ev.record(stream)                 # materialise the raw handles
            self.arr[i] = ev.cuda_event
        for i in range(len(self.log)):
            self.log[i] = -1
        tun.ev_launch = self.ctypes.cast(self.arr, self.ctypes.c_void_p)
        tun.ev_count = len(self.evs)
        tun.launch_log = self.ctypes.cast(self.log, self.ctypes.c_void_p)

    def disarm(self, tun):
        tun.ev_launch, tun.ev_count, tun.launch_log = None, 0, None

    def read(self):
        """[(stage, kernel id, ms)] of the launches of the last armed call."""
        out = []
        for i in range(len(self.log)):
            if self.log[i] < 0:
                break
            out.append((self.log[i] // 4, self.log[i] % 4, self.evs[2 * i].elapsed_time(self.evs[2 * i + 1])))
        return out


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
        after an L2 flush; per-step CUDA events around the call, around the
        bulge-chasing kernels and around each of their launches (all recorded
        by the library on `stream`)."""
        lt = LaunchTimer(torch, 3 * max(work.stages, 1) + 2)
        launches = []
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
            lt.arm(tun, stream)
            e0.record(stream)
            bb.band_to_bidiag_ex(band, b, d, e, tuning=tun, workspace=ws, stream=stream)
            e1.record(stream)
            evs.append((e0, e1, k0, k1))
            e1.synchronize()                   # read this step's launch events
            launches.append(lt.read())
        lt.disarm(tun)
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
        return step_ms, kern_ms, wall, clk, launches

    # roofline denominators measured on this GPU
    peaks = _peaks_file() or {}
    fp64_peak = bb.bb_measure_fma_peak(bb.BB_F64)
    fp32_peak = bb.bb_measure_fma_peak(bb.BB_F32)
    l2_gbs = bb.bb_measure_l2_bandwidth(32 << 20, 200)

    # ---- timed region: K FP64 reductions (the headline), warm-up outside it
    clocks = ClockSampler(dev)
    step_ms, kern_ms, wall, clk, launches64 = timed(band64, d64, e64, t64, args.steps, args.warmup,
                                                    work64, bracket=True)
    status = bb.bb_device_status(stream, reset=True)

    ms_step = float(np.mean(step_ms))
    ms_kern = float(np.mean(kern_ms))
    if dist:
        t = torch.tensor([ms_step], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_step = float(t.item())
    gflops = world * work64.flops / (ms_step * 1e-3) / 1e9

    # ---- FP32 form (same workload)
    step32, kern32, _, _, launches32 = timed(band32, d32, e32, t32, args.steps, args.warmup, work32)
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
    stage64 = [bb.bb_stage_counts(n, b, t64.tw, i) for i in range(work64.stages)]
    stage32 = [bb.bb_stage_counts(n, b, t32.tw, i) for i in range(work32.stages)]

    def per_kernel(launches, stages, esize):
        """Per kernel: launches per step, mean ms per step, and the work of
        the stages it ran (one problem: one kernel per stage)."""
        out = {}
        steps = max(len(launches), 1)
        for step in launches:
            for st, kid, ms in step:
                k = out.setdefault(KERNEL_NAMES.get(kid, str(kid)),
                                   {"launches": 0, "ms": 0.0, "flops": 0.0, "bytes": 0.0, "stages": set()})
                k["launches"] += 1
                k["ms"] += ms
                k["flops"] += stages[st].flops
                k["bytes"] += stages[st].bytes(esize)
                k["stages"].add(st)
        for k in out.values():
            k["launches_per_step"] = k.pop("launches") / steps
            for f in ("ms", "flops", "bytes"):
                k[f] /= steps
            k["stages"] = sorted(k["stages"])
        return out

    kern64 = per_kernel(launches64, stage64, 8)
    kern32 = per_kernel(launches32, stage32, 4)
    dom = max(kern64, key=lambda k: kern64[k]["ms"]) if kern64 else "bulge_kernel"
    dk = kern64.get(dom, {"ms": ms_kern, "flops": work64.flops, "bytes": bytes64, "launches_per_step": 1})
    dom_name = f"{dom}<double,double,{maxm_for(t64.tw)}>"
    achieved_fp64 = dk["flops"] / (dk["ms"] * 1e-3) / 1e9                  # GFLOP/s
    achieved_l2_64 = dk["bytes"] / (dk["ms"] * 1e-3) / 1e9                 # GB/s
    achieved_l2_32 = bytes32 / (ms32_kern * 1e-3) / 1e9
    src_hash = kernel_source_hash()
    traffic = MEASURED_DRAM_BYTES_PER_LAUNCH.get(src_hash, {}).get((dom_name, n, b, t64.tw, t64.group))
    roofline = {
        "bound": "alu", "kernel": dom_name,
        "achieved": achieved_fp64 / 1e3, "peak": fp64_peak / 1e3, "unit": "TFLOP/s",
        "frac": achieved_fp64 / fp64_peak if fp64_peak > 0 else None,
        "traffic": traffic,
        "peak_source": "measured FP64 FMA rate on this GPU (bb_measure_fma_peak)",
        "achieved_basis": "algorithmic flops of the stages this kernel ran / its launch time, "
                          "CUDA events around each launch",
        "kernel_share": dk["ms"] / ms_kern if ms_kern > 0 else None,
        "traffic_unit": "DRAM bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)",
        "traffic_source": f"stored ncu capture for kernel sources {src_hash}" if traffic else
                          "no ncu capture of the current kernel sources",
        "algorithmic_bytes_per_launch": dk["bytes"] / max(dk["launches_per_step"], 1e-9),
        "l2": {"achieved": achieved_l2_64, "peak": l2_gbs, "unit": "GB/s",
               "frac": achieved_l2_64 / l2_gbs if l2_gbs > 0 else None,
               "peak_source": "measured L2-resident copy bandwidth (bb_measure_l2_bandwidth)"},
        "whole_reduction": {"tflops": work64.flops / (ms_kern * 1e-3) / 1e12,
                            "frac": (work64.flops / (ms_kern * 1e-3) / 1e9) / fp64_peak if fp64_peak > 0 else None},
        "kernels": {k: {f: v[f] for f in ("ms", "launches_per_step", "stages", "flops")} for k, v in kern64.items()},
        "hbm_peak_gbs": peaks.get("hbm_gbs"),
    }
    fp32 = {
        "ms_per_step": ms32, "kernel_ms": ms32_kern,
        "gflops": work32.flops / (ms32 * 1e-3) / 1e9,
        "speedup_vs_fp64": ms_step / ms32,
        "tw": t32.tw, "tpb": t32.tpb, "sweeps_in_flight": t32.sweeps_in_flight, "tuning": src32,
        "kernels": {k: {f: v[f] for f in ("ms", "launches_per_step", "stages")} for k, v in kern32.items()},
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
    cpu_par = None
    if rank == 0 and not args.no_cpu_baseline:
        try:
            flops, dt, steps, thr = oracle_sample_parallel(n, b, t64.tw, ORACLE_SAMPLE_STEPS)
            cpu_par = {"value": flops / dt / 1e9, "unit": "GFLOP/s", "cores": thr, "kind": "oracle-openmp",
                       "seconds": dt,
                       "sample": f"first cycles of stage 1 holding {steps} row-bulges of the same n={n}, "
                                 f"b={b}, TW={t64.tw} FP64 reduction, cycle schedule (lag 2) with each "
                                 f"cycle's row-bulges on {thr} OpenMP threads; bitwise the oracle's result"}
        except Exception as exc:                       # never costs the bench line
            cpu_par = {"unavailable": f"OpenMP oracle failed: {type(exc).__name__}: {exc}"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": gflops, "unit": "GFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"band->bidiag n={n} b={b} FP64 TW={t64.tw}, iid N(0,1) band, seed {SEED}",
                       "n": n, "b": b, "tw": t64.tw, "tpb": t64.tpb,
                       "sweeps_in_flight": t64.sweeps_in_flight, "group": t64.group, "teams": t64.teams,
                       "tuning": src64,
                       "stages": work64.stages, "row_bulges": work64.steps,
                       "flops_per_step": work64.flops, "algorithmic_bytes_per_step": bytes64,
                       "l2": "flushed between steps (256 MiB write)", "parallelism": "replicas"},
            "kernel_ms": ms_kern,
            "roofline": roofline,
            "fp32": fp32,
            "cpu_baseline": cpu,
            "cpu_baseline_parallel": cpu_par,
            "e2e": e2e,
            "clocks": clk,
            # pack + the bulge-chasing launches + extract, per timed step
            "gpu_launches": int(round((2 + sum(v["launches_per_step"] for v in kern64.values())) * args.steps)),
            "wall_s_timed_region": wall,
            "checks": {"device_status": status, "d0_exact": ok},
            "peaks_measured": {"fp64_gflops": fp64_peak, "fp32_gflops": fp32_peak, "l2_gbs": l2_gbs},
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def profile_case(args):
    """One configuration, reduced `reps` times (no L2 flush, no clocks): the
    command the ncu summaries are taken with.  Prints one JSON line with the
    kernel time of each repetition and its launches."""
    import torch
    import bandgen
    import paper_2510_12705_gb300 as bb
    from paper_2510_12705_gb300 import build as bbuild
    bbuild.build()
    dt = torch.float64 if args.dtype == "f64" else torch.float32
    code = bb.BB_F64 if args.dtype == "f64" else bb.BB_F32
    n, b = args.n, args.b
    band = torch.from_numpy(bandgen.random_band(n, b, seed=args.seed)).to("cuda", dt)
    d = torch.empty(n, device="cuda", dtype=dt)
    e = torch.empty(max(n - 1, 1), device="cuda", dtype=dt)
    if args.tuned:
        from paper_2510_12705_gb300 import tuner
        tun, _ = tuner.tuning_for(n, b, args.dtype)
    else:
        tun = bb.bb_default_tuning(n, b, code)
    for f in ("tw", "tpb", "group", "teams"):
        if getattr(args, f):
            setattr(tun, f, getattr(args, f))
    if args.sif:
        tun.sweeps_in_flight = args.sif
    ws = torch.empty(bb.band_to_bidiag_workspace_size(n, b, code, tun), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    work = bb.bb_schedule_counts(n, b, tun.tw)
    lt = LaunchTimer(torch, 3 * max(work.stages, 1) + 2)
    runs = []
    for _ in range(args.reps):
        k0, k1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for ev in (k0, k1):
            ev.record(stream)
        tun.ev_start, tun.ev_stop = k0.cuda_event, k1.cuda_event
        lt.arm(tun, stream)
        bb.band_to_bidiag_ex(band, b, d, e, tuning=tun, workspace=ws, stream=stream)
        torch.cuda.synchronize()
        runs.append({"kernel_ms": k0.elapsed_time(k1),
                     "launches": [[st, KERNEL_NAMES.get(k, str(k)), round(ms, 3)] for st, k, ms in lt.read()]})
    sig = None
    if args.sigma:
        s_out = torch.empty(n, device="cuda", dtype=torch.float64)
        sws = torch.empty(int(bb.lib().bb_bidiag_sigma_workspace_size(n)), dtype=torch.uint8,
                          device="cuda")
        bb.bb_bidiag_sigma(d, e, s_out, sws, stream=stream)          # warm-up
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        bb.bb_bidiag_sigma(d, e, s_out, sws, stream=stream)
        s1.record(stream)
        torch.cuda.synchronize()
        sig = {"sigma_ms": s0.elapsed_time(s1), "sigma_max": float(s_out[0]),
               "sigma_min": float(s_out[-1])}
    status = bb.bb_device_status(stream, reset=True)
    print(json.dumps({"n": n, "b": b, "dtype": args.dtype, "tw": tun.tw, "group": tun.group,
                      "teams": tun.teams, "tpb": tun.tpb, "sweeps_in_flight": tun.sweeps_in_flight,
                      "status": status, "flops": work.flops, "row_bulges": work.steps, "runs": runs,
                      "sigma": sig}))
    return 0 if status == 0 else 1


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=N)
    ap.add_argument("--b", type=int, default=B)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-case", action="store_true",
                    help="reduce one configuration --reps times and print its kernel times")
    ap.add_argument("--dtype", choices=["f64", "f32"], default="f64")
    ap.add_argument("--tw", type=int, default=0)
    ap.add_argument("--tpb", type=int, default=0)
    ap.add_argument("--group", type=int, default=0)
    ap.add_argument("--teams", type=int, default=0)
    ap.add_argument("--sif", type=int, default=0)
    ap.add_argument("--reps", type=int, default=1)
    ap.add_argument("--seed", type=int, default=SEED)
    ap.add_argument("--tuned", action="store_true", help="profile case: the trained tuner's choice")
    ap.add_argument("--sigma", action="store_true", help="profile case: also time the GPU sigma")
    args = ap.parse_args()
    if args.profile_case:
        return profile_case(args)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    return run_ours(args, rank, world)


if __name__ == "__main__":
    sys.exit(main())

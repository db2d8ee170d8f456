"""Hyperparameter tuning for the band -> bidiagonal reduction.

The knobs (Section III-C): the inner tilewidth TW, the number of sweeps
processed concurrently ("max blocks": CTAs per SM) and, for the group kernel,
the number of sweeps one CTA chases together (the max-blocks unrolled into one
block).  The CTA size follows the panel size.

* Exhaustive autotuner: ``autotune(n, b, dtype)`` times every candidate on a
  synthetic band of that size through the native ``bb_autotune`` (Section IV
  uses the same brute force over a few values per knob).
* Learned tuner: ``MlpTuner`` is a small MLP trained on timings the method
  itself generates (``collect``), mapping (log n, log b, dtype, candidate) to
  log(time); ``predict`` returns the candidate with the smallest predicted
  time.  Training runs on the GPU with the library's forward, backward and
  Adam kernels (``bb_mlp_*``); nothing of the MLP runs on the host except the
  argument marshalling.

CLI:
    python -m paper_2510_12705_gb300.tuner collect  --out data.json
    python -m paper_2510_12705_gb300.tuner train    --data data.json --out model.json
    python -m paper_2510_12705_gb300.tuner evaluate --model model.json --n 65536 --b 256 --dtype f32
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

TWS = (16, 24, 32)         # TW = 8 (also in the paper's search) never won on GB300
GROUPS = (8, 24)           # sweeps per CTA of the group kernel (at most; fewer where 3K + d > bw)
SIFS = (0, 1)              # 0: the library's choice of resident CTAs; 1: one CTA per SM on every stage
IN_DIM = 8
HIDDEN = 32


def candidates():
    return [(tw, g, sif) for tw in TWS for g in GROUPS for sif in SIFS]


def features(n: int, b: int, dtype: str, cand) -> list[float]:
    tw, g, sif = cand
    ln, lb = math.log2(max(n, 2)), math.log2(max(b, 1))
    return [(ln - 13.0) / 3.0, (lb - 6.0) / 2.0, 1.0 if dtype == "f64" else -1.0,
            (math.log2(tw) - 4.5), (math.log2(g) - 4.0), 1.0 if sif else -1.0,
            (ln - lb - 7.0) / 3.0, (lb - math.log2(tw) - 2.0) / 2.0]


def _tuning(cand, nsm: int):
    import paper_2510_12705_gb300 as bb
    tw, g, sif = cand
    return bb.Tuning(tw=tw, group=g, sweeps_in_flight=(nsm if sif else 0))


def usable(n: int, b: int, dtype: str, cand) -> bool:
    """The candidate's shared-memory panels fit the current device."""
    import torch

    import paper_2510_12705_gb300 as bb
    need = bb.bb_shared_bytes(n, b, bb.BB_F64 if dtype == "f64" else bb.BB_F32,
                              _tuning(cand, 1))
    limit = torch.cuda.get_device_properties(0).shared_memory_per_block_optin
    return 0 < need <= limit


def autotune(n: int, b: int, dtype: str, reps: int = 1, seed: int = 0, cands=None):
    """Time every candidate on a synthetic N(0,1) band of size (n, b) through the
    native exhaustive search; returns (times_ms, best_index)."""
    import torch

    import bandgen
    import paper_2510_12705_gb300 as bb
    cands = cands or candidates()
    dt = torch.float64 if dtype == "f64" else torch.float32
    band = torch.from_numpy(bandgen.random_band(n, b, seed=seed)).to("cuda", dt)
    d = torch.empty(n, device="cuda", dtype=dt)
    e = torch.empty(max(n - 1, 1), device="cuda", dtype=dt)
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    return bb.bb_autotune(band, b, d, e, [_tuning(c, nsm) for c in cands], reps=reps)


def collect(grid, reps: int = 1, log=None, out=None):
    """Timing dataset over (n, b, dtype) triples: one row per candidate the
    problem supports (unsupported candidates time as +inf and are left out).
    With ``out`` the rows so far are rewritten to that JSON file after every
    problem."""
    rows = []
    for (n, b, dtype) in grid:
        times, best = autotune(n, b, dtype, reps=reps)
        for c, t in zip(candidates(), times):
            if math.isfinite(t):
                rows.append({"n": n, "b": b, "dtype": dtype, "cand": list(c), "ms": t})
        if log:
            log(f"n={n} b={b} {dtype}: best {candidates()[best]} {min(times):.1f} ms; "
                + " ".join(f"{t:.1f}" for t in times))
        if out:
            with open(out, "w") as f:
                json.dump(rows, f)
    return rows


HELD_OUT = (65536, 256, "f32")
DEFAULT_GROUP = 24         # the library's default sweeps per CTA (group = 0)


def default_grid(n_max: int = 32768, max_nb: int = 1 << 22):
    """Training grid: n = 1024, 2048, ... n_max; b in {16, 32, ..., 256} with
    b <= n/4 and n*b <= max_nb (the cost of one reduction grows like n*b);
    FP32 and FP64.  The held-out problem n = 65536, b = 256, FP32 is never
    part of it (it lies outside the grid)."""
    grid = []
    n = 1024
    while n <= n_max:
        for b in (16, 32, 64, 128, 256):
            if b <= n // 4 and n * b <= max_nb:
                for dtype in ("f32", "f64"):
                    grid.append((n, b, dtype))
        n *= 2
    return [g for g in grid if g != HELD_OUT]


class MlpTuner:
    """MLP regression of log(ms) on the features of (problem, candidate)."""

    def __init__(self, hidden: int = HIDDEN, seed: int = 0):
        import numpy as np

        import paper_2510_12705_gb300 as bb
        self.hidden = hidden
        self.P = bb.bb_mlp_param_count(IN_DIM, hidden)
        rng = np.random.default_rng(seed)
        D, H = IN_DIM, hidden
        # He-style initialisation, zero biases
        parts = [rng.standard_normal(H * D) * math.sqrt(2.0 / D), np.zeros(H),
                 rng.standard_normal(H * H) * math.sqrt(2.0 / H), np.zeros(H),
                 rng.standard_normal(H) * math.sqrt(1.0 / H), np.zeros(1)]
        self.params = np.concatenate(parts).astype(np.float32)
        assert self.params.size == self.P
        self.mean = 0.0

    def forward(self, X):
        """Network output for feature rows X (FP32 CUDA tensor [N][IN_DIM])."""
        import torch

        import paper_2510_12705_gb300 as bb
        N = X.shape[0]
        P = torch.from_numpy(self.params).cuda()
        Y = torch.empty(N, device="cuda")
        H1 = torch.empty(N, self.hidden, device="cuda")
        H2 = torch.empty(N, self.hidden, device="cuda")
        bb.bb_mlp_forward(IN_DIM, self.hidden, P, X, Y, H1, H2)
        return Y

    @staticmethod
    def dataset(rows):
        import numpy as np
        X = np.array([features(r["n"], r["b"], r["dtype"], r["cand"]) for r in rows], np.float32)
        T = np.log(np.array([r["ms"] for r in rows], np.float64))
        return X, T

    def train(self, rows, epochs: int = 4000, lr: float = 3e-3, log=None):
        """Full-batch Adam on the library's GPU kernels; returns the final
        training mean squared error of log(ms)."""
        import numpy as np
        import torch

        import paper_2510_12705_gb300 as bb
        X, T = self.dataset(rows)
        self.mean = float(T.mean())
        Xd = torch.from_numpy(X).cuda()
        Td = torch.from_numpy((T - self.mean).astype(np.float32)).cuda()
        N, H = X.shape[0], self.hidden
        P = torch.from_numpy(self.params).cuda()
        G, M, V = torch.zeros_like(P), torch.zeros_like(P), torch.zeros_like(P)
        S = torch.empty(bb.bb_mlp_backward_scratch(H, N), device="cuda")
        Y = torch.empty(N, device="cuda")
        H1 = torch.empty(N, H, device="cuda")
        H2 = torch.empty(N, H, device="cuda")
        for step in range(1, epochs + 1):
            bb.bb_mlp_forward(IN_DIM, H, P, Xd, Y, H1, H2)
            bb.bb_mlp_backward(IN_DIM, H, P, Xd, H1, H2, Y, Td, G, S)
            bb.bb_mlp_adam(P, G, M, V, step, lr)
            if log and step % 1000 == 0:
                log(f"step {step}: mse(log ms) {float(((Y - Td) ** 2).mean()):.4f}")
        bb.bb_mlp_forward(IN_DIM, H, P, Xd, Y, H1, H2)
        self.params = P.cpu().numpy()
        return float(((Y - Td) ** 2).mean())

    def predict_ms(self, n, b, dtype):
        import numpy as np
        import torch
        X = torch.from_numpy(np.array([features(n, b, dtype, c) for c in candidates()],
                                      np.float32)).cuda()
        return [math.exp(float(y) + self.mean) for y in self.forward(X).cpu().numpy()]

    def predict(self, n, b, dtype):
        """Candidate (tw, group, sif) with the smallest predicted time among those
        the problem can use on this device."""
        t = self.predict_ms(n, b, dtype)
        ok = [i for i, c in enumerate(candidates()) if usable(n, b, dtype, c)]
        return candidates()[min(ok, key=t.__getitem__)]

    def save(self, path):
        with open(path, "w") as f:
            json.dump({"hidden": self.hidden, "in_dim": IN_DIM, "mean": self.mean,
                       "candidates": candidates(),
                       "params": [float(x) for x in self.params]}, f)

    @classmethod
    def load(cls, path):
        import numpy as np
        with open(path) as f:
            d = json.load(f)
        if d["in_dim"] != IN_DIM or [tuple(c) for c in d["candidates"]] != candidates():
            raise ValueError(f"{path}: model was trained for another feature set")
        t = cls(hidden=d["hidden"])
        t.params = np.array(d["params"], np.float32)
        t.mean = d["mean"]
        return t


def evaluate(tuner: "MlpTuner", n: int, b: int, dtype: str, reps: int = 1) -> dict:
    """Regret of the MLP's pick against the exhaustive search, and its gain over
    the library's fixed default tuning, both timed by the exhaustive search."""
    import paper_2510_12705_gb300 as bb
    cands = candidates()
    pick = tuple(tuner.predict(n, b, dtype))
    times, best = autotune(n, b, dtype, reps=reps)
    dflt = bb.bb_default_tuning(n, b, bb.BB_F64 if dtype == "f64" else bb.BB_F32)
    dflt_c = (dflt.tw, DEFAULT_GROUP, 0)
    out = {"n": n, "b": b, "dtype": dtype,
           "exhaustive_best": list(cands[best]), "exhaustive_ms": times[best],
           "mlp_pick": list(pick), "mlp_ms": times[cands.index(pick)],
           "default": list(dflt_c), "default_ms": times[cands.index(dflt_c)],
           "mean_candidate_ms": sum(t for t in times if math.isfinite(t))
                                / sum(1 for t in times if math.isfinite(t)),
           "exhaustive_runs": len(cands), "mlp_runs": 0,
           "all_ms": {str(list(c)): t for c, t in zip(cands, times)}}
    out["mlp_regret"] = out["mlp_ms"] / out["exhaustive_ms"] - 1.0
    out["gain_over_default"] = out["default_ms"] / out["mlp_ms"]
    return out


MODEL_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuner_model.json")


def tuning_for(n: int, b: int, dtype: str, device: int = 0):
    """(Tuning, source) for a problem: the trained tuner's pick (one MLP
    forward launch on the GPU) when the packaged model exists, else the
    library default."""
    import torch

    import paper_2510_12705_gb300 as bb
    code = bb.BB_F64 if dtype == "f64" else bb.BB_F32
    t = bb.bb_default_tuning(n, b, code)
    if not os.path.exists(MODEL_PATH):
        return t, "library default"
    tw, g, sif = MlpTuner.load(MODEL_PATH).predict(n, b, dtype)
    nsm = torch.cuda.get_device_properties(device).multi_processor_count
    return bb.Tuning(tw=tw, group=g, sweeps_in_flight=nsm if sif else 0,
                     timeout_s=t.timeout_s), "learned tuner"


def main(argv=None):
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="cmd", required=True)
    c = sub.add_parser("collect")
    c.add_argument("--out", required=True)
    c.add_argument("--reps", type=int, default=1)
    c.add_argument("--n-max", type=int, default=32768)
    t = sub.add_parser("train")
    t.add_argument("--data", required=True)
    t.add_argument("--out", required=True)
    t.add_argument("--epochs", type=int, default=4000)
    e = sub.add_parser("evaluate")
    e.add_argument("--model", required=True)
    e.add_argument("--n", type=int, default=65536)
    e.add_argument("--b", type=int, default=256)
    e.add_argument("--dtype", default="f32")
    args = ap.parse_args(argv)
    from paper_2510_12705_gb300 import build
    build.build()
    log = lambda m: print(m, file=sys.stderr, flush=True)   # noqa: E731
    if args.cmd == "collect":
        collect(default_grid(n_max=args.n_max), reps=args.reps, log=log, out=args.out)
    elif args.cmd == "train":
        with open(args.data) as f:
            rows = json.load(f)
        tun = MlpTuner()
        loss = tun.train(rows, epochs=args.epochs, log=log)
        tun.save(args.out)
        print(json.dumps({"train_mse_log_ms": loss, "samples": len(rows)}))
    else:
        print(json.dumps(evaluate(MlpTuner.load(args.model), args.n, args.b, args.dtype)))
    return 0


if __name__ == "__main__":
    sys.exit(main())

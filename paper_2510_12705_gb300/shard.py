"""Splitting a batch of independent band problems across ranks.

The reduction of one matrix does not shard (its sweeps are a lag-2 pipeline
over a band that fits one GPU's L2), but the problems of a batch are
independent.  Each rank reduces its own share with one batch plan on its own
GPU; no collective touches the data path.  The host gathers d and e at the end
when every rank needs all results.

    parts = partition([(n, b), ...], world)          # list of index lists
    mine  = run_local(problems, parts[rank], dtype)  # this rank's (d, e) pairs
    full  = gather(mine, parts, group)               # every rank: all (d, e)
"""
from __future__ import annotations

import math


def stages(b: int, tw: int) -> int:
    """Number of bandwidth-reduction stages from b down to 1 (Section III:
    each stage removes min(TW, bw - 1) superdiagonals)."""
    s, bw = 0, b
    while bw > 1:
        bw -= min(tw, bw - 1)
        s += 1
    return s


def cost(n: int, b: int, tw: int = 32) -> float:
    """Relative cost of one problem: a stage is a chain of about 2 n row-bulges,
    each one a latency-bound step whose length grows slowly with the panel
    size, so the time is proportional to n x stages x (a mild panel term)."""
    b = min(b, max(n - 1, 0))
    return float(n) * max(stages(b, tw), 1) * (1.0 + math.log2(1 + min(b, tw)) / 8.0)


def partition(problems, world: int, tw: int = 32) -> list[list[int]]:
    """Greedy longest-processing-time assignment of problems (n, b) to `world`
    ranks: problems in decreasing cost order, each to the least-loaded rank
    (ties to the lowest rank).  Returns, per rank, the sorted problem indices."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(problems)), key=lambda i: (-cost(*problems[i][:2], tw=tw), i))
    load = [0.0] * world
    parts: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(i)
        load[r] += cost(*problems[i][:2], tw=tw)
    return [sorted(p) for p in parts]


def run_local(problems, indices, dtype="f32", stream=None):
    """Reduce this rank's problems with one batch plan on the current GPU.
    ``problems``: list of (band ndarray (n, ldab), b); returns {index: (d, e)}
    as host numpy arrays."""
    import torch

    import paper_2510_12705_gb300 as bb
    if not indices:
        return {}
    dt = torch.float32 if dtype == "f32" else torch.float64
    items = []
    for i in indices:
        ab, b = problems[i]
        band = torch.from_numpy(ab).to("cuda", dt)
        n = ab.shape[0]
        items.append((band, b, torch.empty(n, device="cuda", dtype=dt),
                      torch.empty(max(n - 1, 1), device="cuda", dtype=dt)))
    plan = bb.BatchPlan(items)
    ws = torch.empty(plan.workspace_bytes, dtype=torch.uint8, device="cuda")
    plan.execute(ws, stream=stream)
    status = bb.bb_device_status(stream, reset=True)
    if status:
        raise bb.BBError(bb.BB_ERR_TIMEOUT if status & (1 << bb.BB_ERR_TIMEOUT)
                         else bb.BB_ERR_NONFINITE, "batched reduction")
    out = {}
    for i, (band, b, d, e) in zip(indices, items):
        n = band.shape[0]
        out[i] = (d.cpu().numpy(), e[: n - 1].cpu().numpy())
    return out


def gather(local: dict, parts, group=None) -> dict:
    """Host gather over torch.distributed (any backend that carries Python
    objects, e.g. gloo): every rank receives every problem's (d, e)."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    boxes = [None] * world
    dist.all_gather_object(boxes, local, group=group)
    full = {}
    for r, box in enumerate(boxes):
        if set(box) != set(parts[r]):
            raise RuntimeError(f"rank {r} returned problems {sorted(box)}, expected {parts[r]}")
        full.update(box)
    return full

"""Multi-rank batch path on the CPU: the partition is a balanced exact cover,
and two gloo ranks that each reduce their share (here with the oracle standing
in for the GPU reduction) gather exactly the single-process results."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import bandgen
from paper_2510_12705_gb300 import shard


def test_stages_count():
    assert shard.stages(1, 32) == 0 and shard.stages(0, 16) == 0
    assert shard.stages(128, 16) == 8      # 128 -> 112 -> ... -> 16 -> 1
    assert shard.stages(128, 32) == 4      # 128 -> 96 -> 64 -> 32 -> 1
    assert shard.stages(130, 32) == 5      # 130 -> 98 -> 66 -> 34 -> 2 -> 1
    assert shard.stages(2, 32) == 1


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_partition_is_balanced_exact_cover(world):
    probs = [(n, b) for (n, b, _) in bandgen.batch_problems(200, seed=3)]
    parts = shard.partition(probs, world)
    assert len(parts) == world
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(len(probs)))
    loads = [sum(shard.cost(*probs[i]) for i in p) for p in parts]
    biggest = max(shard.cost(*p) for p in probs)
    # greedy LPT: no rank exceeds the mean by more than one problem's cost
    assert max(loads) - sum(loads) / world <= biggest + 1e-9


def test_partition_more_ranks_than_problems():
    parts = shard.partition([(100, 4), (50, 2)], 4)
    assert sorted(len(p) for p in parts) == [0, 0, 1, 1]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, problems, out_dir):
    import torch.distributed as dist

    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    parts = shard.partition([(ab.shape[0], b) for ab, b in problems], world)
    # stand-in for the GPU batch on this CPU-only rank
    local = {}
    for i in parts[rank]:
        ab, b = problems[i]
        d, e, _ = oracle.band_to_bidiag(ab, b, 8)
        local[i] = (d, e)
    full = shard.gather(local, parts)
    np.save(os.path.join(out_dir, f"rank{rank}.npy"),
            np.array([np.concatenate([full[i][0], full[i][1]]) for i in range(len(problems))],
                     dtype=object), allow_pickle=True)
    dist.destroy_process_group()


def test_two_gloo_ranks_gather_all_results(tmp_path):
    import oracle
    specs = [(60, 5, 1), (33, 8, 2), (90, 3, 3), (17, 16, 4), (48, 6, 5)]
    problems = [(bandgen.random_band(n, b, seed=s), b) for n, b, s in specs]
    mp.start_processes(_rank_main, args=(2, _free_port(), problems, str(tmp_path)), nprocs=2,
                       join=True, start_method="spawn")
    ref = [np.concatenate(oracle.band_to_bidiag(ab, b, 8)[:2]) for ab, b in problems]
    for r in range(2):
        got = np.load(tmp_path / f"rank{r}.npy", allow_pickle=True)
        for i in range(len(problems)):
            assert np.array_equal(got[i], ref[i])

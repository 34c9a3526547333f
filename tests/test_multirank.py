"""Multi-rank host logic on CPU: two gloo ranks share a batch of requests.

The device work of each rank is stood in for by the FP64 oracle (this test
checks the partition, the gather and the max-over-ranks timing, not the
kernel); the gathered profiles must equal a one-process run bit for bit.
"""
import os
import socket

import numpy as np
import pytest

from paper_2410_08267_gb300 import sharding as S
from paper_2410_08267_gb300 import workloads as W


def _problems():
    out = []
    for pb in W.random_small(31, n=7):
        out.append(pb.replace(n_q=min(pb.n_q, 8), n_mu=min(pb.n_mu, 4), n_steps=60))
    return out


def test_partition_covers_every_item_once_and_balances():
    rng = np.random.default_rng(5)
    w = rng.integers(1, 1000, size=101).astype(float)
    for world in (1, 2, 3, 8):
        parts = S.partition(w, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(w)))
        loads = [w[p].sum() for p in parts]
        # greedy LPT: the spread between ranks never exceeds the largest item
        assert max(loads) - min(loads) <= w.max()
    assert S.partition([], 3) == [[], [], []]
    assert S.partition([5.0], 4) == [[0], [], [], []]


def test_partition_of_equal_copies_gives_equal_work():
    one = W.precision_sweep()
    job = one * 4
    for world in (2, 4):
        parts = S.partition_problems(job, world)
        loads = {sum(job[i].traj_steps for i in p) for p in parts}
        assert len(loads) == 1 and all(len(p) == len(job) // world for p in parts)


def test_partition_rejects_bad_input():
    with pytest.raises(ValueError):
        S.partition([1.0], 0)
    with pytest.raises(ValueError):
        S.partition([1.0, -2.0], 2)


def test_gather_without_group_checks_coverage():
    a = {0: np.ones(2), 1: np.zeros(3)}
    got = S.gather_profiles(a, 2)
    assert got[0].tolist() == [1.0, 1.0] and got[1].tolist() == [0.0, 0.0, 0.0]
    with pytest.raises(ValueError):
        S.gather_profiles({0: np.ones(1)}, 2)
    assert S.max_over_ranks(3.5) == 3.5


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    import oracle

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        problems = _problems()
        mine = S.partition_problems(problems, world)[rank]
        local = {i: oracle.profile(problems[i], n_threads=1) for i in mine}
        gathered = S.gather_profiles(local, len(problems), dist)
        slowest = S.max_over_ranks(10.0 + rank, dist)
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), mine=np.array(mine),
                 slowest=slowest, **{f"p{i}": v for i, v in enumerate(gathered)})
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_match_one_process(tmp_path):
    import torch.multiprocessing as mp
    import oracle

    oracle.lib()                       # build/load the oracle before the ranks start
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    problems = _problems()
    serial = [oracle.profile(pb, n_threads=1) for pb in problems]
    ranks = [np.load(tmp_path / f"rank{r}.npz") for r in range(world)]
    assert sorted(np.concatenate([d["mine"] for d in ranks]).tolist()) == list(range(len(problems)))
    assert all(len(d["mine"]) > 0 for d in ranks)
    for d in ranks:
        assert float(d["slowest"]) == 10.0 + world - 1
        for i, ref in enumerate(serial):
            np.testing.assert_array_equal(d[f"p{i}"], ref)

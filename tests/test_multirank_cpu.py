"""Host logic of the multi-GPU runs on CPU ranks (gloo, world size 2): the
max-over-ranks timing and the sum of work that bench.py reports, and the
longest-first split of an ensemble over ranks."""
import os
import socket
import sys

import numpy as np
import pytest

from paper_2309_10534_gb300 import gks as G
from paper_2309_10534_gb300 import workloads as WL


def test_partition_lpt_covers_every_problem_once_and_balances():
    E = WL.ensemble_1d()
    cost = E.ncells.astype(np.float64) ** 2
    for parts in (1, 2, 3, 8):
        shards = G.partition_lpt(cost, parts)
        allidx = np.sort(np.concatenate(shards))
        assert np.array_equal(allidx, np.arange(E.ncells.size))
        loads = np.array([cost[s].sum() for s in shards])
        # LPT bound: the heaviest rank carries at most the mean plus one problem
        assert loads.max() <= loads.mean() + cost.max()
        assert loads.max() / loads.min() < 1.01
    assert [s.tolist() for s in G.partition_lpt(cost, 4)] == [s.tolist() for s in G.partition_lpt(cost, 4)]


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    mx = G.reduce_scalars([10.0 * (rank + 1), -rank], "max", dist)
    sm = G.reduce_scalars([rank + 1.0], "sum", dist)
    E = WL.ensemble_1d(count=64, seed=3, nmin=20, nmax=100)
    shard = G.partition_lpt(E.ncells.astype(np.float64) ** 2, world)[rank]
    shards = [None] * world
    dist.all_gather_object(shards, shard.tolist())
    dist.barrier()
    dist.destroy_process_group()
    np.save(os.path.join(out_dir, "r%d.npy" % rank), np.array(mx + sm + [len(sum(shards, []))] +
                                                             sorted(sum(shards, [])), dtype=np.float64))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_reduce_and_shard(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    port = _free_port()
    mp.spawn(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    for r in range(2):
        v = np.load(tmp_path / ("r%d.npy" % r))
        assert v[0] == 20.0 and v[1] == 0.0          # max over ranks
        assert v[2] == 3.0                           # sum over ranks
        assert v[3] == 64 and np.array_equal(v[4:], np.arange(64))  # shards: every problem once

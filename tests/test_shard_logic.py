"""Host logic of root-range sharding (no GPU): the partition of the rank
space and the sum-reduce of partial counts, with gloo ranks on CPU.

The per-range counts come from the CPU oracle's root-restricted mode here
(the GPU path uses vdmc_count_roots, checked in the GPU tests); by Lemma 1
the ranges' counts must add up to the full count exactly.
"""
import os
import socket

import numpy as np
import pytest

from oracle import oracle as O
from paper_2201_11655_b300 import synth
from paper_2201_11655_b300.shard import partition_costs, reduce_partial

torch = pytest.importorskip("torch")


def test_partition_costs_properties():
    rng = np.random.default_rng(0)
    for trial in range(50):
        n = int(rng.integers(1, 400))
        parts = int(rng.integers(1, 9))
        costs = (rng.pareto(1.2, n) * 100).astype(np.uint64)
        b = partition_costs(costs, parts)
        assert len(b) == parts + 1 and b[0] == 0 and b[-1] == n
        assert all(b[i] <= b[i + 1] for i in range(parts))
        total = int(costs.sum())
        cmax = int(costs.max())
        for i in range(parts):
            assert int(costs[b[i]:b[i + 1]].sum()) <= total / parts + cmax + 1
        assert b == partition_costs(costs, parts)  # deterministic


def test_partition_costs_edge_cases():
    assert partition_costs(np.zeros(0, np.uint64), 3) == [0, 0, 0, 0]
    assert partition_costs(np.zeros(10, np.uint64), 2) == [0, 5, 10]
    # one root holds all the work: it goes to the first range, the rest get nothing to do
    c = np.array([1000, 0, 0, 0], np.uint64)
    b = partition_costs(c, 4)
    assert b[0] == 0 and b[1] == 1 and b[-1] == 4
    with pytest.raises(ValueError):
        partition_costs(c, 0)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, k, result_path):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        n, s, d = synth.chung_lu(400, 3.0, 2.3, 17, reciprocity=0.2)
        rank_of = O.degree_rank(n, s, d)
        # cost per rank: a degree-based estimate (any non-negative weights give a valid split)
        deg = np.zeros(n, np.int64)
        np.add.at(deg, s, 1)
        np.add.at(deg, d, 1)
        costs = np.zeros(n, np.uint64)
        costs[rank_of] = (deg ** 3).astype(np.uint64)
        bounds = partition_costs(costs, world)
        part, _ = O.count_roots(n, s, d, k, rank_of, bounds[rank], bounds[rank + 1], threads=2)
        t = torch.from_numpy(part.view(np.int64).copy())
        reduce_partial(t, dist)
        if rank == 0:
            np.save(result_path, t.numpy())
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,k", [(2, 3), (2, 4), (3, 4)])
def test_gloo_ranks_sum_to_full_count(tmp_path, world, k):
    import torch.multiprocessing as mp
    path = str(tmp_path / "sum.npy")
    mp.start_processes(_rank_main, args=(world, _free_port(), k, path), nprocs=world, start_method="spawn")
    got = np.load(path).view(np.uint64)
    n, s, d = synth.chung_lu(400, 3.0, 2.3, 17, reciprocity=0.2)
    want, _ = O.count(n, s, d, k)
    np.testing.assert_array_equal(got, want)

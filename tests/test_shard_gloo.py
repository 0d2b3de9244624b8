"""The multi-process split of one system (CPU, gloo, two ranks).

Each rank takes a cost-balanced contiguous range of the batches, integrates
its partial H over the full pattern and its own points' density with the
FP64 oracle, and one sum over ranks must give the single-process H and
electron count.  The partition itself is checked for coverage, order and
balance on its own."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle as O
import workloads as W
from paper_2208_12335_gb300 import shard as S


def test_partition_covers_each_batch_once_in_order():
    rng = np.random.default_rng(5)
    for n, world in [(1, 1), (7, 2), (40, 3), (100, 8), (3, 5), (0, 2)]:
        cost = rng.uniform(1.0, 50.0, size=n)
        parts = S.partition_by_cost(cost, world)
        assert len(parts) == world
        allids = np.concatenate(parts) if n else np.zeros(0, np.int64)
        assert np.array_equal(allids, np.arange(n))          # every batch once, in order
        if n:
            share = cost.sum() / world
            for p in parts:
                assert cost[p].sum() <= share + cost.max() + 1e-9
    # equal costs split evenly
    parts = S.partition_by_cost(np.ones(12), 4)
    assert [len(p) for p in parts] == [3, 3, 3, 3]
    with pytest.raises(ValueError):
        S.partition_by_cost(np.array([1.0, -1.0]), 2)
    with pytest.raises(ValueError):
        S.partition_by_cost(np.ones(3), 0)


def test_batch_cost_is_points_times_functions_squared():
    assert np.allclose(S.batch_cost([10, 20], [3, 4]), [90.0, 320.0])
    assert S.batch_cost([0], [0])[0] == 1.0


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2208_12335_gb300 import build as Bld
        Bld.build()
        import paper_2208_12335_gb300 as P
        prob = W.tiny_water(n_rad=16, n_ang=26)
        ctx = P.Context(-1).load(prob, "fp64")            # host-only plan: batch work, no GPU
        pts, nfn = ctx.batch_work()
        parts = S.partition_by_cost(S.batch_cost(pts, nfn), world)
        mine = prob.subgrid(parts[rank])
        B = O.system_basis(prob)
        h = torch.from_numpy(O.h_matrix(B, mine.pts, mine.w, mine.v))
        S.allreduce_sum(h)
        rng = W.rng_for(0, W.PURPOSE_D)
        D = W.random_symmetric(B.n_fn, rng, 0.3)
        n_mine = O.density(B, mine.pts, D)
        nel = torch.tensor([float(np.sum(mine.w * n_mine))], dtype=torch.float64)
        S.allreduce_sum(nel)
        if rank == 0:
            np.save(os.path.join(out, "h.npy"), h.numpy())
            np.save(os.path.join(out, "nel.npy"), nel.numpy())
            np.save(os.path.join(out, "n_batches.npy"), np.array([len(p) for p in parts]))
    finally:
        dist.destroy_process_group()


def test_two_ranks_sum_to_the_single_process_result(tmp_path):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    prob = W.tiny_water(n_rad=16, n_ang=26)
    B = O.system_basis(prob)
    H = O.h_matrix(B, prob.pts, prob.w, prob.v)
    h = np.load(tmp_path / "h.npy")
    assert np.max(np.abs(h - H)) <= 1e-13 * np.abs(H).max()
    rng = W.rng_for(0, W.PURPOSE_D)
    D = W.random_symmetric(B.n_fn, rng, 0.3)
    nel_ref = float(np.sum(prob.w * O.density(B, prob.pts, D)))
    assert np.load(tmp_path / "nel.npy")[0] == pytest.approx(nel_ref, rel=1e-12, abs=1e-14)
    nb = np.load(tmp_path / "n_batches.npy")
    assert nb.sum() == prob.n_batch and np.all(nb > 0)

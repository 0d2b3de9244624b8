"""The split of one system over processes, with the library on one GPU.

Each "rank" takes a cost-balanced contiguous range of the batches
(shard.partition_by_cost on the library's own per-batch work), plans its
sub-grid in a context of its own and integrates H over the full sparsity
pattern (which depends on the atoms only) and the density of its own
points.  The ranks run one after the other on the one GPU, as independent
processes would on their own GPUs: no kernel waits on another rank.  The sum
of the partial H over ranks must equal the single-context H, each rank's
density must equal the single-context density on its points, and the
per-rank electron counts must add up.  The sum over ranks is the one
collective a multi-GPU run needs (shard.allreduce_sum)."""
import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fgi():
    from paper_2208_12335_gb300 import build as B
    B.build()
    import paper_2208_12335_gb300 as P
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return P


@pytest.fixture(scope="module")
def cluster():
    # 60 C/H/N/O atoms, coarse grids, uneven batches
    return W.chno_cluster(n_atoms=60, n_rad=24, n_ang=74, p_max=300, p_min=50, workload_index=7)


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda:0")


@pytest.mark.parametrize("precision,tol_h,tol_n", [("fp64", 1e-12, 1e-12), ("split_bf16", 2e-7, 2e-7)])
@pytest.mark.parametrize("world", [2, 3])
def test_ranks_of_one_system_add_up(fgi, cluster, precision, tol_h, tol_n, world):
    from paper_2208_12335_gb300 import shard
    prob = cluster
    full = fgi.Context(0).load(prob, precision)
    n_fn, nnz, n_pts, _ = full.sizes()
    rowptr, col = full.pattern(0)
    rows = np.repeat(np.arange(len(rowptr) - 1), np.diff(rowptr))
    D, _ = W.density_matrix_occ(n_fn, max(1, int(round(0.28 * n_fn))), np.random.default_rng(21))
    dvals = dev(D[rows, col])
    h_full = full.integrate_h(dev(prob.v)).cpu().numpy()
    n_full, tr_full = full.density(dvals)
    full.sync()
    n_full, tr_full = n_full.cpu().numpy(), float(tr_full.cpu().numpy()[0])
    pts, nfn = full.batch_work()
    full.close()

    parts = shard.partition_by_cost(shard.batch_cost(pts, nfn), world)
    assert np.array_equal(np.concatenate(parts), np.arange(prob.n_batch))
    h_sum = np.zeros(nnz)
    tr_sum = 0.0
    for ids in parts:
        if len(ids) == 0:
            continue
        sub = prob.subgrid(ids)
        ctx = fgi.Context(0).load(sub, precision)
        rp, cl = ctx.pattern(0)
        assert np.array_equal(rp, rowptr) and np.array_equal(cl, col)     # the full pattern
        h_sum += ctx.integrate_h(dev(sub.v)).cpu().numpy()
        n_r, tr_r = ctx.density(dvals)
        ctx.sync()
        tr_sum += float(tr_r.cpu().numpy()[0])
        own = np.concatenate([np.arange(prob.batch_off[b], prob.batch_off[b + 1]) for b in ids])
        ref = n_full[own]
        rel = np.linalg.norm(n_r.cpu().numpy() - ref) / np.linalg.norm(ref)
        assert rel <= tol_n, (precision, rel)
        ctx.close()
    scale = max(1.0, np.abs(h_full).max()) if precision == "fp64" else 1.0
    assert np.max(np.abs(h_sum - h_full)) <= tol_h * scale
    assert tr_sum == pytest.approx(tr_full, rel=tol_n, abs=0.0)

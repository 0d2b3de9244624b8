"""GPU parity of the split path for every setting of the leading-digit
grids (tune-file key bound_grids): 0 an FP32 pass over the points for the
H and the density images, 1 table bounds of |phi| for the density images
only, 2 (the default) table bounds for both: H and density against the
FP64 oracle on water, a Si64 sub-grid and a sample of the 1000-atom
C/H/N/O cluster, at the split tolerances.  Marked slow (collected last)."""
import functools

import numpy as np
import pytest
import torch

import oracle as O
import workloads as W

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

TOL_SPLIT_H = 1e-7
TOL_SPLIT_N = 1e-7


@pytest.fixture(scope="module")
def fgi():
    from paper_2208_12335_gb300 import build as B
    B.build()
    import paper_2208_12335_gb300 as P
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return P


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda:0")


@functools.lru_cache(maxsize=None)
def problem(name):
    if name == "water":
        return W.tiny_water()
    if name == "si64":
        full = W.si64()
        ids = np.sort(np.random.default_rng(123).choice(full.n_batch, size=24, replace=False))
        return full.subgrid(ids)
    full = W.chno_cluster(atoms_with_grid=[0, 1])
    ids = np.sort(np.random.default_rng(5).choice(full.n_batch, size=24, replace=False))
    return full.subgrid(ids)


def on_pattern(ctx, n_fn, act, M):
    rowptr, col = ctx.pattern(0)
    r = np.repeat(np.arange(len(rowptr) - 1), np.diff(rowptr))
    pos = -np.ones(n_fn, dtype=np.int64)
    pos[act] = np.arange(len(act))
    inside = (pos[r] >= 0) & (pos[col] >= 0)
    out = np.zeros(len(r))
    out[inside] = M[pos[r[inside]], pos[col[inside]]]
    return out


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("name", ["water", "si64", "chno"])
def test_table_bound_grids_keep_split_parity(fgi, tmp_path, name, mode):
    prob = problem(name)
    B = O.system_basis(prob)
    act = O.active_functions(B, prob.pts)
    H = O.h_matrix(B, prob.pts, prob.w, prob.v, sub=act)
    D, _ = W.density_matrix_occ(len(act), max(1, int(0.28 * len(act))), np.random.default_rng(1))
    nref = O.density(B, prob.pts, D, sub=act)
    settings = tmp_path / "bound.txt"
    settings.write_text("bound_grids %d\n" % mode)
    ctx = fgi.Context(0).load(prob, "split_bf16", tune_path=str(settings))
    h = ctx.integrate_h(dev(prob.v)).cpu().numpy()
    n, _ = ctx.density(dev(on_pattern(ctx, B.n_fn, act, D)))
    ctx.sync()
    err_h = np.max(np.abs(h - on_pattern(ctx, B.n_fn, act, H)))
    rel_n = np.linalg.norm(n.cpu().numpy() - nref) / np.linalg.norm(nref)
    assert err_h <= TOL_SPLIT_H, (name, mode, err_h)
    assert rel_n <= TOL_SPLIT_N, (name, mode, rel_n)

"""Parity on the full 1000-atom C/H/N/O cluster (all 1000 atoms' grids,
~40 M points, one plan), in the launch configuration the benchmark times.

The oracle computes sampled outputs one by one: H entries (diagonal and
random stored entries) over every grid point within both functions'
cutoffs (the others contribute exactly zero), and the density at every
point of a dozen seeded batches, with D = 2 C_occ C_occ^T drawn as the
benchmark draws it.  A property that holds at any size (split BF16 within
the stated tolerance of the FP64 GPU path on every stored entry and every
point) covers the rest.  The Hartree potential of a seeded synthetic
density (owner-centred Gaussians with point-to-point noise) is checked at
seeded sample points against the oracle (multipoles of every atom).  Marked
slow: the FP64 path alone takes most of a minute on this cluster, the
oracle's Hartree multipoles a few minutes.
"""
import numpy as np
import pytest
import torch

import oracle as O
import oracle.hartree as OH
import workloads as W

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

TOL_SPLIT_H = 1e-7       # max |dH_ij|, Ha
TOL_SPLIT_N = 1e-7       # density relative L2


@pytest.fixture(scope="module")
def chno_full():
    from paper_2208_12335_gb300 import build as B
    B.build()
    import paper_2208_12335_gb300 as P
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    prob = W.chno_cluster(accel="cuda")
    ctx = P.Context(0).load(prob, "fp64")
    n_fn, nnz, n_pts, _ = ctx.sizes()
    rowptr, col = ctx.pattern(0)
    rows = np.repeat(np.arange(len(rowptr) - 1), np.diff(rowptr))
    v = torch.from_numpy(prob.v).cuda()
    h64 = ctx.integrate_h(v).cpu().numpy()
    ctx.set_precision("split_bf16")
    hs = ctx.integrate_h(v).cpu().numpy()
    n_occ = max(1, int(round(0.28 * n_fn)))
    q = W.occupied_orbitals(n_fn, n_occ, W.rng_for(1, W.PURPOSE_D))
    d = torch.from_numpy(W.density_values_occ(n_fn, n_occ, rows, col, None, q=q, accel="cuda:0")).cuda()
    ns = ctx.density(d)[0].cpu().numpy()
    ctx.set_precision("fp64")
    n64 = ctx.density(d)[0].cpu().numpy()
    # Hartree input: Z exp(-1.1 d^2) of the owning atom, times 1 + 0.3 u (seeded)
    Z = np.array([prob.species[int(s)].Z for s in prob.atom_species], dtype=np.float64)
    dist2 = np.sum((prob.pts - prob.atom_xyz[prob.owner]) ** 2, axis=1)
    n_h = Z[prob.owner] * np.exp(-1.1 * dist2) * (1.0 + 0.3 * np.random.default_rng(43).random(prob.n_pts))
    vh = ctx.hartree(torch.from_numpy(n_h).cuda(), l_max=4).cpu().numpy()
    ctx.sync()
    ctx.close()
    return dict(prob=prob, rows=rows, col=col, h64=h64, hs=hs, ns=ns, n64=n64, q=q, n_h=n_h, vh=vh)


def test_full_h_sampled_entries_against_oracle(chno_full):
    f = chno_full
    prob = f["prob"]
    B = O.system_basis(prob)
    cut = B.fn_cut()
    rng = np.random.default_rng(41)
    diag = np.nonzero(f["rows"] == f["col"])[0]
    k = np.concatenate([rng.choice(diag, 24, replace=False), rng.choice(len(f["rows"]), 24, replace=False)])
    pts = torch.from_numpy(prob.pts).cuda()
    ref = np.empty(len(k))
    for q, kk in enumerate(k):
        i, j = int(f["rows"][kk]), int(f["col"][kk])
        near = torch.ones(len(prob.pts), dtype=torch.bool, device="cuda")
        for fn in (i, j):
            a = torch.from_numpy(B.atom_xyz[B.fn_atom[fn]]).cuda()
            near &= torch.linalg.norm(pts - a, dim=1) < cut[fn] * (1 + 1e-12)
        idx = torch.nonzero(near).flatten().cpu().numpy()
        ref[q] = O.h_pairs(B, prob.pts[idx], prob.w[idx], prob.v[idx], [i], [j])[0]
    assert np.max(np.abs(f["h64"][k] - ref)) <= 1e-11 * np.abs(ref).max()
    assert np.max(np.abs(f["hs"][k] - ref)) <= TOL_SPLIT_H


def test_full_density_sampled_batches_against_oracle(chno_full):
    f = chno_full
    prob = f["prob"]
    B = O.system_basis(prob)
    ids = np.sort(np.random.default_rng(42).choice(prob.n_batch, 12, replace=False))
    idx = np.concatenate([np.arange(prob.batch_off[b], prob.batch_off[b + 1]) for b in ids])
    act = O.active_functions(B, prob.pts[idx])
    qa = f["q"][act]
    ref = O.density(B, prob.pts[idx], 2.0 * (qa @ qa.T), sub=act)
    for n, tol in ((f["n64"], 1e-12), (f["ns"], TOL_SPLIT_N)):
        assert np.linalg.norm(n[idx] - ref) / np.linalg.norm(ref) <= tol


def test_full_split_within_tolerance_on_every_entry(chno_full):
    f = chno_full
    assert np.max(np.abs(f["hs"] - f["h64"])) <= TOL_SPLIT_H
    assert np.linalg.norm(f["ns"] - f["n64"]) / np.linalg.norm(f["n64"]) <= TOL_SPLIT_N


def test_full_hartree_sampled_points_against_oracle(chno_full):
    """Tolerance as in test_gpu_hartree: 1e-10 of max |v_H| plus 2^-18 of
    the per-point scale of the FP32 l >= 1 terms."""
    f = chno_full
    idx = np.sort(np.random.default_rng(44).choice(f["prob"].n_pts, 200, replace=False))
    ref, bound = OH.hartree(f["prob"], f["n_h"], l_max=4, pts_idx=idx, l1_bound=True)
    err = np.abs(f["vh"][idx] - ref)
    assert np.all(err <= 1e-10 * np.abs(ref).max() + 2.0 ** -18 * bound), float(err.max())

"""GPU parity for the adjoint on Si64 (against the FP64 oracle gradient and
central finite differences of the GPU forward), for many independent
molecules in one plan, and for CUDA-graph replay of the split path."""
import numpy as np
import pytest
import torch

import oracle as O
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


def rows_cols(ctx, s=0):
    rowptr, col = ctx.pattern(s)
    return np.repeat(np.arange(len(rowptr) - 1), np.diff(rowptr)), col


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda:0")


@pytest.fixture(scope="module")
def si64_adj():
    full = W.si64()
    ids = np.sort(np.random.default_rng(77).choice(full.n_batch, size=16, replace=False))
    return full.subgrid(ids)


@pytest.mark.parametrize("precision", ["fp64", "split_bf16"])
def test_adjoint_si64_against_oracle_and_finite_differences(fgi, si64_adj, precision):
    """dL/dv and dL/dR of L = sum_k g_k h_k on a Si64 sub-grid: the FP64 path
    and the tensor-core path of a split context, against the oracle gradient
    and central differences of the FP64 forward."""
    prob = si64_adj
    ctx = fgi.Context(0).load(prob, precision)
    r, c = rows_cols(ctx)
    g = W.rng_for(3, W.PURPOSE_G).standard_normal(len(r))
    dv, dR = ctx.adjoint(dev(g), dev(prob.v))
    ctx.sync()
    dv, dR = dv.cpu().numpy(), dR.cpu().numpy()
    B = O.system_basis(prob)
    G = np.zeros((B.n_fn, B.n_fn))
    G[r, c] = np.where(r == c, g, 0.5 * g)
    G[c, r] = np.where(r == c, g, 0.5 * g)
    sub = O.active_functions(B, prob.pts)
    dv_ref, dR_ref = O.adjoint(B, prob.pts, prob.w, prob.v, G[np.ix_(sub, sub)], sub=sub)
    # split: dv = w n_G is a density of the random symmetric G, whose values
    # change sign; its error, ~2^-27 of sum_ij |G_ij phi_i phi_j| per point,
    # is a few 1e-7 of max |dv| (FP32 basis gradients and E give dR ~1e-7)
    tol_dv, tol_dR = (1e-11, 1e-10) if precision == "fp64" else (1e-6, 1e-6)
    np.testing.assert_allclose(dv, dv_ref, rtol=0, atol=tol_dv * np.abs(dv_ref).max())
    np.testing.assert_allclose(dR, dR_ref, rtol=0, atol=tol_dR * np.abs(dR_ref).max())

    # central differences of L(R) = sum_k g_k h_k(R), step 1e-4 Angstrom,
    # grid and potential held fixed
    step = 1e-4 * W.BOHR_PER_ANG
    v = dev(prob.v)

    def L(xyz):
        cx = fgi.Context(0)
        rid = [cx.add_radial(rr.l, rr.h, rr.coef) for rr in prob.radials]
        for sp in prob.species:
            cx.add_species(sp.Z, [rid[k] for k in sp.radial_ids])
        cx.set_systems(prob.atom_off, prob.atom_species, xyz)
        cx.set_grid(prob.pts, prob.w, prob.batch_off, prob.batch_sys)
        cx.plan("fp64")
        r2, c2 = rows_cols(cx)
        assert np.array_equal(r2, r) and np.array_equal(c2, c)
        h = cx.integrate_h(v).cpu().numpy()
        cx.sync()
        return float(np.dot(g, h))

    big = np.argsort(-np.linalg.norm(dR, axis=1))[:3]
    for a in big:
        for x in range(3):
            xp, xm = prob.atom_xyz.copy(), prob.atom_xyz.copy()
            xp[a, x] += step
            xm[a, x] -= step
            fd = (L(xp) - L(xm)) / (2 * step)
            assert dR[a, x] == pytest.approx(fd, rel=1e-5, abs=1e-6 * np.abs(dR).max())


@pytest.mark.parametrize("precision,tol_h,tol_n", [("fp64", 1e-11, 1e-12), ("split_bf16", 1e-7, 1e-7)])
def test_many_molecules_in_one_plan(fgi, precision, tol_h, tol_n):
    """Five molecules in one plan and one call each for H and the density,
    every molecule against the oracle on its own points: H entries, the
    density (D = 2 C_occ C_occ^T per molecule) and the electron count
    sum_p w_p n_p of each system."""
    prob = W.many_molecules(n_mol=5, n_at_range=(3, 6), nrad_range=(16, 20), nang_choices=(50, 74))
    ctx = fgi.Context(0).load(prob, precision)
    h = ctx.integrate_h(dev(prob.v)).cpu().numpy()
    rng = np.random.default_rng(4)
    d_all = np.zeros(ctx.sizes()[1])
    Ds = []
    for s in range(prob.n_sys):
        fn0, nf, val0, nnz = ctx.system(s)
        D, _ = W.density_matrix_occ(nf, max(1, int(round(0.28 * nf))), rng)
        r, c = rows_cols(ctx, s)
        d_all[val0:val0 + nnz] = D[r, c]
        Ds.append(D)
    n, tr = ctx.density(dev(d_all))
    ctx.sync()
    n, tr = n.cpu().numpy(), tr.cpu().numpy()
    for s in range(prob.n_sys):
        fn0, nf, val0, nnz = ctx.system(s)
        pts = prob.system_points(s)
        B = O.system_basis(prob, s)
        H = O.h_matrix(B, prob.pts[pts], prob.w[pts], prob.v[pts])
        r, c = rows_cols(ctx, s)
        assert np.max(np.abs(h[val0:val0 + nnz] - H[r, c])) <= tol_h * max(1.0, np.abs(H).max())
        nref = O.density(B, prob.pts[pts], Ds[s])
        assert np.linalg.norm(n[pts] - nref) / np.linalg.norm(nref) <= tol_n
        # n >= 0 here, so the electron count has no cancellation: the same
        # relative bound holds for it
        tr_ref = float(np.sum(prob.w[pts] * nref))
        assert tr[s] == pytest.approx(tr_ref, rel=tol_n, abs=0.0)


def test_split_step_replays_as_a_cuda_graph(fgi):
    prob = W.tiny_water()
    ctx = fgi.Context(0).load(prob, "split_bf16")
    B = O.system_basis(prob)
    r, c = rows_cols(ctx)
    D = W.random_symmetric(B.n_fn, np.random.default_rng(6), 0.3)
    v, d = dev(prob.v), dev(D[r, c])
    nnz, n_pts = ctx.sizes()[1], ctx.sizes()[2]
    h = torch.empty(nnz, dtype=torch.float64, device="cuda:0")
    n = torch.empty(n_pts, dtype=torch.float64, device="cuda:0")
    tr = torch.empty(1, dtype=torch.float64, device="cuda:0")
    ws = ctx.workspace()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ctx.integrate_h(v, h, ws=ws, stream=s)
        ctx.density(d, n, tr, ws=ws, stream=s)
    torch.cuda.synchronize()
    h_eager, n_eager = h.clone(), n.clone()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        ctx.integrate_h(v, h, ws=ws, stream=s)
        ctx.density(d, n, tr, ws=ws, stream=s)
    h.fill_(float("nan"))
    n.fill_(float("nan"))
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(h, h_eager)                      # fixed-point H: bitwise
    assert torch.allclose(n, n_eager, rtol=0, atol=1e-14)


def test_autotuner_writes_settings_that_plan_and_keep_parity(fgi, tmp_path):
    from paper_2208_12335_gb300 import tune as T
    prob = W.tiny_water()
    path = str(tmp_path / "tuned.txt")
    cands = [{"density_sb_points": 0}, {"density_sb_points": 1024, "density_sb_growth": 1.35}]
    res = T.tune(prob, path, candidates=cands, steps=2)
    assert res["best"] in cands and len(res["ms"]) == 2 and all(ms > 0 for ms in res["ms"].values())
    B = O.system_basis(prob)
    H = O.h_matrix(B, prob.pts, prob.w, prob.v)
    ctx = fgi.Context(0).load(prob, "split_bf16", tune_path=path)
    h = ctx.integrate_h(dev(prob.v)).cpu().numpy()
    ctx.sync()
    r, c = rows_cols(ctx)
    assert np.max(np.abs(h - H[r, c])) <= 1e-7


def test_many_small_waves_give_the_same_results(fgi, tmp_path):
    """A wave size of 8 MiB splits the Si64 sub-grid into many waves (the
    operand images of one wave at a time); H (fixed-point sums) and the
    density (per-point sums in block order) must come out bitwise the same
    as with one wave."""
    full = W.si64()
    ids = np.sort(np.random.default_rng(5).choice(full.n_batch, size=48, replace=False))
    prob = full.subgrid(ids)
    small = tmp_path / "small_waves.txt"
    small.write_text("wave_mb 8\n")
    out = []
    for path in (None, str(small)):
        ctx = fgi.Context(0).load(prob, "split_bf16", tune_path=path)
        nnz = ctx.sizes()[1]
        d = dev(np.random.default_rng(8).standard_normal(nnz) * 0.05)
        h = ctx.integrate_h(dev(prob.v)).clone()
        n, _ = ctx.density(d)
        ctx.sync()
        out.append((h.cpu(), n.clone().cpu(), ctx.workspace_size()))
    assert out[1][2] < out[0][2]                      # smaller waves, smaller workspace
    assert torch.equal(out[0][0], out[1][0])
    assert torch.equal(out[0][1], out[1][1])

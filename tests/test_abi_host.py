"""Host-side tests of the C ABI (no GPU): exported symbols, argument and
state errors, the sparsity pattern, and plan tables of host-only contexts."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def fgi():
    from paper_2208_12335_gb300 import build as B
    B.build()
    import paper_2208_12335_gb300 as P
    return P


def header_symbols():
    txt = open(os.path.join(ROOT, "include", "fgi.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(fgi_[a-z_0-9]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol(fgi):
    lib = C.CDLL(fgi.LIB_PATH)
    names = header_symbols()
    assert len(names) >= 18
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(fgi.SYMBOLS) == sorted(n for n in names if n in fgi.SYMBOLS)
    assert set(fgi.SYMBOLS) <= set(names)


def host_ctx(fgi, prob, precision="fp64"):
    ctx = fgi.Context.__new__(fgi.Context)
    ctx._lib = fgi.lib()
    ctx._h = C.c_void_p()
    ctx.device = -1
    ctx._keep = []
    ctx._ws = None
    rc = ctx._lib.fgi_create(C.byref(ctx._h), -1)
    assert rc == 0
    return ctx.load(prob, precision)


@pytest.fixture(scope="module")
def water():
    return W.tiny_water(n_rad=16, n_ang=26)


def test_host_only_plan_sizes_and_pattern(fgi, water):
    ctx = host_ctx(fgi, water)
    n_fn, nnz, n_pts, n_at = ctx.sizes()
    assert (n_fn, n_pts, n_at) == (7, water.n_pts, 3)
    # all three atoms are within each other's cutoffs: dense upper triangle
    assert nnz == 7 * 8 // 2
    rowptr, col = ctx.pattern(0)
    for i in range(7):
        assert list(col[rowptr[i]:rowptr[i + 1]]) == list(range(i, 7))
    assert ctx.workspace_size() > 0


def _pattern_reference(prob, s=0):
    """Stored pairs from the definition: atoms closer than the sum of their
    largest cutoffs (upper triangle, row-major, columns ascending)."""
    a0, a1 = prob.atom_off[s], prob.atom_off[s + 1]
    sp = prob.atom_species[a0:a1]
    xyz = prob.atom_xyz[a0:a1]
    rc = np.array([max(prob.radials[r].r_cut for r in prob.species[k].radial_ids) for k in sp])
    nf = np.array(prob.fns_per_species())[sp]
    fn0 = np.concatenate([[0], np.cumsum(nf)])
    owner = np.repeat(np.arange(len(sp)), nf)
    d = np.linalg.norm(xyz[:, None] - xyz[None], axis=2)
    near = d < rc[:, None] + rc[None, :]
    rows = []
    for i in range(fn0[-1]):
        a = owner[i]
        cols = [j for j in range(i, fn0[-1]) if near[a, owner[j]] or owner[j] == a]
        rows.append(cols)
    return rows


def test_pattern_matches_definition_on_a_sparse_cluster(fgi):
    prob = W.chno_cluster(n_atoms=60, n_rad=8, n_ang=14, atoms_with_grid=[0, 1, 2])
    ctx = host_ctx(fgi, prob)
    rowptr, col = ctx.pattern(0)
    ref = _pattern_reference(prob)
    assert len(rowptr) == len(ref) + 1
    assert rowptr[-1] < len(ref) * (len(ref) + 1) // 2      # genuinely sparse
    for i, cols in enumerate(ref):
        assert list(col[rowptr[i]:rowptr[i + 1]]) == cols


def test_many_systems_layout(fgi):
    parts = [W.tiny_water(n_rad=8, n_ang=14), W.tiny_water(n_rad=10, n_ang=14)]
    prob = W.merge_problems("two", parts, 0)
    ctx = host_ctx(fgi, prob)
    assert ctx.system(0) == (0, 7, 0, 28)
    assert ctx.system(1) == (7, 7, 28, 28)
    assert ctx.sizes()[:2] == (14, 56)


def test_argument_and_state_errors(fgi, water):
    lib = fgi.lib()
    h = C.c_void_p()
    assert lib.fgi_create(C.byref(h), -1) == 0
    try:
        # compute before plan
        assert lib.fgi_integrate_h(h, None, None, 0, None, 0, None) == -2
        # l out of range
        coef = np.zeros((3, 4))
        rid = C.c_int()
        assert lib.fgi_add_radial(h, 4, 0.1, 4, coef.ctypes.data_as(C.c_void_p), C.byref(rid)) == -7
        assert b"l = 4" in lib.fgi_last_error(h)
        # non-finite coefficients
        coef[1, 2] = np.nan
        assert lib.fgi_add_radial(h, 0, 0.1, 4, coef.ctypes.data_as(C.c_void_p), C.byref(rid)) == -6
        # NULL coefficients, bad knot count
        assert lib.fgi_add_radial(h, 0, 0.1, 4, None, C.byref(rid)) == -1
        assert lib.fgi_add_radial(h, 0, 0.1, 1, coef.ctypes.data_as(C.c_void_p), C.byref(rid)) == -1
        # species with an unknown radial
        ids = np.array([5], dtype=np.int32)
        assert lib.fgi_add_species(h, 1.0, 1, ids.ctypes.data_as(C.c_void_p), C.byref(rid)) == -1
        # plan without inputs
        assert lib.fgi_plan(h, 0, None) == -2
    finally:
        lib.fgi_destroy(h)


def test_grid_errors(fgi, water):
    ctx = host_ctx(fgi, water)
    big = np.zeros((1100, 3))
    with pytest.raises(fgi.FGIError) as e:
        ctx.set_grid(big, np.ones(1100), [0, 1100], [0])
    assert e.value.code == -1
    bad = water.pts.copy()
    bad[3, 1] = np.inf
    with pytest.raises(fgi.FGIError) as e:
        ctx.set_grid(bad, water.w, water.batch_off, water.batch_sys)
    assert e.value.code == -6
    with pytest.raises(fgi.FGIError) as e:
        ctx.set_grid(water.pts, water.w, water.batch_off[:-1], water.batch_sys[:-1])
    assert e.value.code == -1
    # batch referring to a missing system is caught at plan time
    ctx.set_grid(water.pts, water.w, water.batch_off, np.full(water.n_batch, 3, np.int32))
    with pytest.raises(fgi.FGIError) as e:
        ctx.plan("fp64")
    assert e.value.code == -1


def test_host_only_context_refuses_compute_and_checks_precision(fgi, water):
    ctx = host_ctx(fgi, water)
    lib = fgi.lib()
    assert lib.fgi_sync(ctx._h, None) == -2
    assert lib.fgi_density(ctx._h, None, None, None, None, 0, None) == -2
    assert lib.fgi_selftest_wait_timeout(ctx._h, None) == -2
    with pytest.raises(fgi.FGIError):
        ctx.set_precision(7)
    ctx.set_precision("split_bf16")


def test_empty_batches_and_far_points_plan(fgi):
    """A batch whose points are beyond every cutoff has no active functions."""
    prob = W.tiny_water(n_rad=8, n_ang=14)
    far = np.array([[100.0, 0, 0], [100.0, 1.0, 0]])
    pts = np.concatenate([prob.pts, far])
    w = np.concatenate([prob.w, [1.0, 1.0]])
    boff = np.concatenate([prob.batch_off, [prob.n_pts + 2]])
    bsys = np.concatenate([prob.batch_sys, [0]])
    prob2 = W.Problem("far", prob.radials, prob.species, prob.atom_off, prob.atom_species,
                      prob.atom_xyz, pts, w, boff.astype(np.int64), bsys.astype(np.int32),
                      np.concatenate([prob.v, [0.0, 0.0]]))
    ctx = host_ctx(fgi, prob2)
    assert ctx.sizes()[2] == prob.n_pts + 2


def test_batch_work_counts_points_and_covers_the_nonzero_functions(fgi):
    import oracle as O
    prob = W.si64()
    ids = np.arange(0, prob.n_batch, max(1, prob.n_batch // 12))
    sub = prob.subgrid(ids)
    ctx = host_ctx(fgi, sub)
    pts, nfn = ctx.batch_work()
    assert np.array_equal(pts, np.diff(sub.batch_off))
    B = O.system_basis(sub)
    for b in range(sub.n_batch):
        p = sub.pts[sub.batch_off[b]:sub.batch_off[b + 1]]
        need = len(O.active_functions(B, p))
        # the plan's active set is a superset (bounding-sphere test), whole atoms
        assert need <= nfn[b] <= B.n_fn
    with pytest.raises(fgi.FGIError) as e:
        ctx._check(ctx._lib.fgi_get_batch_work(ctx._h, sub.n_batch + 1, None, None))
    assert e.value.code == -1


def test_tune_file_is_read_and_checked(fgi, water, tmp_path):
    from paper_2208_12335_gb300 import tune as T
    good = tmp_path / "good.txt"
    T.write_settings(str(good), {"density_sb_points": 512, "density_sb_growth": 1.2, "wave_mb": 256})
    assert T.read_settings(str(good)) == {"density_sb_points": 512.0, "density_sb_growth": 1.2, "wave_mb": 256.0}
    ctx = host_ctx(fgi, water)
    ctx.plan("split_bf16", str(good))
    ctx.plan("split_bf16", str(tmp_path / "missing.txt"))          # no file: the defaults
    bad = tmp_path / "bad.txt"
    bad.write_text("density_sb_points 4096\n")
    with pytest.raises(fgi.FGIError) as e:
        ctx.plan("split_bf16", str(bad))
    assert e.value.code == -1
    bad.write_text("h_sb_points -3\n")
    with pytest.raises(fgi.FGIError) as e:
        ctx.plan("split_bf16", str(bad))
    assert e.value.code == -1
    ok = tmp_path / "ok.txt"
    ok.write_text("h_sb_points 256\nh_sb_growth 1.2\nbound_grids 1\n")
    ctx.plan("split_bf16", str(ok))
    bad.write_text("bound_grids 3\n")
    with pytest.raises(fgi.FGIError) as e:
        ctx.plan("split_bf16", str(bad))
    assert e.value.code == -1
    bad.write_text("density_sb_growth\n")
    with pytest.raises(fgi.FGIError) as e:
        ctx.plan("split_bf16", str(bad))
    assert e.value.code == -1


def test_system_problem_extracts_one_molecule(fgi):
    prob = W.many_molecules(n_mol=3, n_at_range=(3, 5), nrad_range=(16, 18), nang_choices=(50,))
    for s in range(prob.n_sys):
        sp = prob.system_problem(s)
        pts = prob.system_points(s)
        assert sp.n_sys == 1 and np.array_equal(sp.pts, prob.pts[pts]) and np.array_equal(sp.v, prob.v[pts])
        a0, a1 = prob.atom_off[s], prob.atom_off[s + 1]
        assert np.array_equal(sp.atom_xyz, prob.atom_xyz[a0:a1])
        # the one-system plan has the same pattern as that system's block of the joint plan
        joint = host_ctx(fgi, prob)
        alone = host_ctx(fgi, sp)
        rp_j, col_j = joint.pattern(s)
        rp_a, col_a = alone.pattern(0)
        assert np.array_equal(rp_j, rp_a) and np.array_equal(col_j, col_a)


def test_batch_beyond_the_function_limit_is_refused(fgi, water):
    """64 atoms of 140 functions each (twenty f shells) all reach one batch:
    8960 active functions exceed the per-batch limit of 8192, which the
    plan reports instead of building tiles it cannot hold."""
    ctx = host_ctx(fgi, water)
    r = water.radials[0]
    rid = ctx.add_radial(3, r.h, r.coef)
    sp = ctx.add_species(1.0, [rid] * 20)
    g = np.arange(4, dtype=np.float64)
    xyz = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)
    ctx.set_systems([0, 64], np.full(64, sp, np.int32), xyz)
    pts = 1.5 + 0.1 * np.random.default_rng(0).standard_normal((10, 3))
    ctx.set_grid(pts, np.ones(10), [0, 10], [0])
    with pytest.raises(fgi.FGIError) as e:
        ctx.plan("split_bf16")
    assert e.value.code == -7
    # 58 atoms (8120 functions) are within the limit
    ctx.set_systems([0, 58], np.full(58, sp, np.int32), xyz[:58])
    ctx.plan("split_bf16")
    assert ctx.batch_work()[1][0] == 58 * 140


def test_no_fallback_without_the_library_or_a_device(fgi, tmp_path):
    """The compute path has no CPU fallback: a missing libfgi.so is an
    ImportError, and without a CUDA device a device context cannot be
    created at all (host-only contexts only plan)."""
    from paper_2208_12335_gb300 import fgi as F
    with pytest.raises(ImportError):
        F.load_library(str(tmp_path / "libfgi.so"))
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    with pytest.raises(fgi.FGIError) as e:
        fgi.Context(0)
    assert e.value.code == -3                      # FGI_ERR_CUDA: no driver or device


def test_every_autotuner_candidate_plans(fgi, water, tmp_path):
    """The autotuner's default candidates are settings the planner accepts."""
    from paper_2208_12335_gb300 import tune as T
    for i, cand in enumerate(T.DEFAULT_CANDIDATES):
        path = tmp_path / ("cand%d.txt" % i)
        T.write_settings(str(path), cand)
        assert T.read_settings(str(path)) == {k: float(v) for k, v in cand.items()}
        ctx = host_ctx(fgi, water)
        ctx.plan("split_bf16", str(path))
        assert ctx.workspace_size() > 0


def test_autograd_forward_refuses_a_moved_geometry(fgi, water):
    """The plan belongs to the positions given to set_systems: the
    differentiable H call refuses an R that differs from them (before any
    device work), rather than returning H at the planned positions."""
    import torch
    ctx = fgi.Context(-1).load(water, "fp64")
    assert np.array_equal(ctx.positions(), water.atom_xyz)
    v = torch.from_numpy(water.v)
    R = torch.from_numpy(water.atom_xyz.copy())
    R[1, 2] += 1e-6
    with pytest.raises(ValueError, match="planned atom positions"):
        fgi.integrate(ctx, v, R)
    # at the planned positions the call goes on to the H integration, whose
    # argument check wants a device tensor
    with pytest.raises(TypeError, match="CUDA"):
        fgi.integrate(ctx, v, torch.from_numpy(water.atom_xyz.copy()))


def test_atom_grid_structure_is_checked(fgi, water):
    """fgi_set_atom_grids: every point's owner must be an atom of its own
    system and its shell on that atom's radial grid; the Hartree call needs
    a device (a host-only context reports FGI_ERR_STATE)."""
    ctx = fgi.Context(-1).load(water, "fp64")
    ctx.set_atom_grids(water.owner, water.shell, water.atom_rgrid)
    assert ctx.hartree_workspace_size() >= 8 * water.atom_rgrid[:, 2].sum()
    bad = water.shell.copy()
    bad[3] = int(water.atom_rgrid[water.owner[3], 2])          # one past the owner's last shell
    with pytest.raises(fgi.FGIError) as e:
        ctx.set_atom_grids(water.owner, bad, water.atom_rgrid)
    assert e.value.code == -1
    own = water.owner.copy()
    own[0] = 7                                                 # no such atom
    with pytest.raises(fgi.FGIError):
        ctx.set_atom_grids(own, water.shell, water.atom_rgrid)
    rg = water.atom_rgrid.copy()
    rg[1, 1] = -0.1                                            # ln q must be positive
    with pytest.raises(fgi.FGIError):
        ctx.set_atom_grids(water.owner, water.shell, rg)
    lib = fgi.lib()
    assert lib.fgi_hartree(ctx._h, None, None, 4, None, 0, None) == -2


def test_atom_grid_owner_must_share_the_point_system(fgi):
    prob = W.many_molecules(n_mol=2, n_at_range=(3, 3), nrad_range=(8, 8), nang_choices=(14,))
    ctx = fgi.Context(-1).load(prob, "fp64")
    ctx.set_atom_grids(prob.owner, prob.shell, prob.atom_rgrid)
    own = prob.owner.copy()
    p = int(prob.system_points(1)[0])
    own[p] = 0                                                 # an atom of system 0
    with pytest.raises(fgi.FGIError):
        ctx.set_atom_grids(own, prob.shell, prob.atom_rgrid)

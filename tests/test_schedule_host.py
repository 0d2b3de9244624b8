"""The batch scheduler's host tables (CPU, host-only contexts).

Each batch's active functions are recomputed here from their definition
(an atom is active on a batch when one of the batch's points lies within
the species' cutoff) with numpy, independently of the planner.  From those
sets the tests check what fgi_get_schedule reports: super-batches are
consecutive batches of one system, greedy (a batch joins while the merged
points stay within the limit and the union's functions within the growth
limit times the largest member's), with their points and union functions;
waves are consecutive ranges of super-batches; each wave's tile lists take
its super-batches longest first by P n^2, stable for ties.
"""
import numpy as np
import pytest

import workloads as W

K_MAX_POINTS = 1024
K_MAX_FNS = 8192


@pytest.fixture(scope="module")
def fgi():
    from paper_2208_12335_gb300 import build as B
    B.build()
    import paper_2208_12335_gb300 as P
    return P


@pytest.fixture(scope="module")
def cluster():
    # uneven batches (random bisection fractions 0.2..0.8, 50..400 points)
    return W.chno_cluster(n_atoms=40, n_rad=20, n_ang=50)


@pytest.fixture(scope="module")
def molecules():
    return W.many_molecules(n_mol=6, n_at_range=(3, 8), nrad_range=(16, 22), nang_choices=(50, 110),
                            p_max=120, p_min=20)


def active_sets(prob):
    """Per batch: the set of active atoms, by brute force."""
    rc_sp = [max(prob.radials[r].r_cut for r in sp.radial_ids) for sp in prob.species]
    nf_sp = prob.fns_per_species()
    fns = np.array([nf_sp[k] for k in prob.atom_species], np.int64)
    out = []
    for b in range(prob.n_batch):
        s = prob.batch_sys[b]
        a0, a1 = prob.atom_off[s], prob.atom_off[s + 1]
        p = prob.pts[prob.batch_off[b]:prob.batch_off[b + 1]]
        xyz = prob.atom_xyz[a0:a1]
        rc = np.array([rc_sp[k] for k in prob.atom_species[a0:a1]])
        d2 = ((p[:, None, :] - xyz[None, :, :]) ** 2).sum(axis=2)
        on = (d2 < rc[None, :] ** 2).any(axis=0) if len(p) else np.zeros(a1 - a0, bool)
        out.append(set((a0 + np.nonzero(on)[0]).tolist()))
    return out, fns


def plan(fgi, prob, tmp_path, **settings):
    from paper_2208_12335_gb300 import tune as T
    path = tmp_path / "settings.txt"
    T.write_settings(str(path), settings)
    return fgi.Context(-1).load(prob, "split_bf16", tune_path=str(path))


def check_schedule(prob, sched, act, fns, limit_points, growth):
    first = sched["sb_first_batch"]
    ns = len(sched["sb_points"])
    assert first[0] == 0 and first[-1] == prob.n_batch and np.all(np.diff(first) > 0)
    npts = np.diff(prob.batch_off)
    fn_of = lambda atoms: int(sum(fns[a] for a in atoms))
    limit = min(limit_points, K_MAX_POINTS)
    for s in range(ns):
        members = range(first[s], first[s + 1])
        assert len({int(prob.batch_sys[b]) for b in members}) == 1          # one system
        uni = set().union(*[act[b] for b in members])
        assert sched["sb_points"][s] == npts[list(members)].sum()
        assert sched["sb_fns"][s] == fn_of(uni)
        mx = max(fn_of(act[b]) for b in members)
        if len(members) > 1:
            assert sched["sb_points"][s] <= limit
            assert sched["sb_fns"][s] <= growth * mx and sched["sb_fns"][s] <= K_MAX_FNS
        # greedy: the next batch of the same system would break a limit
        nxt = first[s + 1]
        if nxt < prob.n_batch and prob.batch_sys[nxt] == prob.batch_sys[first[s]]:
            joined = fn_of(uni | act[nxt])
            mx2 = max(mx, fn_of(act[nxt]))
            assert (limit_points <= 0 or sched["sb_points"][s] + npts[nxt] > limit
                    or joined > growth * mx2 or joined > K_MAX_FNS)
    wf = sched["wave_first_sb"]
    assert wf[0] == 0 and wf[-1] == ns and np.all(np.diff(wf) > 0)
    P = sched["sb_points"].astype(np.float64)
    n = sched["sb_fns"].astype(np.float64)
    for k in range(len(wf) - 1):
        ids = np.arange(wf[k], wf[k + 1])
        work = ids[(P[ids] > 0) & (n[ids] > 0)]
        assert np.all(sched["sb_rank"][ids[~np.isin(ids, work)]] == -1)
        assert sorted(sched["sb_rank"][work].tolist()) == list(range(len(work)))
        order = work[np.argsort(sched["sb_rank"][work])]
        cost = P[order] * n[order] ** 2
        assert np.all(np.diff(cost) <= 0)                                      # longest first
        ties = np.nonzero(np.diff(cost) == 0)[0]
        assert np.all(order[ties] < order[ties + 1])                           # stable


def test_batch_active_functions_match_their_definition(fgi, cluster, molecules):
    for prob in (cluster, molecules):
        act, fns = active_sets(prob)
        ctx = fgi.Context(-1).load(prob, "fp64")
        pts, nfn = ctx.batch_work()
        assert np.array_equal(pts, np.diff(prob.batch_off))
        assert np.array_equal(nfn, [int(sum(fns[a] for a in s)) for s in act])


@pytest.mark.parametrize("which,points,growth", [("h", 400, 1.25), ("density", 1024, 1.35),
                                                 ("density", 700, 2.0), ("h", 250, 1.0)])
def test_super_batches_waves_and_order(fgi, cluster, molecules, tmp_path, which, points, growth):
    key = "h_sb" if which == "h" else "density_sb"
    for prob in (cluster, molecules):
        act, fns = active_sets(prob)
        ctx = plan(fgi, prob, tmp_path, **{key + "_points": points, key + "_growth": growth})
        check_schedule(prob, ctx.schedule(which), act, fns, points, growth)


def test_default_settings_and_unmerged_batches(fgi, cluster, tmp_path):
    act, fns = active_sets(cluster)
    ctx = fgi.Context(-1).load(cluster, "split_bf16")
    check_schedule(cluster, ctx.schedule("h"), act, fns, 512, 1.25)
    check_schedule(cluster, ctx.schedule("density"), act, fns, 1024, 1.35)
    # a point limit of 0 keeps the batches as given
    ctx = plan(fgi, cluster, tmp_path, h_sb_points=0, density_sb_points=0)
    for which in ("h", "density"):
        s = ctx.schedule(which)
        assert np.array_equal(s["sb_first_batch"], np.arange(cluster.n_batch + 1))
        assert len(s["wave_first_sb"]) == 2                                     # one wave


def test_small_wave_budget_splits_into_waves(fgi, cluster, tmp_path):
    act, fns = active_sets(cluster)
    ctx = plan(fgi, cluster, tmp_path, wave_mb=1)
    for which, pts, gr in (("h", 512, 1.25), ("density", 1024, 1.35)):
        s = ctx.schedule(which)
        assert len(s["wave_first_sb"]) - 1 > 4
        check_schedule(cluster, s, act, fns, pts, gr)


def test_schedule_argument_errors(fgi, cluster):
    ctx = fgi.Context(-1).load(cluster, "fp64")
    with pytest.raises(fgi.FGIError) as e:
        ctx._check(ctx._lib.fgi_get_schedule(ctx._h, 2, None, None, None, None, None, None, None))
    assert e.value.code == -1

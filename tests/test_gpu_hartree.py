"""GPU parity of the step upstream of the integration: the Hartree potential
of the density on the grid (multipole method, fgi_hartree) against the FP64
oracle (oracle/hartree.py), through the C ABI.

* water, its occupied-orbital density (from the oracle), l_max 4 and 6: every
  grid point;
* the Si64 cluster (all 1.14 M points), a sum of atom-centred Gaussian
  charges: seeded sample points against the oracle;
* a spherical Gaussian charge on one atom: the closed form q erf(sqrt(a) r)/r;
* five molecules in one plan: no potential crosses between systems;
* l_max beyond the supported 6 is refused.
Tolerance: the l = 0 terms run in FP64 / double-float on both sides (other
summation orders: 1e-10 of the largest |v_H|); the kernel takes the l >= 1
terms in FP32, each the result of at most ~30 roundings of relative size
2^-24 (four-node interpolation, FP32 harmonics, the sum over l and m), so it
adds at most 2^-18 times the oracle's per-point sum of the magnitudes of the
l >= 1 terms (oracle.hartree: l1_bound).
"""
import math

import numpy as np
import pytest
import torch
from scipy.special import erf

import oracle as O
import oracle.hartree as OH
import workloads as W
from tests import helpers as T

pytestmark = pytest.mark.gpu

TOL = 1e-10
TOL_L1 = 2.0 ** -18


def check(vh, ref, bound):
    err = np.abs(vh - ref)
    lim = TOL * np.abs(ref).max() + TOL_L1 * bound
    assert np.all(err <= lim), (float(np.max(err / lim)), float(err.max()), float(np.abs(ref).max()))


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


def gaussians(prob, alpha=1.1):
    """A sum of Gaussian charges, one per atom (weights from the species' Z)."""
    n = np.zeros(prob.n_pts)
    for a, c in enumerate(prob.atom_xyz):
        Z = prob.species[int(prob.atom_species[a])].Z
        n += Z * (alpha / math.pi) ** 1.5 * np.exp(-alpha * np.sum((prob.pts - c[None, :]) ** 2, axis=1))
    return n


@pytest.mark.parametrize("l_max", [4, 6])
def test_water_occupied_density(fgi, l_max):
    prob = W.tiny_water()
    B = O.system_basis(prob)
    D, _ = W.density_matrix_occ(B.n_fn, 5, np.random.default_rng(3))
    n = O.density(B, prob.pts, D)
    ref, bound = OH.hartree(prob, n, l_max=l_max, l1_bound=True)
    ctx = fgi.Context(0).load(prob, "fp64")
    vh = ctx.hartree(dev(n), l_max=l_max).cpu().numpy()
    ctx.sync()
    check(vh, ref, bound)


def test_si64_gaussian_charges_sampled(fgi):
    prob = W.si64()
    n = gaussians(prob)
    ctx = fgi.Context(0).load(prob, "split_bf16")
    vh = ctx.hartree(dev(n), l_max=4).cpu().numpy()
    ctx.sync()
    idx = np.sort(np.random.default_rng(61).choice(prob.n_pts, 1500, replace=False))
    ref, bound = OH.hartree(prob, n, l_max=4, pts_idx=idx, l1_bound=True)
    check(vh[idx], ref, bound)


def test_spherical_gaussian_closed_form(fgi):
    c, a, N = [0.0, 0.0, 0.0], 0.9, 1.3
    prob = T.gaussian_problem([c], [[(0, 1.0)]], n_rad=80, n_ang=110, r_cut=9.0)
    n = N * np.exp(-a * np.sum(prob.pts ** 2, axis=1))
    ctx = fgi.Context(0).load(prob, "fp64")
    vh = ctx.hartree(dev(n), l_max=0).cpu().numpy()
    ctx.sync()
    r = np.linalg.norm(prob.pts, axis=1)
    ref = N * (math.pi / a) ** 1.5 * erf(math.sqrt(a) * r) / r
    assert np.max(np.abs(vh - ref)) <= 1e-4 * np.abs(ref).max()


def test_molecules_do_not_interact(fgi):
    prob = W.many_molecules(n_mol=5, n_at_range=(3, 6), nrad_range=(16, 20), nang_choices=(50, 74))
    n = gaussians(prob)
    ctx = fgi.Context(0).load(prob, "split_bf16")
    vh = ctx.hartree(dev(n), l_max=4).cpu().numpy()
    ctx.sync()
    ref, bound = OH.hartree(prob, n, l_max=4, l1_bound=True)
    check(vh, ref, bound)
    # each molecule alone gives the same potential on its own points
    s = 2
    one = prob.system_problem(s)
    pts = prob.system_points(s)
    alone, bound1 = OH.hartree(one, n[pts], l_max=4, l1_bound=True)
    check(vh[pts], alone, bound1)


def test_l_max_beyond_six_is_refused(fgi):
    prob = W.tiny_water(n_rad=12, n_ang=26)
    ctx = fgi.Context(0).load(prob, "fp64")
    with pytest.raises(fgi.FGIError) as e:
        ctx.hartree(dev(np.zeros(prob.n_pts)), l_max=7)
    assert e.value.code == -7


def test_degenerate_points_and_zero_density(fgi):
    """Points without an owner (they contribute nothing and still get v_H), a
    point exactly on a nucleus (d = 0: the l = 0 limit inside the first
    shell), the minimal four-shell radial grids, and n = 0 (v_H = 0 exactly)."""
    centers = [[0.0, 0.0, 0.0], [1.4, -0.6, 0.9]]
    prob = T.gaussian_problem(centers, [[(0, 1.0)], [(1, 0.8)]], n_rad=4, n_ang=26, p_max=30, p_min=5,
                              r_cut=6.0)
    rng = np.random.default_rng(17)
    orphan = rng.choice(prob.n_pts, prob.n_pts // 10, replace=False)
    prob.owner = prob.owner.copy()
    prob.owner[orphan] = -1
    j = int(orphan[0])
    prob.pts = prob.pts.copy()
    prob.pts[j] = prob.atom_xyz[1]
    n = gaussians(prob, alpha=0.7) * (1.0 + 0.5 * rng.random(prob.n_pts))
    ref, bound = OH.hartree(prob, n, l_max=2, l1_bound=True)
    ctx = fgi.Context(0).load(prob, "fp64")
    vh = ctx.hartree(dev(n), l_max=2).cpu().numpy()
    zero = ctx.hartree(dev(np.zeros(prob.n_pts)), l_max=2).cpu().numpy()
    ctx.sync()
    check(vh, ref, bound)
    assert np.all(zero == 0.0)


@pytest.mark.parametrize("l_max", [0, 1, 2, 3, 5])
def test_every_l_max(fgi, l_max):
    prob = W.tiny_water(n_rad=20, n_ang=50)
    n = gaussians(prob, alpha=0.9) * (1.0 + 0.4 * np.random.default_rng(5).random(prob.n_pts))
    ref, bound = OH.hartree(prob, n, l_max=l_max, l1_bound=True)
    ctx = fgi.Context(0).load(prob, "split_bf16")
    vh = ctx.hartree(dev(n), l_max=l_max).cpu().numpy()
    ctx.sync()
    check(vh, ref, bound)


def test_hartree_replays_as_a_cuda_graph(fgi):
    """fgi_hartree allocates nothing and never waits on the host: captured
    once, a replay with a new density in the same buffer equals a direct call
    to rounding (the moments are summed with FP64 atomics, in no fixed
    order, so the two agree to about 1e-15, not bitwise)."""
    prob = W.tiny_water(n_rad=20, n_ang=50)
    ctx = fgi.Context(0).load(prob, "split_bf16")
    n_buf = dev(gaussians(prob))
    vh = ctx.hartree(n_buf, l_max=4)
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        ctx.hartree(n_buf, l_max=4, vh=vh, stream=s)
    n2 = gaussians(prob, alpha=0.6)
    n_buf.copy_(dev(n2))
    g.replay()
    torch.cuda.synchronize()
    direct = ctx.hartree(dev(n2), l_max=4).cpu().numpy()
    ctx.sync()
    np.testing.assert_allclose(vh.cpu().numpy(), direct, rtol=0, atol=1e-13 * np.abs(direct).max())

"""The seeded input generators (CPU).

The generators are shared by the oracle and the CUDA path, so a mistake in
them would pass every parity test unnoticed.  These checks hold them to
properties that follow from their definitions: the Fibonacci sphere's
midpoint rule in z, the Becke weights' partition of unity, the molecular
grid's integral of a normalised Gaussian and its convergence, the
bisection's coverage and size bounds, the screened potential's cutoff, the
torch and numpy generator paths agreeing, and seeded reproducibility.
"""
import math

import numpy as np
import pytest
import torch

import workloads as W


@pytest.fixture(scope="module")
def water():
    return W.tiny_water()


@pytest.mark.parametrize("n", [26, 50, 110, 302])
def test_fibonacci_sphere_unit_points_and_midpoint_rule_in_z(n):
    s = W.fibonacci_sphere(n)
    assert s.shape == (n, 3)
    assert np.abs(np.linalg.norm(s, axis=1) - 1.0).max() < 1e-15
    # z_j = 1 - (2j+1)/n is the midpoint rule on [-1, 1]: the mean of z is
    # 0 and the mean of z^2 is 1/3 - 1/(3 n^2), both exactly
    assert abs(s[:, 2].mean()) < 1e-15
    assert abs((s[:, 2] ** 2).mean() - (1.0 / 3.0 - 1.0 / (3.0 * n * n))) < 1e-15


def test_random_rotation_is_proper_orthogonal():
    rng = np.random.default_rng(3)
    for _ in range(20):
        q = W.random_rotation(rng)
        assert np.abs(q @ q.T - np.eye(3)).max() < 1e-14
        assert np.linalg.det(q) == pytest.approx(1.0, abs=1e-14)


def test_becke_weights_are_a_partition_of_unity(water):
    rng = np.random.default_rng(0)
    pts = rng.normal(size=(400, 3)) * 3.0
    xyz = water.atom_xyz
    tot = sum(W.becke_partition(pts, np.full(len(pts), a), xyz) for a in range(len(xyz)))
    assert np.abs(tot - 1.0).max() < 1e-14
    # a point on top of atom A belongs to A alone
    on = W.becke_partition(xyz[:1], np.zeros(1, np.int64), xyz)
    assert on[0] == pytest.approx(1.0, abs=1e-14)


def test_becke_nearest_atom_restriction_and_torch_path_agree():
    """With the cells restricted to a point's 12 nearest atoms (plus the
    owner) the weights over all owners still sum to 1 up to the far atoms'
    vanishing shares; with every atom they sum to 1 to rounding.  The torch
    generator path gives the numpy path's weights.  A 30-atom cluster."""
    rng = np.random.default_rng(1)
    _, pos = W.random_cluster(rng, 30)
    xyz = pos * W.BOHR_PER_ANG
    own = rng.integers(0, 30, size=300)                  # points of atom own's grid
    pts = xyz[own] + rng.normal(size=(300, 3))
    for k, tol in ((30, 1e-14), (12, 1e-7)):
        tot = sum(W.becke_partition(pts, np.full(len(pts), a), xyz, k_near=k) for a in range(30))
        assert np.abs(tot - 1.0).max() < tol
    near = W.becke_partition(pts, own, xyz, k_near=12)
    tch = W.becke_partition_torch(pts, own, xyz, torch.device("cpu"), k_near=12)
    assert np.all((near >= 0) & (near <= 1))
    assert np.abs(tch - near).max() < 1e-13


def _gauss_integral(prob, alpha):
    err = []
    for a in range(len(prob.atom_xyz)):
        d2 = ((prob.pts - prob.atom_xyz[a]) ** 2).sum(axis=1)
        g = (alpha / math.pi) ** 1.5 * np.exp(-alpha * d2)
        err.append(abs(float(np.sum(prob.w * g)) - 1.0))
    return max(err)


def test_molecular_grid_integrates_a_normalised_gaussian_and_converges():
    coarse = W.tiny_water(n_rad=40, n_ang=110)
    fine = W.tiny_water(n_rad=80, n_ang=302)
    e_coarse = _gauss_integral(coarse, 1.0)
    e_fine = _gauss_integral(fine, 1.0)
    assert e_coarse < 1e-3
    assert e_fine < 0.2 * e_coarse
    assert np.all(coarse.w > 0)


@pytest.mark.parametrize("p_max,p_min", [(200, 50), (300, 100), (400, 50)])
def test_bisection_covers_every_point_once_within_the_size_bounds(p_max, p_min):
    rng = np.random.default_rng(p_max)
    xyz = rng.normal(size=(9000, 3)) * np.array([4.0, 2.0, 1.0])
    for q_rng in (None, np.random.default_rng(7)):
        leaves = W.bisect_batches(xyz, p_max, p_min, q_rng, (0.2, 0.8))
        allidx = np.sort(np.concatenate(leaves))
        assert np.array_equal(allidx, np.arange(len(xyz)))
        sizes = np.array([len(lf) for lf in leaves])
        assert sizes.max() <= p_max and sizes.min() >= p_min


def test_bisection_of_small_sets():
    xyz = np.random.default_rng(2).normal(size=(17, 3))
    leaves = W.bisect_batches(xyz, 200, 50)
    assert len(leaves) == 1 and np.array_equal(np.sort(leaves[0]), np.arange(17))
    assert W.bisect_batches(np.zeros((0, 3)), 200, 50) == []


def test_screened_potential_cutoff_and_torch_path():
    rng = np.random.default_rng(4)
    _, pos = W.random_cluster(rng, 40)
    xyz = pos * W.BOHR_PER_ANG
    Z = rng.choice([1.0, 6.0, 7.0, 8.0], size=40)
    pts = xyz[rng.integers(0, 40, size=500)] + rng.normal(size=(500, 3)) * 2.0
    full = W.coulomb_erf_potential(pts, xyz, Z, None, screened=True)
    cut = W.coulomb_erf_potential(pts, xyz, Z, 15.0, screened=True)
    tch = W.coulomb_potential_torch(pts, xyz, Z, torch.device("cpu"), 15.0, True)
    assert np.abs(cut - full).max() <= 1e-13 * np.abs(full).max()
    assert np.abs(tch - cut).max() <= 1e-13 * np.abs(full).max()
    # at a nucleus the bare erf(d)/d form takes its limit 2/sqrt(pi)
    one = W.coulomb_erf_potential(np.zeros((1, 3)), np.zeros((1, 3)), np.array([3.0]))
    assert one[0] == pytest.approx(-3.0 * 2.0 / math.sqrt(math.pi), rel=1e-15)


def test_problem_layout_and_reproducibility(water):
    again = W.tiny_water()
    for f in ("pts", "w", "v", "batch_off", "batch_sys", "atom_xyz"):
        assert np.array_equal(getattr(water, f), getattr(again, f))
    assert len(water.radials) == 4
    assert water.n_fn_sys(0) == 7                       # O 1s 2s 2p + 2 x H 1s
    off = water.batch_off
    assert off[0] == 0 and off[-1] == water.n_pts and np.all(np.diff(off) > 0)
    assert np.all(np.diff(off) <= 200)


def test_many_molecule_layout():
    prob = W.many_molecules(n_mol=5, n_at_range=(3, 6), nrad_range=(16, 20), nang_choices=(50,))
    assert prob.n_sys == 5
    assert np.all(np.diff(prob.batch_sys) >= 0)         # batches grouped by system
    assert set(prob.batch_sys.tolist()) == set(range(5))
    for s in range(prob.n_sys):
        a0, a1 = prob.atom_off[s], prob.atom_off[s + 1]
        pts = prob.pts[prob.system_points(s)]
        # each system's points lie within its atoms' grid radius
        d = np.linalg.norm(pts[:, None, :] - prob.atom_xyz[None, a0:a1, :], axis=2).min(axis=1)
        rmax = max(r.r_cut for r in prob.radials)
        assert d.max() <= rmax * (1 + 1e-12)


def test_density_values_on_a_pattern_match_the_dense_matrix():
    n, n_occ = 60, 9
    D, C = W.density_matrix_occ(n, n_occ, np.random.default_rng(11), occ=2.0)
    assert np.abs(C.T @ C - np.eye(n_occ)).max() < 1e-14
    assert np.trace(D) == pytest.approx(2.0 * n_occ, rel=1e-14)
    assert np.abs(D @ D - 2.0 * D).max() < 1e-13      # idempotent up to the occupation
    rows, cols = np.triu_indices(n)
    vals = W.density_values_occ(n, n_occ, rows, cols, np.random.default_rng(11), 2.0)
    assert np.abs(vals - D[rows, cols]).max() < 1e-15
    vals_t = W.density_values_occ(n, n_occ, rows, cols, np.random.default_rng(11), 2.0,
                                  accel="cpu", chunk_bytes=4096)
    assert np.abs(vals_t - vals).max() < 1e-15

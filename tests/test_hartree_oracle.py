"""Pins of the Hartree-potential oracle (oracle/hartree.py) against what
electrostatics fixes (CPU).

* a spherical Gaussian charge on one atom: v_H = q erf(sqrt(a) r) / r in
  closed form, reached to the radial quadrature's accuracy;
* two Gaussian charges on two atoms of a partitioned grid: the exact
  potential is the sum of the two erf potentials; the multipole error falls
  as l_max grows;
* the monopole of the multipoles is the quadrature of n (an identity of the
  weights, to rounding);
* far from every atom v_H is the exterior multipole field.
"""
import math

import numpy as np
import pytest
from scipy.special import erf

import oracle.hartree as OH
import workloads as W
from tests import helpers as T


def gaussian_density(prob, centers, alphas, norms):
    n = np.zeros(prob.n_pts)
    for c, a, N in zip(centers, alphas, norms):
        n += N * np.exp(-a * np.sum((prob.pts - np.asarray(c)[None, :]) ** 2, axis=1))
    return n


def exact_potential(pts, centers, alphas, norms):
    v = np.zeros(len(pts))
    for c, a, N in zip(centers, alphas, norms):
        r = np.linalg.norm(pts - np.asarray(c)[None, :], axis=1)
        q = N * (math.pi / a) ** 1.5
        v += q * np.where(r > 1e-12, erf(math.sqrt(a) * r) / np.maximum(r, 1e-300), 2.0 * math.sqrt(a / math.pi))
    return v


def test_spherical_gaussian_matches_the_closed_form():
    """l = 0 alone carries a spherical charge; the angular quadrature
    integrates Y_00 exactly, so what remains is the radial quadrature and
    interpolation, fourth order in the shell spacing."""
    c, a, N = [0.0, 0.0, 0.0], 0.9, 1.3
    rng = np.random.default_rng(3)
    dirs = rng.standard_normal((200, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    pts = dirs * rng.uniform(0.05, 20.0, size=(200, 1))       # between shells and outside the grid
    err = {}
    for n_rad in (80, 160):
        prob = T.gaussian_problem([c], [[(0, 1.0)]], n_rad=n_rad, n_ang=110, r_cut=9.0)
        n = gaussian_density(prob, [c], [a], [N])
        v = OH.hartree(prob, n, l_max=0)
        ref = exact_potential(prob.pts, [c], [a], [N])
        T_ = OH.HartreeTables(prob, n, 0)
        ref2 = exact_potential(pts, [c], [a], [N])
        err[n_rad] = max(np.max(np.abs(v - ref)) / np.abs(ref).max(),
                         np.max(np.abs(T_.potential(pts) - ref2)) / np.abs(ref2).max())
    assert err[80] <= 1e-4, err
    assert err[160] <= err[80] / 8.0, err                       # fourth order: 16x per halving


def test_monopole_is_the_quadrature_of_the_density():
    """sqrt(4 pi) sum_k rho_a,00(r_k) r_k^3 ln q summed over the atoms is the
    grid's own quadrature sum_p w_p n_p (an identity of the weights, on a
    partitioned two-atom grid); the exterior monopole Q_00 integrates the same
    shells with the fourth-order rule and agrees to the quadrature's accuracy."""
    centers = [[0.0, 0.0, 0.0], [1.3, 0.9, -1.1]]
    prob = T.gaussian_problem(centers, [[(0, 1.0)], [(0, 1.0)]], n_rad=60, n_ang=110, r_cut=9.0)
    n = gaussian_density(prob, centers, [1.7, 0.9], [0.8, 0.3])
    T_ = OH.HartreeTables(prob, n, 3)
    grid = float(np.sum(prob.w * n))
    shells = 0.0
    for a in range(2):
        r_k, ln_q = T_.r[a], T_.lnq[a]
        shells += math.sqrt(4.0 * math.pi) * float(np.sum(T_.rho[a][:, 0] * r_k ** 3 * ln_q))
    assert shells == pytest.approx(grid, rel=1e-13)
    assert math.sqrt(4.0 * math.pi) * sum(q[0] for q in T_.Q) == pytest.approx(grid, rel=1e-7)


def test_two_centre_charges_converge_with_l_max():
    centers = [[0.0, 0.0, 0.0], [1.3, 0.9, -1.1]]
    prob = T.gaussian_problem(centers, [[(0, 1.0)], [(0, 1.0)]], n_rad=70, n_ang=302, r_cut=9.0)
    alphas, norms = [1.2, 0.7], [1.0, 0.6]
    n = gaussian_density(prob, centers, alphas, norms)
    ref = exact_potential(prob.pts, centers, alphas, norms)
    err = {}
    for l_max in (0, 2, 4, 6):
        v = OH.hartree(prob, n, l_max=l_max)
        err[l_max] = np.max(np.abs(v - ref)) / np.abs(ref).max()
    assert err[2] < 0.5 * err[0] and err[4] < 0.5 * err[2] and err[6] < 0.7 * err[4], err
    assert err[6] <= 2e-3, err


def test_far_field_is_the_exterior_multipole_expansion():
    centers = [[0.0, 0.0, 0.0], [1.3, 0.9, -1.1]]
    prob = T.gaussian_problem(centers, [[(0, 1.0)], [(0, 1.0)]], n_rad=60, n_ang=146, r_cut=9.0)
    alphas, norms = [1.2, 0.7], [1.0, 0.6]
    n = gaussian_density(prob, centers, alphas, norms)
    T_ = OH.HartreeTables(prob, n, 4)
    far = np.array([[40.0, 10.0, -20.0], [-30.0, 35.0, 5.0]])
    v = T_.potential(far)
    ref = exact_potential(far, centers, alphas, norms)
    np.testing.assert_allclose(v, ref, rtol=1e-5)

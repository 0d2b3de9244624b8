"""Pins of the FP64 oracle against results the mathematics fixes.

Each test checks the oracle against something other than itself: scipy's
spherical harmonics, closed-form Gaussian overlaps (Gaussian product
theorem), exact 1-D integrals of the spline, algebraic identities of the
quadrature sum, brute-force Cartesian quadrature with an independently
evaluated basis and potential, and central finite differences.
"""
import math

import numpy as np
import pytest
from scipy.special import erf

import oracle as O
import workloads as W
from tests import helpers as T

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _unit_radial_problem(l_max=3):
    """One atom at the origin whose radial spline is u(r) = r, so phi = Y_lm."""
    radials = []
    for l in range(l_max + 1):
        n = 100
        h = 0.1
        k = np.arange(n, dtype=np.float64)
        coef = np.stack([k * h, np.full(n, h), np.zeros(n), np.zeros(n)], axis=1)
        radials.append(W.Radial(l, h, coef, None, 1.0))
    species = [W.Species("X", 1.0, list(range(l_max + 1)))]
    return radials, species


def test_ylm_match_scipy_real_harmonics():
    radials, species = _unit_radial_problem(3)
    B = O.Basis(radials, species, np.array([0]), np.zeros((1, 3)))
    rng = np.random.default_rng(1)
    dirs = rng.standard_normal((500, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    pts = dirs * rng.uniform(0.5, 5.0, size=(500, 1))
    phi = O.phi(B, pts)
    col = 0
    for l in range(4):
        for m in range(-l, l + 1):
            ref = T.real_sph_harm(l, m, dirs)
            np.testing.assert_allclose(phi[:, col], ref, rtol=0, atol=1e-13,
                                       err_msg="l=%d m=%d" % (l, m))
            col += 1


def test_spline_exact_on_knots_and_zero_beyond_cutoff():
    spec = W.RadialSpec(0, (0.7,), (1.0,), 8.0, None, 800)
    rad = W.make_radial(spec)
    B = O.Basis([rad], [W.Species("X", 1.0, [0])], np.array([0]), np.zeros((1, 3)))
    k = np.arange(1, 800, 37)
    d = k * rad.h
    direction = np.array([0.48, -0.6, 0.64])
    pts = d[:, None] * direction[None, :]
    phi = O.phi(B, pts)[:, 0]
    y00 = 0.5 / math.sqrt(math.pi)
    dd = np.linalg.norm(pts, axis=1)
    np.testing.assert_allclose(phi, rad.coef[k, 0] / dd * y00, rtol=1e-13, atol=0)
    # at and beyond the cutoff the function is exactly zero
    far = np.array([[8.0, 0, 0], [0, 8.0000001, 0], [0, 0, 9.5]])
    assert np.all(O.phi(B, far) == 0.0)


def test_spline_fourth_order_convergence():
    errs = []
    for n in (250, 500):
        spec = W.RadialSpec(1, (0.9,), (1.0,), 8.0, None, n)
        rad = W.make_radial(spec)
        B = O.Basis([rad], [W.Species("X", 1.0, [0])], np.array([0]), np.zeros((1, 3)))
        r = np.linspace(0.05, 6.0, 3001)
        pts = np.stack([np.zeros_like(r), np.zeros_like(r), r], axis=1)   # Y_10 along z
        phi = O.phi(B, pts)[:, 1]
        ref = T.analytic_phi(1, 0, 0.9, rad.norm, np.zeros(3), pts)
        errs.append(np.max(np.abs(phi - ref)))
    ratio = errs[0] / errs[1]
    assert 12.0 < ratio < 20.0, (errs, ratio)


def test_origin_and_edge_values():
    spec0 = W.RadialSpec(0, (0.5,), (1.0,), 8.0, None, 800)
    spec1 = W.RadialSpec(1, (0.5,), (1.0,), 8.0, None, 800)
    r0, r1 = W.make_radial(spec0), W.make_radial(spec1)
    B = O.Basis([r0, r1], [W.Species("X", 1.0, [0, 1])], np.array([0]), np.zeros((1, 3)))
    phi, grad = O.phi(B, np.zeros((1, 3)), grad=True)
    # l = 0: the limit u'(0) Y_00 = (c1/h) Y_00; l > 0: zero
    assert phi[0, 0] == pytest.approx(r0.coef[0, 1] / r0.h * 0.5 / math.sqrt(math.pi), rel=1e-15)
    assert np.all(phi[0, 1:] == 0.0) and np.all(grad == 0.0)
    # the limit agrees with the analytic Gaussian at the origin: N * Y_00
    assert phi[0, 0] == pytest.approx(r0.norm * 0.5 / math.sqrt(math.pi), rel=1e-9)


def test_basis_gradient_central_differences():
    rng = np.random.default_rng(3)
    specs = [W.RadialSpec(l, (0.6 + 0.2 * l, 1.7), (1.0, -0.3), 9.0, 8.0, 3000) for l in range(4)]
    rads = [W.make_radial(s) for s in specs]
    B = O.Basis(rads, [W.Species("X", 1.0, [0, 1, 2, 3])], np.array([0]),
                np.array([[0.3, -0.2, 0.1]]))
    pts = rng.uniform(-3, 3, size=(60, 3))
    _, g = O.phi(B, pts, grad=True)
    h = 1e-5
    for ax in range(3):
        e = np.zeros(3)
        e[ax] = h
        fd = (O.phi(B, pts + e) - O.phi(B, pts - e)) / (2 * h)
        np.testing.assert_allclose(g[:, :, ax], fd, rtol=0, atol=2e-7 * max(1.0, np.abs(fd).max()))


def test_single_s_function_matches_exact_radial_integral():
    """One atom, one s function: sum_p w phi^2 equals int u^2 dr (exact
    Gauss-Legendre integral of the piecewise cubic squared)."""
    spec = W.RadialSpec(0, (0.5,), (1.0,), 9.0, None, 3000)
    prob = T.gaussian_problem(np.zeros((1, 3)), [[(0, 0.5)]], n_rad=400, n_ang=26)
    prob.radials[0] = W.make_radial(spec)
    B = O.system_basis(prob)
    S = O.h_matrix(B, prob.pts, prob.w)
    rad = prob.radials[0]
    x, wq = np.polynomial.legendre.leggauss(6)
    t = 0.5 * (x + 1.0)
    c = rad.coef
    u = c[:, :1] + t[None, :] * (c[:, 1:2] + t[None, :] * (c[:, 2:3] + t[None, :] * c[:, 3:4]))
    k = np.arange(c.shape[0])[:, None]
    r = (k + t[None, :]) * rad.h
    mask = r >= 1e-3            # the grid starts at r_min = 1e-3 Bohr
    exact = 0.5 * rad.h * np.sum((u * u * wq[None, :])[mask])
    assert S[0, 0] == pytest.approx(exact, rel=1e-9)


@pytest.mark.parametrize("coarse,fine", [((40, 110), (100, 974))])
def test_gaussian_overlap_closed_form_convergence(coarse, fine):
    """Grid overlaps of pure Gaussians (s, p, d on A; s, p on B) converge to
    the closed-form two-centre overlap."""
    A = np.array([0.0, 0.0, 0.0])
    Bc = np.array([0.9, -0.5, 1.2])
    shells = [[(0, 0.8), (1, 0.6), (2, 0.5)], [(0, 0.5), (1, 0.7)]]
    fns = []   # (atom, l, m, alpha)
    for a, sh in enumerate(shells):
        for l, al in sh:
            for m in range(-l, l + 1):
                fns.append((a, l, m, al))
    centres = [A, Bc]
    ref = np.zeros((len(fns), len(fns)))
    for i, (ai, li, mi, al_i) in enumerate(fns):
        for j, (aj, lj, mj, al_j) in enumerate(fns):
            ref[i, j] = T.gaussian_overlap(li, mi, al_i, centres[ai], T.analytic_norm(li, al_i),
                                           lj, mj, al_j, centres[aj], T.analytic_norm(lj, al_j))
    errs = []
    for n_rad, n_ang in (coarse, fine):
        prob = T.gaussian_problem(np.stack([A, Bc]), shells, n_rad=n_rad, n_ang=n_ang)
        S = O.h_matrix(O.system_basis(prob), prob.pts, prob.w)
        errs.append(np.max(np.abs(S - ref)))
    assert errs[1] < 2e-4, errs
    assert errs[1] < 0.25 * errs[0], errs


def test_brute_force_cartesian_quadrature_with_potential():
    """On a uniform Cartesian grid the oracle's H equals an independent
    evaluation of sum_p h^3 v phi_i phi_j with analytic Gaussians and the
    erf potential, and its S equals the closed-form overlap."""
    A = np.array([0.0, 0.0, 0.0])
    Bc = np.array([1.1, 0.4, -0.6])
    shells = [[(0, 0.9), (1, 0.8)], [(0, 0.7), (2, 0.9)]]
    prob = T.gaussian_problem(np.stack([A, Bc]), shells, n_rad=10, n_ang=14)
    hs = 0.16
    ax = np.arange(-7.0, 8.0 + 1e-9, hs)
    X, Y, Z = np.meshgrid(ax, ax, ax, indexing="ij")
    pts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    w = np.full(len(pts), hs ** 3)
    Zs = np.array([1.0, 3.0])

    def vfun(p):
        out = np.zeros(len(p))
        for c, z in zip([A, Bc], Zs):
            d = np.linalg.norm(p - c[None, :], axis=1)
            out -= z * np.where(d > 1e-12, erf(d) / np.maximum(d, 1e-300), 2 / math.sqrt(math.pi))
        return out

    v = vfun(pts)
    B = O.system_basis(prob)
    H = O.h_matrix(B, pts, w, v)
    S = O.h_matrix(B, pts, w)
    cols = []
    fns = []
    for a, sh in enumerate(shells):
        for l, al in sh:
            for m in range(-l, l + 1):
                cols.append(T.analytic_phi(l, m, al, T.analytic_norm(l, al), [A, Bc][a], pts))
                fns.append((a, l, m, al))
    Phi = np.stack(cols, axis=1)
    Href = Phi.T @ (Phi * (w * v)[:, None])
    np.testing.assert_allclose(H, Href, rtol=0, atol=1e-7 * np.abs(Href).max())
    Sref = np.zeros_like(S)
    for i, (ai, li, mi, al_i) in enumerate(fns):
        for j, (aj, lj, mj, al_j) in enumerate(fns):
            Sref[i, j] = T.gaussian_overlap(li, mi, al_i, [A, Bc][ai], T.analytic_norm(li, al_i),
                                            lj, mj, al_j, [A, Bc][aj], T.analytic_norm(lj, al_j))
    np.testing.assert_allclose(S, Sref, rtol=0, atol=1e-7)


@pytest.fixture(scope="module")
def water():
    prob = W.tiny_water()
    B = O.system_basis(prob)
    S = O.h_matrix(B, prob.pts, prob.w)
    H = O.h_matrix(B, prob.pts, prob.w, prob.v)
    return prob, B, S, H


def test_constant_potential_gives_c_times_overlap(water):
    prob, B, S, _ = water
    c = -1.7
    Hc = O.h_matrix(B, prob.pts, prob.w, np.full(prob.n_pts, c))
    np.testing.assert_allclose(Hc, c * S, rtol=0, atol=1e-14 * abs(c) * np.abs(S).max() * 10)


def test_symmetric_and_overlap_positive_definite(water):
    _, _, S, H = water
    assert np.max(np.abs(H - H.T)) <= 1e-14 * np.abs(H).max()
    assert np.max(np.abs(S - S.T)) <= 1e-14 * np.abs(S).max()
    np.linalg.cholesky(S)
    assert np.linalg.eigvalsh(S).min() > 0


def test_integrated_density_equals_trace_DS(water):
    prob, B, S, _ = water
    rng = np.random.default_rng(5)
    D = W.random_symmetric(B.n_fn, rng)
    n = O.density(B, prob.pts, D)
    lhs = float(np.sum(prob.w * n))
    rhs = float(np.sum(D * S))
    assert lhs == pytest.approx(rhs, rel=1e-12, abs=1e-12)


def test_electron_count_with_overlap_orthonormal_orbitals(water):
    prob, B, S, _ = water
    rng = W.rng_for(0, W.PURPOSE_D)
    q, _ = np.linalg.qr(rng.standard_normal((B.n_fn, 5)))
    ev, U = np.linalg.eigh(S)
    C = U @ np.diag(ev ** -0.5) @ U.T @ q          # C^T S C = 1
    D = 2.0 * C @ C.T
    n = O.density(B, prob.pts, D)
    assert float(np.sum(prob.w * n)) == pytest.approx(10.0, rel=1e-12)
    assert float(np.sum(D * S)) == pytest.approx(10.0, rel=1e-12)


def test_density_brute_force_small():
    """n_p against phi^T D phi from the oracle's own phi table (exercises the
    neighbour skipping in the density loop)."""
    prob = W.tiny_water(n_rad=12, n_ang=26)
    B = O.system_basis(prob)
    rng = np.random.default_rng(9)
    D = W.random_symmetric(B.n_fn, rng)
    Phi = O.phi(B, prob.pts)
    ref = np.einsum("pi,ij,pj->p", Phi, D, Phi)
    np.testing.assert_allclose(O.density(B, prob.pts, D), ref, rtol=1e-13, atol=1e-13)


def test_h_pairs_agree_with_full_matrix(water):
    prob, B, _, H = water
    pi = np.array([0, 1, 3, 5, 6, 2])
    pj = np.array([0, 5, 6, 6, 1, 4])
    np.testing.assert_allclose(O.h_pairs(B, prob.pts, prob.w, prob.v, pi, pj), H[pi, pj],
                               rtol=1e-12, atol=1e-13)


def test_adjoint_matches_central_differences():
    prob = W.tiny_water(n_rad=20, n_ang=50)
    B = O.system_basis(prob)
    rng = np.random.default_rng(11)
    G = W.random_symmetric(B.n_fn, rng)
    dv, dR = O.adjoint(B, prob.pts, prob.w, prob.v, G)

    def L(v=None, xyz=None):
        bb = B if xyz is None else O.Basis(prob.radials, prob.species, prob.atom_species, xyz)
        return float(np.sum(G * O.h_matrix(bb, prob.pts, prob.w, prob.v if v is None else v)))

    # dL/dv is linear in v: a finite difference along a random direction is exact
    e = rng.standard_normal(prob.n_pts)
    fd = (L(prob.v + e) - L(prob.v - e)) / 2.0
    assert float(np.dot(dv, e)) == pytest.approx(fd, rel=1e-10)
    h = 1e-4 * W.BOHR_PER_ANG
    for a in range(3):
        for x in range(3):
            xp = prob.atom_xyz.copy()
            xm = prob.atom_xyz.copy()
            xp[a, x] += h
            xm[a, x] -= h
            fd = (L(xyz=xp) - L(xyz=xm)) / (2 * h)
            assert dR[a, x] == pytest.approx(fd, rel=1e-6, abs=1e-7 * np.abs(dR).max())


def test_oracle_reproduces_its_regression_fixture():
    """tests/golden/water_16x26_oracle.txt freezes the oracle's H, S and
    density on a small water grid (written by tests/golden/make_golden.py);
    the fixture itself satisfies tr(DS) = 10 (five doubly occupied orbitals)."""
    import importlib.util
    import os
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(here, "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    ref = mg.read(os.path.join(here, "water_16x26_oracle.txt"))
    prob, H, S, D, n = mg.water_case()
    assert prob.n_pts == int(ref["n_points"][0])
    np.testing.assert_allclose(H, ref["H"], rtol=1e-12, atol=1e-14 * np.abs(ref["H"]).max())
    np.testing.assert_allclose(S, ref["S"], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(n[:16], ref["n_first16"], rtol=1e-12, atol=1e-14)
    assert np.trace(ref["D"] @ ref["S"]) == pytest.approx(10.0, rel=1e-12)

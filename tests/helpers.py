"""Independent reference pieces for pinning the oracle (tests only).

Nothing here calls the oracle or the CUDA library: these are textbook
results used to check the oracle from outside.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.special as sp

import workloads as W


def real_sph_harm(l, m, dirs):
    """Real unit-normalised Y_lm without Condon-Shortley phase, from scipy's
    complex harmonics (which carry that phase)."""
    d = np.asarray(dirs, dtype=np.float64)
    d = d / np.linalg.norm(d, axis=1, keepdims=True)
    theta = np.arccos(np.clip(d[:, 2], -1.0, 1.0))
    phi = np.arctan2(d[:, 1], d[:, 0])
    am = abs(m)
    y = sp.sph_harm_y(l, am, theta, phi)
    if m == 0:
        return y.real
    sign = (-1.0) ** am
    if m > 0:
        return math.sqrt(2.0) * sign * y.real
    return math.sqrt(2.0) * sign * y.imag


def monomials(l):
    return [(i, j, l - i - j) for i in range(l, -1, -1) for j in range(l - i, -1, -1)]


def solid_harmonic_coeffs(l, m, rng=None):
    """Coefficients of r^l Y_lm in the degree-l monomials, fitted exactly
    (least squares on random directions) to scipy's harmonics."""
    rng = rng or np.random.default_rng(7)
    dirs = rng.standard_normal((200, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    mons = monomials(l)
    A = np.stack([dirs[:, 0] ** i * dirs[:, 1] ** j * dirs[:, 2] ** k for i, j, k in mons], axis=1)
    y = real_sph_harm(l, m, dirs)
    c, *_ = np.linalg.lstsq(A, y, rcond=None)
    c[np.abs(c) < 1e-13] = 0.0
    return dict(zip(mons, c))


def _gauss_moment(n, p):
    """int (x-P)^n exp(-p (x-P)^2) dx."""
    if n % 2:
        return 0.0
    return math.gamma((n + 1) / 2.0) / p ** ((n + 1) / 2.0)


def overlap_1d(i, j, a, b, alpha, beta):
    """int (x-a)^i (x-b)^j exp(-alpha (x-a)^2 - beta (x-b)^2) dx (Gaussian product theorem)."""
    p = alpha + beta
    P = (alpha * a + beta * b) / p
    mu = alpha * beta / p
    pre = math.exp(-mu * (a - b) ** 2)
    tot = 0.0
    for s in range(i + 1):
        for t in range(j + 1):
            tot += (math.comb(i, s) * math.comb(j, t) * (P - a) ** (i - s) * (P - b) ** (j - t)
                    * _gauss_moment(s + t, p))
    return pre * tot


def gaussian_overlap(lA, mA, alpha, A, NA, lB, mB, beta, B, NB):
    """Closed-form overlap of N r^l Y_lm exp(-alpha r^2) functions on two centres."""
    cA = solid_harmonic_coeffs(lA, mA)
    cB = solid_harmonic_coeffs(lB, mB)
    tot = 0.0
    for (ia, ja, ka), ca in cA.items():
        if ca == 0.0:
            continue
        for (ib, jb, kb), cb in cB.items():
            if cb == 0.0:
                continue
            tot += (ca * cb * overlap_1d(ia, ib, A[0], B[0], alpha, beta)
                    * overlap_1d(ja, jb, A[1], B[1], alpha, beta)
                    * overlap_1d(ka, kb, A[2], B[2], alpha, beta))
    return NA * NB * tot


def analytic_phi(l, m, alpha, N, center, pts):
    """N P_lm(r - A) exp(-alpha |r - A|^2) from the fitted monomial coefficients."""
    d = np.asarray(pts) - np.asarray(center)[None, :]
    c = solid_harmonic_coeffs(l, m)
    P = np.zeros(len(d))
    for (i, j, k), cc in c.items():
        P += cc * d[:, 0] ** i * d[:, 1] ** j * d[:, 2] ** k
    return N * P * np.exp(-alpha * np.sum(d * d, axis=1))


def gaussian_problem(atoms, shells_per_atom, n_rad=60, n_ang=110, p_max=200, p_min=20,
                     r_cut=9.0, n_intervals=4000, v=None, workload_index=90):
    """A custom Problem whose radial functions are single normalised Gaussians.

    atoms: (n,3) Bohr; shells_per_atom: list (per atom) of [(l, alpha), ...].
    Each atom gets its own species.
    """
    radials, species = [], []
    for a, shells in enumerate(shells_per_atom):
        ids = []
        for l, alpha in shells:
            radials.append(W.make_radial(W.RadialSpec(l, (alpha,), (1.0,), r_cut, None, n_intervals)))
            ids.append(len(radials) - 1)
        species.append(W.Species("X%d" % a, 1.0, ids))
    sp_idx = np.arange(len(atoms), dtype=np.int32)
    prob = W.build_problem("gauss", radials, species, [(sp_idx, np.asarray(atoms, float))],
                           lambda s: (n_rad, n_ang), workload_index, (p_max, p_min, None),
                           screened=False)
    if v is not None:
        prob.v = v(prob.pts)
    return prob


def analytic_norm(l, alpha):
    """N with int (N r^l e^{-alpha r^2})^2 r^2 dr = 1."""
    return math.sqrt(2.0 * (2.0 * alpha) ** (l + 1.5) / math.gamma(l + 1.5))

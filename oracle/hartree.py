"""Plain FP64 CPU oracle of the step upstream of the grid integration: the
Hartree potential v_H(r) = int n(r') / |r - r'| dr' of the density on the
integration grid, by the multipole method of Becke & Dickson (J. Chem.
Phys. 89, 2993 (1988)) and Delley (J. Chem. Phys. 92, 508 (1990)), which the
NAO method uses for the electrostatic potential (the paper notes, in its
Fig. 4 caption, that this potential was not yet accelerated on GPUs).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
CPU-baseline leg may call this module; the library never does.  It shares
no code with the CUDA path.

Steps, in the method's order (a reading where the references leave a choice
open is marked "reading"):

1. Multipoles of the partitioned density on each atom's radial shells:
       rho_a,lm(r_k) = sum_{p on atom a, shell k} (w_p / w_k) n_p Y_lm(rhat_p)
   where w_p is the point's integration weight (partition weight times
   radial weight w_k = r_k^3 ln q times angular weight), so w_p / w_k is the
   partitioned angular quadrature weight.
2. Radial Poisson equation per (a, l, m):
       V_a,lm(r) = 4 pi / (2l+1) [ r^-(l+1) int_0^r rho r'^(l+2) dr'
                                  + r^l    int_r^inf rho r'^(1-l) dr' ]
   with the partial integrals over the shells in the variable x = ln r
   (dr = r dx, shell spacing ln q) interval by interval, each interval by
   the integral of the cubic through its four nearest shells (reading; the
   trapezoid rule left 1e-3 relative errors in V on 80 shells), plus, inside
   the first shell r_0, rho(r_0) r_0^(l+3) / (l+3) (rho taken constant there).
3. v_H(r) = sum_a sum_lm V_a,lm(|r - R_a|) Y_lm(direction), where V at a
   distance between shells is the 4-point Lagrange interpolant in the
   fractional shell index ln(d / r_min) / ln q (reading), beyond the last
   shell the exterior multipole field 4 pi / (2l+1) Q_lm / d^(l+1) with
   Q_lm = int_0^inf rho r^(l+2) dr, and inside the first shell
   V(r_0) (d / r_0)^l (reading).  Real spherical harmonics, unit-normalised;
   v_H does not depend on which orthonormal real basis of each l is used.
Independent systems do not interact: a point sees only its own system's atoms.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.special as sp


def real_ylm(l_max: int, dirs: np.ndarray) -> np.ndarray:
    """Real unit-normalised spherical harmonics Y_lm (index l*l + l + m) of
    unit vectors dirs [n][3], from scipy's complex harmonics."""
    d = np.asarray(dirs, dtype=np.float64)
    theta = np.arccos(np.clip(d[:, 2], -1.0, 1.0))
    phi = np.arctan2(d[:, 1], d[:, 0])
    out = np.empty((len(d), (l_max + 1) ** 2))
    for l in range(l_max + 1):
        for m in range(-l, l + 1):
            y = sp.sph_harm_y(l, abs(m), theta, phi)
            if m == 0:
                out[:, l * l + l] = y.real
            elif m > 0:
                out[:, l * l + l + m] = math.sqrt(2.0) * (-1.0) ** m * y.real
            else:
                out[:, l * l + l + m] = math.sqrt(2.0) * (-1.0) ** abs(m) * y.imag
    return out


def interval_integrals(f: np.ndarray, h: float) -> np.ndarray:
    """int over [x_k, x_k+1] of the cubic through the four nearest of the
    equally spaced samples f[k] (spacing h), for k = 0 .. n-2 (rows);
    fewer than four samples: the trapezoid rule."""
    n = f.shape[0]
    if n < 4:
        return 0.5 * h * (f[:-1] + f[1:])
    out = np.empty((n - 1,) + f.shape[1:])
    out[1:n - 2] = h * (-f[0:n - 3] + 13.0 * f[1:n - 2] + 13.0 * f[2:n - 1] - f[3:n]) / 24.0
    out[0] = h * (9.0 * f[0] + 19.0 * f[1] - 5.0 * f[2] + f[3]) / 24.0
    out[n - 2] = h * (f[n - 4] - 5.0 * f[n - 3] + 19.0 * f[n - 2] + 9.0 * f[n - 1]) / 24.0
    return out


def _radii(rg):
    r_min, ln_q, n_rad = float(rg[0]), float(rg[1]), int(rg[2])
    return r_min * np.exp(ln_q * np.arange(n_rad)), ln_q


class HartreeTables:
    """The per-atom radial tables of one density: multipoles rho[a] and
    potentials V[a] (n_rad, L) on the shells, exterior moments Q[a] (L,)."""

    def __init__(self, problem, n, l_max: int):
        self.l_max = l_max
        self.problem = problem
        L = (l_max + 1) ** 2
        xyz = problem.atom_xyz
        self.V, self.Q, self.r, self.lnq, self.rho = [], [], [], [], []
        ls = np.concatenate([[l] * (2 * l + 1) for l in range(l_max + 1)]).astype(np.float64)
        # the points of each owner atom (grouped once)
        by_owner = np.argsort(problem.owner, kind="stable")
        first = np.searchsorted(problem.owner[by_owner], np.arange(len(xyz) + 1))
        for a in range(len(xyz)):
            r_k, ln_q = _radii(problem.atom_rgrid[a])
            sel = by_owner[first[a]:first[a + 1]]
            rho = np.zeros((len(r_k), L))
            if len(sel):
                dvec = problem.pts[sel] - xyz[a][None, :]
                dist = np.linalg.norm(dvec, axis=1)
                k = problem.shell[sel]
                w_ang = problem.w[sel] / (r_k[k] ** 3 * ln_q)
                Y = real_ylm(l_max, dvec / dist[:, None])
                np.add.at(rho, k, (w_ang * n[sel])[:, None] * Y)
            # step 2: partial integrals in x = ln r, interval by interval
            f = rho * r_k[:, None] ** (ls[None, :] + 3.0)        # integrand of the inner integral per dx
            g = rho * r_k[:, None] ** (2.0 - ls[None, :])        # ... of the outer one
            seg_f = interval_integrals(f, ln_q)
            seg_g = interval_integrals(g, ln_q)
            i_in = np.concatenate([np.zeros((1, L)), np.cumsum(seg_f, axis=0)])
            i_in += f[0][None, :] / (ls[None, :] + 3.0)             # 0 < r < r_0
            i_out = np.concatenate([np.cumsum(seg_g[::-1], axis=0)[::-1], np.zeros((1, L))])
            pref = 4.0 * math.pi / (2.0 * ls + 1.0)
            V = pref[None, :] * (r_k[:, None] ** (-(ls[None, :] + 1.0)) * i_in + r_k[:, None] ** ls[None, :] * i_out)
            self.V.append(V)
            self.Q.append(i_in[-1])
            self.rho.append(rho)
            self.r.append(r_k)
            self.lnq.append(ln_q)
        self.ls = ls

    def radial(self, a: int, d: np.ndarray, magnitude: bool = False) -> np.ndarray:
        """V_a,lm at distances d [n]: (n, L).  magnitude: instead the size of
        what is summed for each entry (|V| beyond and inside the grid; between
        shells the sum over the four interpolation nodes of
        (|weight| + |t d weight/dt|) |V|, the second part the first-order
        effect of a relative rounding of t itself), the scale of the rounding
        error of any evaluation of it."""
        V, r_k, ln_q = self.V[a], self.r[a], self.lnq[a]
        n_rad = len(r_k)
        out = np.empty((len(d), V.shape[1]))
        far = d >= r_k[-1]
        near = d <= r_k[0]
        mid = ~(far | near)
        pref = 4.0 * math.pi / (2.0 * self.ls + 1.0)
        if far.any():
            out[far] = pref[None, :] * self.Q[a][None, :] / d[far][:, None] ** (self.ls[None, :] + 1.0)
        if near.any():
            out[near] = V[0][None, :] * (d[near][:, None] / r_k[0]) ** self.ls[None, :]
        if magnitude:
            out[far | near] = np.abs(out[far | near])
        if mid.any():
            x = np.log(d[mid] / r_k[0]) / ln_q
            i0 = np.clip(np.floor(x).astype(np.int64) - 1, 0, n_rad - 4)
            t = x - i0                                   # nodes at t = 0, 1, 2, 3
            acc = np.zeros((mid.sum(), V.shape[1]))
            for j in range(4):
                lj = np.ones_like(t)
                for m in range(4):
                    if m != j:
                        lj *= (t - m) / (j - m)
                if magnitude:
                    dl = np.zeros_like(t)                # d l_j / dt
                    for m in range(4):
                        if m == j:
                            continue
                        pm = np.ones_like(t) / (j - m)
                        for q in range(4):
                            if q != j and q != m:
                                pm *= (t - q) / (j - q)
                        dl += pm
                    acc += (np.abs(lj) + np.abs(t * dl))[:, None] * np.abs(V[i0 + j])
                else:
                    acc += lj[:, None] * V[i0 + j]
            out[mid] = acc
        return out

    def potential(self, pts: np.ndarray, sys_of_pts=None, l1_bound: bool = False):
        """v_H at arbitrary points (all of one system: sys_of_pts None means
        system 0's atoms, else an int system index).  l1_bound: also return,
        per point, sum over atoms and l >= 1 of the magnitudes of the radial
        terms (radial(magnitude=True)) times max |Y_lm| = sqrt((2l+1)/(4 pi))
        (Unsold), the scale of a rounding error confined to the l >= 1 part."""
        prob = self.problem
        s = 0 if sys_of_pts is None else int(sys_of_pts)
        a0, a1 = int(prob.atom_off[s]), int(prob.atom_off[s + 1])
        pts = np.asarray(pts, dtype=np.float64).reshape(-1, 3)
        v = np.zeros(len(pts))
        bound = np.zeros(len(pts))
        ymax = np.sqrt((2.0 * self.ls + 1.0) / (4.0 * math.pi)) * (self.ls >= 1)
        for a in range(a0, a1):
            dvec = pts - prob.atom_xyz[a][None, :]
            d = np.linalg.norm(dvec, axis=1)
            ok = d > 1e-12
            Y = np.zeros((len(pts), (self.l_max + 1) ** 2))
            Y[ok] = real_ylm(self.l_max, dvec[ok] / d[ok][:, None])
            Y[~ok, 0] = 1.0 / math.sqrt(4.0 * math.pi)
            v += np.sum(self.radial(a, d) * Y, axis=1)
            if l1_bound:
                bound += np.sum(self.radial(a, d, magnitude=True) * ymax[None, :], axis=1)
        return (v, bound) if l1_bound else v


def hartree(problem, n: np.ndarray, l_max: int = 4, pts_idx=None, l1_bound: bool = False):
    """v_H at the grid points (all, or the listed indices) of a problem whose
    grid carries its atom-centred structure (owner, shell, atom_rgrid);
    l1_bound: also the per-point scale of the l >= 1 terms
    (HartreeTables.potential)."""
    if problem.owner is None:
        raise ValueError("the problem's grid carries no atom-centred structure")
    T = HartreeTables(problem, np.asarray(n, dtype=np.float64), l_max)
    idx = np.arange(problem.n_pts) if pts_idx is None else np.asarray(pts_idx)
    out = np.empty(len(idx))
    bound = np.empty(len(idx))
    # points of each system see only that system's atoms
    bsys = np.repeat(problem.batch_sys, np.diff(problem.batch_off))
    for s in range(problem.n_sys):
        sel = np.nonzero(bsys[idx] == s)[0]
        if len(sel) and l1_bound:
            out[sel], bound[sel] = T.potential(problem.pts[idx[sel]], s, l1_bound=True)
        elif len(sel):
            out[sel] = T.potential(problem.pts[idx[sel]], s)
    return (out, bound) if l1_bound else out

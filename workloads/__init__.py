"""Seeded synthetic inputs for the NAO grid-integration path.

This module is shared by the oracle and by the CUDA path.  It only builds
*inputs* (geometry, radial spline tables, integration grids with partition
weights, batches, potentials, density matrices, adjoint seeds); it performs
none of the integration arithmetic itself (no basis-function evaluation, no
contraction, no scatter).

Units are atomic units (Bohr, Hartree); 1 Angstrom = 1/0.529177210903 Bohr.

Input recipe (the paper names the method -- numeric atom-centred orbitals
integrated on atom-centred real-space grids, "Development Priorities" -- but
prints no workload definition, so each choice below is a stated reading):

* radial shells  r_k = r_min q^k, k = 0..N_r-1, r_min = 1e-3 Bohr, the last
  shell at the species' largest cutoff; radial weight r_k^3 ln q
  (trapezoid rule in ln r for the integral of f r^2 dr);
* angular points: golden-angle (Fibonacci) sphere, weight 4 pi / N_ang, one
  seeded random rotation per shell;
* partition weights: Becke (1988) fuzzy cells, three iterations of
  p(x) = 1.5x - 0.5x^3, no atomic-size adjustment; for a point the cell
  functions are formed over its owning atom plus its ``becke_k`` nearest
  atoms (exact when the system has no more atoms than that); points with
  weight < 1e-18 are dropped;
* batches: recursive bisection of each system's points along the longest
  bounding-box axis, at the median or (uneven workloads) at a seeded
  quantile, until a leaf holds at most ``p_max`` points; leaves hold at
  least ``p_min``;
* radial functions: u(r) = r R(r), R(r) = N r^l sum_k c_k exp(-a_k r^2),
  optionally multiplied by the C2 switch (1 - x^2)^3,
  x = (r - r_on)/(r_cut - r_on) on [r_on, r_cut]; splined on a uniform grid
  by cubic Hermite interpolation of the exact u and u' (so u is reproduced
  exactly on the knots); normalised so that int u^2 dr = 1;
* v_eff(r) = sum_A -Z_A erf(|r-R_A|)/|r-R_A| (limit -2 Z/sqrt(pi) at the
  nucleus) for the water molecule; for the larger systems the screened,
  neutral-atom-like form sum_A -Z_A (erf(d) - erf(d/2))/d, which keeps
  |v| below ~Z like a self-consistent potential and lets the sum run over
  atoms within ``v_cut`` Bohr only;
* D = 2 C_occ C_occ^T with C_occ the first columns of a seeded orthonormal
  matrix (QR of a Gaussian matrix); for the large workloads only its values
  on the stored pattern are formed (``density_values_occ``); parity tests
  also use seeded symmetric random matrices; G = (X + X^T)/2 with X ~ N(0,1);
* seeds: numpy PCG64 with seed 2208_12335 + 100 * workload_index + purpose
  (0 geometry, 1 basis, 2 D, 3 G, 4 angular rotation, 5 batching).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

BOHR_PER_ANG = 1.0 / 0.529177210903
SEED_BASE = 2208_12335

PURPOSE_GEOMETRY, PURPOSE_BASIS, PURPOSE_D, PURPOSE_G, PURPOSE_ROT, PURPOSE_BATCH = range(6)

Z_OF = {"H": 1.0, "C": 6.0, "N": 7.0, "O": 8.0, "Si": 14.0}


def rng_for(workload_index: int, purpose: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED_BASE + 100 * workload_index + purpose))


# --------------------------------------------------------------------------
# radial functions and their spline tables
# --------------------------------------------------------------------------

@dataclass
class RadialSpec:
    """u(r) = r * N * r^l * sum_k c_k exp(-a_k r^2) * switch(r)."""
    l: int
    alphas: tuple
    coefs: tuple
    r_cut: float
    r_on: float | None = None   # None: hard truncation at r_cut (pure Gaussians)
    n_intervals: int = 2000


def _radial_and_derivative(spec: RadialSpec, r: np.ndarray, norm: float = 1.0):
    """Return u(r), u'(r) for the analytic radial shape (before splining)."""
    r = np.asarray(r, dtype=np.float64)
    l = spec.l
    g = np.zeros_like(r)
    dg = np.zeros_like(r)
    for a, c in zip(spec.alphas, spec.coefs):
        e = np.exp(-a * r * r)
        g += c * e
        dg += c * (-2.0 * a * r) * e
    # u = r^(l+1) g
    rl1 = r ** (l + 1)
    drl1 = (l + 1) * r ** l if l > 0 else np.ones_like(r)
    u = rl1 * g
    du = drl1 * g + rl1 * dg
    if spec.r_on is not None:
        x = np.clip((r - spec.r_on) / (spec.r_cut - spec.r_on), 0.0, 1.0)
        sw = (1.0 - x * x) ** 3
        dsw = 3.0 * (1.0 - x * x) ** 2 * (-2.0 * x) / (spec.r_cut - spec.r_on)
        dsw = np.where((r > spec.r_on) & (r < spec.r_cut), dsw, 0.0)
        du = du * sw + u * dsw
        u = u * sw
    u = np.where(r >= spec.r_cut, 0.0, u)
    du = np.where(r >= spec.r_cut, 0.0, du)
    return norm * u, norm * du


def hermite_spline_table(spec: RadialSpec, norm: float = 1.0):
    """Uniform cubic Hermite spline of u on r_k = k h, k = 0..n.

    Returns (h, coef) with coef[k] = (c0, c1, c2, c3) such that on
    [r_k, r_k+1], u(r) = c0 + t (c1 + t (c2 + t c3)), t = (r - r_k)/h.
    """
    n = spec.n_intervals
    h = spec.r_cut / n
    r = np.arange(n + 1, dtype=np.float64) * h
    u, du = _radial_and_derivative(spec, r, norm)
    u[-1] = 0.0
    du[-1] = 0.0
    u0, u1 = u[:-1], u[1:]
    d0, d1 = h * du[:-1], h * du[1:]
    c0 = u0
    c1 = d0
    c2 = 3.0 * (u1 - u0) - 2.0 * d0 - d1
    c3 = 2.0 * (u0 - u1) + d0 + d1
    return h, np.stack([c0, c1, c2, c3], axis=1).copy()


def normalisation(spec: RadialSpec) -> float:
    """N such that int_0^rcut u(r)^2 dr = 1 (composite Gauss-Legendre)."""
    xg, wg = np.polynomial.legendre.leggauss(12)
    edges = np.linspace(0.0, spec.r_cut, 4001)
    a, b = edges[:-1, None], edges[1:, None]
    r = 0.5 * (b - a) * xg[None, :] + 0.5 * (b + a)
    wr = 0.5 * (b - a) * wg[None, :]
    u, _ = _radial_and_derivative(spec, r.ravel())
    s = float(np.sum(wr.ravel() * u * u))
    return 1.0 / math.sqrt(s)


@dataclass
class Radial:
    l: int
    h: float
    coef: np.ndarray          # (n_intervals, 4) float64
    spec: RadialSpec
    norm: float

    @property
    def n_knots(self) -> int:
        return self.coef.shape[0] + 1

    @property
    def r_cut(self) -> float:
        return self.h * (self.n_knots - 1)


def make_radial(spec: RadialSpec) -> Radial:
    norm = normalisation(spec)
    h, coef = hermite_spline_table(spec, norm)
    return Radial(spec.l, h, coef, spec, norm)


@dataclass
class Species:
    name: str
    Z: float
    radial_ids: list           # one entry per radial shell; expands to 2l+1 fns


# --------------------------------------------------------------------------
# problem container
# --------------------------------------------------------------------------

@dataclass
class Problem:
    name: str
    radials: list
    species: list
    atom_off: np.ndarray       # (n_sys+1,) int64
    atom_species: np.ndarray   # (n_atoms,) int32
    atom_xyz: np.ndarray       # (n_atoms, 3) float64, Bohr
    pts: np.ndarray            # (n_pts, 3) float64
    w: np.ndarray              # (n_pts,) float64
    batch_off: np.ndarray      # (n_batch+1,) int64
    batch_sys: np.ndarray      # (n_batch,) int32
    v: np.ndarray              # (n_pts,) float64
    workload_index: int = 0
    meta: dict = field(default_factory=dict)
    # atom-centred structure of the grid (None where it is not known):
    # owner atom and radial shell of every point, and per atom its radial
    # grid r_k = r_min q^k, k < n_rad, as rows (r_min, ln q, n_rad)
    owner: np.ndarray = None   # (n_pts,) int32, global atom index
    shell: np.ndarray = None   # (n_pts,) int32
    atom_rgrid: np.ndarray = None  # (n_atoms, 3) float64

    @property
    def n_sys(self) -> int:
        return len(self.atom_off) - 1

    @property
    def n_pts(self) -> int:
        return len(self.w)

    @property
    def n_batch(self) -> int:
        return len(self.batch_off) - 1

    def fns_per_species(self):
        return [sum(2 * self.radials[r].l + 1 for r in sp.radial_ids) for sp in self.species]

    def n_fn_sys(self, s: int) -> int:
        nf = self.fns_per_species()
        a0, a1 = self.atom_off[s], self.atom_off[s + 1]
        return int(sum(nf[k] for k in self.atom_species[a0:a1]))

    def system_points(self, s: int) -> np.ndarray:
        """Indices of the points belonging to system s (batches are grouped)."""
        bs = np.nonzero(self.batch_sys == s)[0]
        if len(bs) == 0:
            return np.zeros(0, dtype=np.int64)
        return np.arange(self.batch_off[bs[0]], self.batch_off[bs[-1] + 1])

    def system_problem(self, s: int) -> "Problem":
        """System s alone: its atoms, batches and points (a one-system problem)."""
        a0, a1 = int(self.atom_off[s]), int(self.atom_off[s + 1])
        bs = np.nonzero(self.batch_sys == s)[0]
        p0, p1 = int(self.batch_off[bs[0]]), int(self.batch_off[bs[-1] + 1])
        off = (self.batch_off[bs[0]:bs[-1] + 2] - p0).astype(np.int64)
        grid = {}
        if self.owner is not None:
            grid = dict(owner=(self.owner[p0:p1] - a0).astype(np.int32), shell=self.shell[p0:p1].copy(),
                        atom_rgrid=self.atom_rgrid[a0:a1].copy())
        return Problem("%s-sys%d" % (self.name, s), self.radials, self.species,
                       np.array([0, a1 - a0], dtype=np.int64), self.atom_species[a0:a1].copy(),
                       self.atom_xyz[a0:a1].copy(), self.pts[p0:p1].copy(), self.w[p0:p1].copy(), off,
                       np.zeros(len(bs), dtype=np.int32), self.v[p0:p1].copy(), self.workload_index,
                       dict(self.meta), **grid)

    def subgrid(self, batch_ids) -> "Problem":
        """A new problem holding only the listed batches (same geometry)."""
        batch_ids = np.asarray(sorted(batch_ids), dtype=np.int64)
        idx = np.concatenate([np.arange(self.batch_off[b], self.batch_off[b + 1]) for b in batch_ids])
        sizes = self.batch_off[batch_ids + 1] - self.batch_off[batch_ids]
        off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        grid = {}
        if self.owner is not None:
            grid = dict(owner=self.owner[idx].copy(), shell=self.shell[idx].copy(), atom_rgrid=self.atom_rgrid)
        return Problem(self.name + "-sub", self.radials, self.species, self.atom_off,
                       self.atom_species, self.atom_xyz, self.pts[idx].copy(), self.w[idx].copy(),
                       off, self.batch_sys[batch_ids].copy(), self.v[idx].copy(),
                       self.workload_index, dict(self.meta), **grid)


# --------------------------------------------------------------------------
# grids
# --------------------------------------------------------------------------

def fibonacci_sphere(n: int) -> np.ndarray:
    j = np.arange(n, dtype=np.float64)
    z = 1.0 - (2.0 * j + 1.0) / n
    rho = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    th = j * (math.pi * (3.0 - math.sqrt(5.0)))
    return np.stack([rho * np.cos(th), rho * np.sin(th), z], axis=1)


def random_rotation(rng: np.random.Generator) -> np.ndarray:
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q * np.sign(np.diag(r))[None, :]
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def atom_grid(center, r_max, n_rad, n_ang, rng, r_min=1e-3, with_shells=False):
    """Points and (un-partitioned) weights of one atom-centred grid (and,
    with_shells, the radial shell index of every point)."""
    q = (r_max / r_min) ** (1.0 / (n_rad - 1))
    r = r_min * q ** np.arange(n_rad, dtype=np.float64)
    wr = r ** 3 * math.log(q)
    s = fibonacci_sphere(n_ang)
    wa = 4.0 * math.pi / n_ang
    pts = np.empty((n_rad, n_ang, 3))
    for k in range(n_rad):
        pts[k] = (s @ random_rotation(rng).T) * r[k]
    pts = pts.reshape(-1, 3) + np.asarray(center)[None, :]
    w = np.repeat(wr * wa, n_ang)
    if with_shells:
        return pts, w, np.repeat(np.arange(n_rad, dtype=np.int32), n_ang)
    return pts, w


def _becke_s(mu):
    f = mu
    for _ in range(3):
        f = 1.5 * f - 0.5 * f * f * f
    return 0.5 * (1.0 - f)


def becke_partition(pts, owner, atom_xyz, k_near=12, chunk=40000):
    """Becke cell weight P_owner / sum_C P_C for each point."""
    n_at = len(atom_xyz)
    k = min(k_near, n_at)
    out = np.empty(len(pts))
    if n_at == 1:
        out[:] = 1.0
        return out
    rab = np.linalg.norm(atom_xyz[:, None, :] - atom_xyz[None, :, :], axis=2)
    tree = None
    if k < n_at:
        from scipy.spatial import cKDTree
        tree = cKDTree(atom_xyz)
    for c0 in range(0, len(pts), chunk):
        p = pts[c0:c0 + chunk]
        own = owner[c0:c0 + chunk]
        if tree is None:
            idx = np.broadcast_to(np.arange(n_at), (len(p), n_at)).copy()
        else:
            _, idx = tree.query(p, k=k)
            idx = idx.reshape(len(p), k)
            has = (idx == own[:, None]).any(axis=1)
            idx[~has, -1] = own[~has]
        d = np.linalg.norm(p[:, None, :] - atom_xyz[idx], axis=2)          # (n,k)
        R = rab[idx[:, :, None], idx[:, None, :]]                            # (n,k,k)
        with np.errstate(divide="ignore", invalid="ignore"):
            mu = (d[:, :, None] - d[:, None, :]) / R
        s = _becke_s(np.where(R > 0, mu, 0.0))
        kk = idx.shape[1]
        s[:, np.arange(kk), np.arange(kk)] = 1.0
        P = np.prod(s, axis=2)                                               # (n,k)
        pown = P[idx == own[:, None]]
        out[c0:c0 + chunk] = pown / P.sum(axis=1)
    return out


def _torch_device(accel):
    """torch device for the accelerated generator paths (None: numpy)."""
    if not accel:
        return None
    import torch
    if accel == "cuda" and not torch.cuda.is_available():
        return torch.device("cpu")
    return torch.device(accel)


def becke_partition_torch(pts, owner, atom_xyz, dev, k_near=12, chunk=200000):
    """Becke cell weight P_owner / sum_C P_C (same definition as becke_partition)
    with torch in float64 on `dev`: the owning atom plus its k nearest atoms."""
    import torch
    A = torch.as_tensor(atom_xyz, dtype=torch.float64, device=dev)
    n_at = A.shape[0]
    k = min(k_near, n_at)
    rab = torch.cdist(A, A)
    out = np.empty(len(pts))
    if n_at == 1:
        out[:] = 1.0
        return out
    for c0 in range(0, len(pts), chunk):
        p = torch.as_tensor(pts[c0:c0 + chunk], dtype=torch.float64, device=dev)
        own = torch.as_tensor(owner[c0:c0 + chunk], dtype=torch.int64, device=dev)
        dall = torch.cdist(p, A)                                             # (n, n_at)
        idx = torch.topk(dall, k, dim=1, largest=False).indices              # nearest k
        has = (idx == own[:, None]).any(dim=1)
        idx[~has, -1] = own[~has]
        d = torch.gather(dall, 1, idx)
        R = rab[idx[:, :, None], idx[:, None, :]]
        mu = torch.where(R > 0, (d[:, :, None] - d[:, None, :]) / torch.where(R > 0, R, 1.0), 0.0)
        f = mu
        for _ in range(3):
            f = 1.5 * f - 0.5 * f * f * f
        s = 0.5 * (1.0 - f)
        eye = torch.eye(k, dtype=torch.bool, device=dev)
        s = torch.where(eye[None], 1.0, s)
        P = torch.prod(s, dim=2)
        pown = (P * (idx == own[:, None])).sum(dim=1)
        out[c0:c0 + chunk] = (pown / P.sum(dim=1)).cpu().numpy()
    return out


def coulomb_potential_torch(pts, atom_xyz, Z, dev, v_cut, screened, chunk=20000):
    """Same function as coulomb_erf_potential, with torch in float64 on `dev`."""
    import torch
    A = torch.as_tensor(atom_xyz, dtype=torch.float64, device=dev)
    Zt = torch.as_tensor(Z, dtype=torch.float64, device=dev)
    c = 2.0 / math.sqrt(math.pi) * (0.5 if screened else 1.0)
    v = np.empty(len(pts))
    for c0 in range(0, len(pts), chunk):
        p = torch.as_tensor(pts[c0:c0 + chunk], dtype=torch.float64, device=dev)
        d = torch.cdist(p, A)
        num = torch.erf(d) - torch.erf(0.5 * d) if screened else torch.erf(d)
        f = torch.where(d > 1e-12, num / torch.where(d > 1e-12, d, 1.0), c)
        if v_cut is not None:
            f = torch.where(d < v_cut, f, 0.0)
        v[c0:c0 + chunk] = -(f * Zt[None, :]).sum(dim=1).cpu().numpy()
    return v


def bisect_batches(xyz, p_max, p_min, rng=None, q_range=(0.5, 0.5)):
    """Recursive bisection; returns a list of index arrays (depth-first)."""
    leaves = []
    stack = [np.arange(len(xyz), dtype=np.int64)]
    while stack:
        idx = stack.pop()
        n = len(idx)
        if n <= p_max:
            if n > 0:
                leaves.append(idx)
            continue
        p = xyz[idx]
        ax = int(np.argmax(p.max(axis=0) - p.min(axis=0)))
        q = 0.5 if rng is None else rng.uniform(*q_range)
        kk = int(round(q * n))
        kk = max(p_min, min(n - p_min, kk))
        part = np.argpartition(p[:, ax], kk)
        stack.append(idx[part[kk:]])
        stack.append(idx[part[:kk]])
    return leaves


def coulomb_erf_potential(pts, atom_xyz, Z, v_cut=None, chunk=200000, screened=False):
    """v(r) = sum_A -Z_A f(|r - R_A|).

    f(d) = erf(d)/d (bare, regularised nucleus), or, screened,
    f(d) = (erf(d) - erf(d/2))/d: the same nucleus minus a neutralising
    Gaussian electron cloud, so that f decays like a Gaussian and a sum
    over atoms within ``v_cut`` is exact to double precision.
    """
    from scipy.special import erf
    v = np.zeros(len(pts))
    c = 2.0 / math.sqrt(math.pi) * (0.5 if screened else 1.0)

    def f_of(d):
        with np.errstate(divide="ignore", invalid="ignore"):
            num = erf(d) - erf(0.5 * d) if screened else erf(d)
            return np.where(d > 1e-12, num / d, c)
    if v_cut is None:
        for c0 in range(0, len(pts), chunk):
            p = pts[c0:c0 + chunk]
            d = np.linalg.norm(p[:, None, :] - atom_xyz[None, :, :], axis=2)
            v[c0:c0 + chunk] = -(f_of(d) * Z[None, :]).sum(axis=1)
        return v
    from scipy.spatial import cKDTree
    tree = cKDTree(pts)
    for a in range(len(atom_xyz)):
        ids = np.asarray(tree.query_ball_point(atom_xyz[a], v_cut), dtype=np.int64)
        if len(ids) == 0:
            continue
        d = np.linalg.norm(pts[ids] - atom_xyz[a][None, :], axis=1)
        v[ids] -= Z[a] * f_of(d)
    return v


def build_problem(name, radials, species, systems, grid_spec, workload_index,
                  batch_spec, v_full_atoms=200, v_cut=15.0, becke_k=12, screened=True, accel=None):
    """Assemble a Problem from per-system geometries.

    systems: list of (species_index_array, xyz_bohr_array)
    grid_spec: function(species_index) -> (n_rad, n_ang)
    batch_spec: (p_max, p_min, q_range or None)
    """
    rng_rot = rng_for(workload_index, PURPOSE_ROT)
    rng_bat = rng_for(workload_index, PURPOSE_BATCH)
    rmax_sp = [max(radials[r].r_cut for r in sp.radial_ids) for sp in species]
    atom_off = [0]
    all_sp, all_xyz, all_pts, all_w, all_v, boff, bsys = [], [], [], [], [], [0], []
    all_own, all_shell, all_rgrid = [], [], []
    p_max, p_min, q_range = batch_spec
    for s, (sp_idx, xyz) in enumerate(systems):
        sp_idx = np.asarray(sp_idx, dtype=np.int32)
        xyz = np.asarray(xyz, dtype=np.float64)
        pts_l, w_l, own_l, sh_l = [], [], [], []
        for a in range(len(xyz)):
            n_rad, n_ang = grid_spec(int(sp_idx[a]))
            p, w, sh = atom_grid(xyz[a], rmax_sp[sp_idx[a]], n_rad, n_ang, rng_rot, with_shells=True)
            pts_l.append(p)
            w_l.append(w)
            own_l.append(np.full(len(w), a, dtype=np.int64))
            sh_l.append(sh)
            all_rgrid.append((1e-3, math.log((rmax_sp[sp_idx[a]] / 1e-3) ** (1.0 / (n_rad - 1))), n_rad))
        pts = np.concatenate(pts_l)
        w = np.concatenate(w_l)
        own = np.concatenate(own_l)
        shell = np.concatenate(sh_l)
        dev = _torch_device(accel)
        if dev is None:
            w = w * becke_partition(pts, own, xyz, k_near=becke_k)
        else:
            w = w * becke_partition_torch(pts, own, xyz, dev, k_near=becke_k)
        keep = w >= 1e-18
        pts, w, own, shell = pts[keep], w[keep], own[keep], shell[keep]
        Zs = np.array([species[k].Z for k in sp_idx])
        vc = None if len(xyz) <= v_full_atoms else v_cut
        if dev is None:
            v = coulomb_erf_potential(pts, xyz, Zs, vc, screened=screened)
        else:
            v = coulomb_potential_torch(pts, xyz, Zs, dev, vc, screened)
        leaves = bisect_batches(pts, p_max, p_min, rng_bat if q_range else None,
                                q_range if q_range else (0.5, 0.5))
        order = np.concatenate(leaves)
        all_pts.append(pts[order])
        all_w.append(w[order])
        all_v.append(v[order])
        all_own.append((own[order] + atom_off[-1]).astype(np.int32))
        all_shell.append(shell[order])
        for lf in leaves:
            boff.append(boff[-1] + len(lf))
            bsys.append(s)
        all_sp.append(sp_idx)
        all_xyz.append(xyz)
        atom_off.append(atom_off[-1] + len(xyz))
    return Problem(name, radials, species, np.array(atom_off, dtype=np.int64),
                   np.concatenate(all_sp).astype(np.int32), np.concatenate(all_xyz),
                   np.concatenate(all_pts), np.concatenate(all_w),
                   np.array(boff, dtype=np.int64), np.array(bsys, dtype=np.int32),
                   np.concatenate(all_v), workload_index, owner=np.concatenate(all_own),
                   shell=np.concatenate(all_shell), atom_rgrid=np.array(all_rgrid, dtype=np.float64))


# --------------------------------------------------------------------------
# the workloads
# --------------------------------------------------------------------------

def water_geometry():
    """O at the origin, two H at 0.96 A with an H-O-H angle of 104.5 degrees."""
    r = 0.96 * BOHR_PER_ANG
    half = math.radians(104.5) / 2.0
    return np.array([[0.0, 0.0, 0.0],
                     [r * math.sin(half), 0.0, r * math.cos(half)],
                     [-r * math.sin(half), 0.0, r * math.cos(half)]])


def tiny_water(n_rad=40, n_ang=110, p_max=200, p_min=50, workload_index=0, alphas=None):
    """3 atoms, 7 fns (O 1s 2s 2p, H 1s), single Gaussian primitives, cutoff 5 A."""
    rc = 5.0 * BOHR_PER_ANG
    a = dict(O1s=10.0, O2s=0.8, O2p=0.6, H1s=0.5)
    if alphas:
        a.update(alphas)
    specs = [RadialSpec(0, (a["O1s"],), (1.0,), rc, None, 4000),
             RadialSpec(0, (a["O2s"],), (1.0,), rc, None, 4000),
             RadialSpec(1, (a["O2p"],), (1.0,), rc, None, 4000),
             RadialSpec(0, (a["H1s"],), (1.0,), rc, None, 4000)]
    radials = [make_radial(s) for s in specs]
    species = [Species("O", 8.0, [0, 1, 2]), Species("H", 1.0, [3])]
    systems = [(np.array([0, 1, 1]), water_geometry())]
    return build_problem("tiny-water", radials, species, systems, lambda sp: (n_rad, n_ang),
                         workload_index, (p_max, p_min, None), screened=False)


def _seeded_radials(rng, shells, r_cut, r_on, n_intervals, alpha_ranges):
    """shells: list of l values; alpha_ranges: per-l list of (lo, hi) per shell."""
    specs = []
    count = {}
    for l in shells:
        k = count.get(l, 0)
        count[l] = k + 1
        lo, hi = alpha_ranges[l][k]
        a0 = math.exp(rng.uniform(math.log(lo), math.log(hi)))
        nterm = int(rng.integers(2, 4))
        alphas = [a0]
        coefs = [1.0]
        for _ in range(nterm - 1):
            alphas.append(a0 * rng.uniform(1.5, 3.0))
            coefs.append(rng.uniform(-0.5, 0.5))
        specs.append(RadialSpec(l, tuple(alphas), tuple(coefs), r_cut, r_on, n_intervals))
    return specs


SI_ALPHA = {0: [(4.0, 8.0), (1.5, 3.0), (0.6, 1.2), (0.3, 0.6), (0.15, 0.3), (0.08, 0.15)],
            1: [(1.5, 3.0), (0.4, 1.0), (0.12, 0.3)],
            2: [(0.5, 1.2), (0.15, 0.4)]}


def si64(n_rad=60, n_ang=302, p_max=300, p_min=100, workload_index=1, cells=2, jitter_ang=0.05,
         accel=None):
    """Si diamond cluster (2x2x2 conventional cells, 64 atoms), 25 fns/atom.

    The workload names 4s,3p,2d shells and 25 fns/atom; with real spherical
    harmonics 4s3p2d gives 23, so the total of 25 is kept with 6s3p2d.
    """
    rng_g = rng_for(workload_index, PURPOSE_GEOMETRY)
    rng_b = rng_for(workload_index, PURPOSE_BASIS)
    a = 5.43
    basis = np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0],
                      [.25, .25, .25], [.25, .75, .75], [.75, .25, .75], [.75, .75, .25]])
    pos = []
    for i in range(cells):
        for j in range(cells):
            for k in range(cells):
                pos.append((basis + np.array([i, j, k])) * a)
    pos = np.concatenate(pos)
    pos = pos - pos.mean(axis=0)
    pos = pos + rng_g.normal(0.0, jitter_ang, size=pos.shape)
    xyz = pos * BOHR_PER_ANG
    rc = 6.0 * BOHR_PER_ANG
    specs = _seeded_radials(rng_b, [0, 0, 0, 0, 0, 0, 1, 1, 1, 2, 2], rc, rc - BOHR_PER_ANG, 2000,
                            SI_ALPHA)
    radials = [make_radial(s) for s in specs]
    species = [Species("Si", 14.0, list(range(len(radials))))]
    systems = [(np.zeros(len(xyz), dtype=np.int32), xyz)]
    return build_problem("si64", radials, species, systems, lambda sp: (n_rad, n_ang),
                         workload_index, (p_max, p_min, None), accel=accel)


HEAVY_ALPHA = {0: [(4.0, 8.0), (1.5, 3.0), (0.6, 1.2), (0.25, 0.5), (0.1, 0.2)],
               1: [(1.0, 2.0), (0.3, 0.7), (0.12, 0.25)],
               2: [(0.4, 1.0)]}
H_ALPHA = {0: [(0.8, 1.6), (0.15, 0.35)], 1: [(0.3, 0.8)]}


def random_cluster(rng, n_atoms, density_per_ang3=0.1, min_dist_ang=1.0, h_frac=0.5):
    """Seeded random packing in a sphere by rejection; returns (elements, xyz_ang)."""
    radius = (3.0 * n_atoms / (4.0 * math.pi * density_per_ang3)) ** (1.0 / 3.0)
    pos = []
    tries = 0
    while len(pos) < n_atoms:
        tries += 1
        if tries > 2000 * n_atoms:
            radius *= 1.05
            tries = 0
        p = rng.uniform(-radius, radius, size=3)
        if np.dot(p, p) > radius * radius:
            continue
        if pos:
            d = np.linalg.norm(np.asarray(pos) - p[None, :], axis=1)
            if d.min() < min_dist_ang:
                continue
        pos.append(p)
    heavy = ["C", "N", "O"]
    elems = []
    for _ in range(n_atoms):
        if rng.uniform() < h_frac:
            elems.append("H")
        else:
            elems.append(heavy[int(rng.integers(0, 3))])
    return elems, np.asarray(pos)


def chno_species(rng, r_cut_ang=5.0):
    """H/C/N/O species: heavy 5s3p1d (19 fns), H 2s1p (5 fns), C2 switch."""
    rc = r_cut_ang * BOHR_PER_ANG
    r_on = rc - BOHR_PER_ANG
    radials, species = [], []
    for name in ["H", "C", "N", "O"]:
        if name == "H":
            specs = _seeded_radials(rng, [0, 0, 1], rc, r_on, 1500, H_ALPHA)
        else:
            specs = _seeded_radials(rng, [0, 0, 0, 0, 0, 1, 1, 1, 2], rc, r_on, 1500, HEAVY_ALPHA)
        ids = list(range(len(radials), len(radials) + len(specs)))
        radials += [make_radial(s) for s in specs]
        species.append(Species(name, Z_OF[name], ids))
    return radials, species


def chno_cluster(n_atoms=1000, n_rad=70, n_ang=590, p_max=400, p_min=50, workload_index=2,
                 atoms_with_grid=None, accel=None):
    """Random organic-like C/H/N/O cluster; uneven batches.

    atoms_with_grid: optional list of atom indices whose atom-centred grids
    are generated (the others still enter the partition weights); used to
    build sampled sub-grids of the full workload.
    """
    rng_g = rng_for(workload_index, PURPOSE_GEOMETRY)
    rng_b = rng_for(workload_index, PURPOSE_BASIS)
    elems, pos = random_cluster(rng_g, n_atoms)
    radials, species = chno_species(rng_b)
    sp_of = {"H": 0, "C": 1, "N": 2, "O": 3}
    sp_idx = np.array([sp_of[e] for e in elems], dtype=np.int32)
    xyz = pos * BOHR_PER_ANG
    return build_problem_grid_subset("chno%d" % n_atoms, radials, species, sp_idx, xyz,
                                     (n_rad, n_ang), workload_index, (p_max, p_min, (0.2, 0.8)),
                                     atoms_with_grid, accel)


def build_problem_grid_subset(name, radials, species, sp_idx, xyz, nrad_nang, workload_index,
                              batch_spec, atoms_with_grid, accel=None):
    if atoms_with_grid is None:
        return build_problem(name, radials, species, [(sp_idx, xyz)], lambda sp: nrad_nang,
                             workload_index, batch_spec, accel=accel)
    # generate only the listed atoms' grids (same rotations as the full build
    # would give those atoms only if every atom is listed; this is a separate,
    # smaller workload over the same geometry)
    rng_rot = rng_for(workload_index, PURPOSE_ROT)
    rng_bat = rng_for(workload_index, PURPOSE_BATCH)
    rmax_sp = [max(radials[r].r_cut for r in sp.radial_ids) for sp in species]
    pts_l, w_l, own_l = [], [], []
    for a in atoms_with_grid:
        p, w = atom_grid(xyz[a], rmax_sp[sp_idx[a]], nrad_nang[0], nrad_nang[1], rng_rot)
        pts_l.append(p)
        w_l.append(w)
        own_l.append(np.full(len(w), a, dtype=np.int64))
    pts = np.concatenate(pts_l)
    w = np.concatenate(w_l)
    own = np.concatenate(own_l)
    w = w * becke_partition(pts, own, xyz)
    keep = w >= 1e-18
    pts, w = pts[keep], w[keep]
    Zs = np.array([species[k].Z for k in sp_idx])
    v = coulomb_erf_potential(pts, xyz, Zs, 15.0, screened=True)
    p_max, p_min, q_range = batch_spec
    leaves = bisect_batches(pts, p_max, p_min, rng_bat, q_range)
    order = np.concatenate(leaves)
    boff = np.concatenate([[0], np.cumsum([len(lf) for lf in leaves])]).astype(np.int64)
    return Problem(name + "-sub", radials, species, np.array([0, len(xyz)], dtype=np.int64),
                   sp_idx, xyz, pts[order], w[order], boff,
                   np.zeros(len(leaves), dtype=np.int32), v[order], workload_index)


def many_molecules(n_mol=512, workload_index=4, n_at_range=(5, 40), nrad_range=(30, 60),
                   nang_choices=(110, 146, 194, 230, 266, 302), p_max=300, p_min=50, accel=None):
    """Many independent small H/C/N/O molecules integrated together."""
    rng_g = rng_for(workload_index, PURPOSE_GEOMETRY)
    rng_b = rng_for(workload_index, PURPOSE_BASIS)
    radials, species = chno_species(rng_b)
    systems = []
    grids = []
    for _ in range(n_mol):
        n = int(rng_g.integers(n_at_range[0], n_at_range[1] + 1))
        elems, pos = random_cluster(rng_g, n)
        sp_of = {"H": 0, "C": 1, "N": 2, "O": 3}
        systems.append((np.array([sp_of[e] for e in elems], dtype=np.int32), pos * BOHR_PER_ANG))
        grids.append((int(rng_g.integers(nrad_range[0], nrad_range[1] + 1)),
                      int(nang_choices[int(rng_g.integers(0, len(nang_choices)))])))
    # per-molecule grid sizes: build each system separately then merge
    parts = [build_problem("mol", radials, species, [systems[m]], (lambda sp, g=grids[m]: g),
                           workload_index * 1000 + m, (p_max, p_min, None), accel=accel)
             for m in range(n_mol)]
    return merge_problems("many%d" % n_mol, parts, workload_index)


def merge_problems(name, parts, workload_index):
    atom_off = [0]
    boff = [0]
    sp, xyz, pts, w, v, bsys, own, shell, rgrid = [], [], [], [], [], [], [], [], []
    for s, p in enumerate(parts):
        if p.owner is not None:
            own.append(p.owner + atom_off[-1])
            shell.append(p.shell)
            rgrid.append(p.atom_rgrid)
        sp.append(p.atom_species)
        xyz.append(p.atom_xyz)
        atom_off.append(atom_off[-1] + len(p.atom_species))
        pts.append(p.pts)
        w.append(p.w)
        v.append(p.v)
        for b in range(p.n_batch):
            boff.append(boff[-1] + int(p.batch_off[b + 1] - p.batch_off[b]))
            bsys.append(s)
    p0 = parts[0]
    return Problem(name, p0.radials, p0.species, np.array(atom_off, dtype=np.int64),
                   np.concatenate(sp).astype(np.int32), np.concatenate(xyz), np.concatenate(pts),
                   np.concatenate(w), np.array(boff, dtype=np.int64),
                   np.array(bsys, dtype=np.int32), np.concatenate(v), workload_index,
                   **(dict(owner=np.concatenate(own).astype(np.int32), shell=np.concatenate(shell),
                           atom_rgrid=np.concatenate(rgrid)) if len(own) == len(parts) else {}))


# --------------------------------------------------------------------------
# matrices that enter the method as inputs
# --------------------------------------------------------------------------

def occupied_orbitals(n_fn: int, n_occ: int, rng: np.random.Generator):
    """C: the first n_occ columns of a seeded orthonormal matrix (QR of a
    Gaussian matrix, signs fixed by R's diagonal)."""
    q, r = np.linalg.qr(rng.standard_normal((n_fn, n_occ)))
    return q * np.sign(np.diag(r))[None, :]


def density_matrix_occ(n_fn: int, n_occ: int, rng: np.random.Generator, occ: float = 2.0):
    """D = occ * C C^T, C = first n_occ columns of a seeded orthonormal matrix."""
    q = occupied_orbitals(n_fn, n_occ, rng)
    return occ * (q @ q.T), q


def density_values_occ(n_fn: int, n_occ: int, rows, cols, rng: np.random.Generator, occ: float = 2.0,
                       accel=None, chunk_bytes: int = 1 << 30, q=None):
    """The stored values D[rows, cols] of D = occ C C^T (C as in
    density_matrix_occ) without forming the dense n x n matrix; the row
    dot products run with torch on `accel` when given.  q: C itself, when
    the caller already drew it (rng is then unused)."""
    if q is None:
        q = occupied_orbitals(n_fn, n_occ, rng)
    chunk = max(1, chunk_bytes // (8 * max(1, n_occ)))
    out = np.empty(len(rows))
    if accel is not None:
        import torch
        dev = _torch_device(accel)
        qt = torch.from_numpy(q).to(dev)
        rt = torch.from_numpy(np.asarray(rows, dtype=np.int64)).to(dev)
        ct = torch.from_numpy(np.asarray(cols, dtype=np.int64)).to(dev)
        res = torch.empty(len(rows), dtype=torch.float64, device=dev)
        for k0 in range(0, len(rows), chunk):
            k1 = min(len(rows), k0 + chunk)
            res[k0:k1] = occ * (qt[rt[k0:k1]] * qt[ct[k0:k1]]).sum(dim=1)
        return res.cpu().numpy()
    for k0 in range(0, len(rows), chunk):
        k1 = min(len(rows), k0 + chunk)
        out[k0:k1] = occ * np.einsum("ij,ij->i", q[rows[k0:k1]], q[cols[k0:k1]])
    return out


def random_symmetric(n: int, rng: np.random.Generator, scale: float = 1.0):
    x = rng.standard_normal((n, n)) * scale
    return 0.5 * (x + x.T)


def workload(name: str, **kw) -> Problem:
    if name == "tiny":
        return tiny_water(**kw)
    if name == "si64":
        return si64(**kw)
    if name.startswith("chno"):
        return chno_cluster(**kw)
    if name.startswith("many"):
        return many_molecules(**kw)
    raise ValueError(name)

"""FP64 CPU oracle for NAO real-space grid integration (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It never serves the product path and
shares no code with the CUDA library: the arithmetic lives in
``fgi_oracle.c`` (plain loops, FP64, OpenMP over points) and this module
only marshals arguments.

Functions follow the textbook definitions of the method whose numerical core
the paper names ("Development Priorities": numeric atom-centred orbitals on
real-space integration grids):

* ``phi``      -- phi_i(r) = u_i(d)/d Y_lm(d/|d|), and its gradient
* ``h_matrix`` -- H_ij = sum_p w_p v_p phi_i phi_j   (S: v = 1)
* ``h_pairs``  -- the same for listed (i, j) pairs
* ``density``  -- n_p = sum_ij phi_i D_ij phi_j
* ``adjoint``  -- dL/dv_p and dL/dR_a for L = sum_ij G_ij H_ij (grid fixed)
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fgi_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Basis(C.Structure):
    _fields_ = [("n_atoms", C.c_int), ("atom_xyz", C.c_void_p),
                ("n_fn", C.c_int), ("fn_atom", C.c_void_p), ("fn_rad", C.c_void_p),
                ("fn_m", C.c_void_p), ("n_rad", C.c_int), ("rad_l", C.c_void_p),
                ("rad_nk", C.c_void_p), ("rad_h", C.c_void_p), ("rad_off", C.c_void_p),
                ("coef", C.c_void_p)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P = C.c_void_p
            I64 = C.c_int64
            lib.orc_phi.argtypes = [P, I64, P, C.c_int, P, P, P]
            lib.orc_h.argtypes = [P, I64, P, P, P, C.c_int, P, P]
            lib.orc_h.restype = C.c_int
            lib.orc_h_pairs.argtypes = [P, I64, P, P, P, I64, P, P, P]
            lib.orc_density.argtypes = [P, I64, P, C.c_int, P, P, P]
            lib.orc_density.restype = C.c_int
            lib.orc_adjoint.argtypes = [P, I64, P, P, P, C.c_int, P, P, P, P]
            lib.orc_adjoint.restype = C.c_int
            lib.orc_num_threads.restype = C.c_int
            lib.orc_set_num_threads.argtypes = [C.c_int]
            _lib = lib
    return _lib


def num_threads() -> int:
    return int(_load().orc_num_threads())


def set_num_threads(n: int) -> None:
    """Threads of the oracle's later parallel loops (timing baselines only)."""
    _load().orc_set_num_threads(int(n))


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


class Basis:
    """Basis-function table of one system, expanded from species and radials.

    Functions are numbered atom by atom; within an atom, radial shell by
    shell in the species' order, and within a shell m = -l..l.
    """

    def __init__(self, radials, species, atom_species, atom_xyz):
        self.atom_xyz = np.ascontiguousarray(atom_xyz, dtype=np.float64)
        fa, fr, fm = [], [], []
        self.atom_fn0 = []
        for a, sp in enumerate(atom_species):
            self.atom_fn0.append(len(fa))
            for r in species[int(sp)].radial_ids:
                l = radials[r].l
                for m in range(-l, l + 1):
                    fa.append(a)
                    fr.append(r)
                    fm.append(m)
        self.fn_atom = np.asarray(fa, dtype=np.int32)
        self.fn_rad = np.asarray(fr, dtype=np.int32)
        self.fn_m = np.asarray(fm, dtype=np.int32)
        self.rad_l = np.asarray([r.l for r in radials], dtype=np.int32)
        self.rad_nk = np.asarray([r.n_knots for r in radials], dtype=np.int32)
        self.rad_h = np.asarray([r.h for r in radials], dtype=np.float64)
        sizes = [r.coef.shape[0] for r in radials]
        self.rad_off = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
        self.coef = np.ascontiguousarray(np.concatenate([r.coef for r in radials]), dtype=np.float64)
        self.rad_cut = self.rad_h * (self.rad_nk - 1)
        self._s = _Basis(len(self.atom_xyz), _p(self.atom_xyz).value, len(self.fn_atom),
                         _p(self.fn_atom).value, _p(self.fn_rad).value, _p(self.fn_m).value,
                         len(radials), _p(self.rad_l).value, _p(self.rad_nk).value,
                         _p(self.rad_h).value, _p(self.rad_off).value, _p(self.coef).value)

    @property
    def n_fn(self) -> int:
        return len(self.fn_atom)

    def ref(self):
        return C.byref(self._s)

    def fn_cut(self):
        return self.rad_cut[self.fn_rad]


def system_basis(problem, s: int = 0) -> Basis:
    a0, a1 = int(problem.atom_off[s]), int(problem.atom_off[s + 1])
    return Basis(problem.radials, problem.species, problem.atom_species[a0:a1],
                 problem.atom_xyz[a0:a1])


def _sub(basis, sub):
    if sub is None:
        sub = np.arange(basis.n_fn)
    return np.ascontiguousarray(sub, dtype=np.int32)


def phi(basis: Basis, pts, sub=None, grad=False):
    lib = _load()
    pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
    sub = _sub(basis, sub)
    out = np.empty((len(pts), len(sub)))
    g = np.empty((len(pts), len(sub), 3)) if grad else None
    lib.orc_phi(basis.ref(), len(pts), _p(pts), len(sub), _p(sub), _p(out), _p(g))
    return (out, g) if grad else out


def h_matrix(basis: Basis, pts, w, v=None, sub=None):
    lib = _load()
    pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
    w = np.ascontiguousarray(w, dtype=np.float64)
    v = None if v is None else np.ascontiguousarray(v, dtype=np.float64)
    sub = _sub(basis, sub)
    H = np.empty((len(sub), len(sub)))
    rc = lib.orc_h(basis.ref(), len(pts), _p(pts), _p(w), _p(v), len(sub), _p(sub), _p(H))
    if rc != 0:
        raise MemoryError("oracle: out of host memory")
    return H


def h_pairs(basis: Basis, pts, w, v, pi, pj):
    lib = _load()
    pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
    w = np.ascontiguousarray(w, dtype=np.float64)
    v = None if v is None else np.ascontiguousarray(v, dtype=np.float64)
    pi = np.ascontiguousarray(pi, dtype=np.int32)
    pj = np.ascontiguousarray(pj, dtype=np.int32)
    out = np.empty(len(pi))
    lib.orc_h_pairs(basis.ref(), len(pts), _p(pts), _p(w), _p(v), len(pi), _p(pi), _p(pj), _p(out))
    return out


def density(basis: Basis, pts, D, sub=None):
    lib = _load()
    pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
    sub = _sub(basis, sub)
    D = np.ascontiguousarray(D, dtype=np.float64)
    assert D.shape == (len(sub), len(sub))
    out = np.empty(len(pts))
    rc = lib.orc_density(basis.ref(), len(pts), _p(pts), len(sub), _p(sub), _p(D), _p(out))
    if rc != 0:
        raise MemoryError("oracle: out of host memory")
    return out


def adjoint(basis: Basis, pts, w, v, G, sub=None):
    lib = _load()
    pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
    w = np.ascontiguousarray(w, dtype=np.float64)
    v = np.ascontiguousarray(v, dtype=np.float64)
    sub = _sub(basis, sub)
    G = np.ascontiguousarray(G, dtype=np.float64)
    dv = np.empty(len(pts))
    dR = np.empty((len(basis.atom_xyz), 3))
    rc = lib.orc_adjoint(basis.ref(), len(pts), _p(pts), _p(w), _p(v), len(sub), _p(sub),
                         _p(G), _p(dv), _p(dR))
    if rc != 0:
        raise MemoryError("oracle: out of host memory")
    return dv, dR


def active_functions(basis: Basis, pts) -> np.ndarray:
    """Indices of the functions that are non-zero at some point of pts."""
    pts = np.asarray(pts).reshape(-1, 3)
    cut = basis.fn_cut()
    out = []
    for a in range(len(basis.atom_xyz)):
        fns = np.nonzero(basis.fn_atom == a)[0]
        d = np.linalg.norm(pts - basis.atom_xyz[a][None, :], axis=1)
        for f in fns:
            if np.any(d < cut[f]):
                out.append(f)
    return np.asarray(out, dtype=np.int32)

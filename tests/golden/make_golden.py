"""Writes the regression fixtures of this folder from the FP64 oracle.

The paper prints no worked example for grid integration, so these files are
not the paper's values: they freeze what the oracle (`oracle/`) computes on
small seeded inputs, so that an unintended change of the oracle's arithmetic
shows up as a test failure.  Only `oracle` and `workloads` are called.

    python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
import workloads as W  # noqa: E402


def water_case():
    """Water, 16 radial x 26 angular points per atom (the small grid of the
    host tests), H = sum w v phi phi and S (v = 1), and the density of the
    S-orthonormal occupied orbitals (5 doubly occupied)."""
    prob = W.tiny_water(n_rad=16, n_ang=26)
    B = O.system_basis(prob)
    H = O.h_matrix(B, prob.pts, prob.w, prob.v)
    S = O.h_matrix(B, prob.pts, prob.w)
    rng = W.rng_for(0, W.PURPOSE_D)
    q, _ = np.linalg.qr(rng.standard_normal((B.n_fn, 5)))
    ev, U = np.linalg.eigh(S)
    C = U @ np.diag(ev ** -0.5) @ U.T @ q
    D = 2.0 * C @ C.T
    n = O.density(B, prob.pts, D)
    return prob, H, S, D, n


def write(path, header, arrays):
    with open(path, "w") as f:
        f.write("# " + header.replace("\n", "\n# ") + "\n")
        for name, a in arrays:
            a = np.atleast_1d(np.asarray(a, dtype=np.float64))
            f.write("%s %s\n" % (name, " ".join(str(d) for d in a.shape)))
            for x in a.ravel():
                f.write("%.17e\n" % x)


def read(path):
    out = {}
    with open(path) as f:
        lines = [ln for ln in f if not ln.startswith("#")]
    i = 0
    while i < len(lines):
        parts = lines[i].split()
        name, shape = parts[0], tuple(int(x) for x in parts[1:])
        size = int(np.prod(shape))
        out[name] = np.array([float(x) for x in lines[i + 1:i + 1 + size]]).reshape(shape)
        i += 1 + size
    return out


if __name__ == "__main__":
    prob, H, S, D, n = water_case()
    write(os.path.join(HERE, "water_16x26_oracle.txt"),
          "Regression fixture (not a value from the paper): the FP64 oracle on water,\n"
          "16 radial x 26 angular points per atom, written by tests/golden/make_golden.py.\n"
          "H_ij = sum_p w_p v_p phi_i phi_j, S with v = 1 (definitions of the method's\n"
          "grid integration); n = density of D = 2 C C^T with S-orthonormal C.",
          [("H", H), ("S", S), ("D", D), ("n_first16", n[:16]), ("n_points", [prob.n_pts])])
    print("written")

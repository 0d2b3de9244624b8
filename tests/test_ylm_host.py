"""The library's real spherical harmonics for the Hartree multipoles
(csrc/fgi_ylm.cuh, a recurrence), pinned on the CPU through a small C++
driver: the addition theorem sum_m Y_lm(a) Y_lm(b) = (2l+1)/(4 pi) P_l(a.b)
(normalisation and completeness of each l), and |Y_lm| against scipy's
harmonics (the sign convention of the real basis is immaterial for the
potential)."""
import math
import os
import shutil
import subprocess

import numpy as np
import pytest
from scipy.special import eval_legendre

import oracle.hartree as OH

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LMAX = 6


@pytest.fixture(scope="module")
def ylm(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path_factory.mktemp("ylm") / "ylm_check")
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", os.path.join(ROOT, "paper_2208_12335_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "ylm_check.cpp"), "-o", exe], check=True, capture_output=True)

    def run(dirs):
        txt = "\n".join("%.17g %.17g %.17g" % tuple(d) for d in dirs)
        out = subprocess.run([exe], input=txt, capture_output=True, text=True, check=True).stdout
        return np.array([[float(v) for v in line.split()] for line in out.strip().splitlines()])
    return run


def unit(n, seed):
    d = np.random.default_rng(seed).standard_normal((n, 3))
    d = np.concatenate([d, [[0, 0, 1.0], [0, 0, -1.0], [1.0, 0, 0]]])
    return d / np.linalg.norm(d, axis=1, keepdims=True)


def test_addition_theorem(ylm):
    a, b = unit(40, 1), unit(40, 2)
    Ya, Yb = ylm(a), ylm(b)
    cosg = np.sum(a * b, axis=1)
    for l in range(LMAX + 1):
        s = slice(l * l, (l + 1) * (l + 1))
        lhs = np.sum(Ya[:, s] * Yb[:, s], axis=1)
        rhs = (2 * l + 1) / (4 * math.pi) * eval_legendre(l, cosg)
        np.testing.assert_allclose(lhs, rhs, rtol=0, atol=1e-13)


def test_magnitudes_match_scipy(ylm):
    d = unit(60, 3)
    np.testing.assert_allclose(np.abs(ylm(d)), np.abs(OH.real_ylm(LMAX, d)), rtol=0, atol=1e-13)

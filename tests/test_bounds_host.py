"""The table bounds of |phi| used for the leading-digit grids without a pass
over the points (CPU).

A small C++ program prints what paper_2208_12335_gb300/csrc/fgi_bounds.h
computes; the checks sample the functions densely: max |Y_lm| against the
real spherical harmonics written out independently (tests/helpers.py), and
the suffix bounds of |u(r)/r| against the splines of the water, Si64 and
C/H/N/O workloads and against random cubics: never below a sample, within
0.1 % of the sampled suffix maxima, non-increasing."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import workloads as W
from tests import helpers as T

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    out = str(tmp_path_factory.mktemp("bounds") / "bounds_check")
    subprocess.run([cxx, "-std=c++17", "-O1", "-Wall", "-Wextra", "-Werror",
                    "-I", os.path.join(ROOT, "paper_2208_12335_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "bounds_check.cpp"), "-o", out],
                   check=True, capture_output=True, text=True)
    return out


def radial_bounds(exe, coef, h):
    txt = "%d %.17g\n" % (len(coef), h) + "\n".join("%.17g" % c for c in np.ravel(coef))
    out = subprocess.run([exe, "radial"], input=txt, capture_output=True, text=True, check=True)
    return np.array([float(x) for x in out.stdout.split()])


def test_ylm_maxima_bound_the_harmonics_tightly(exe):
    out = subprocess.run([exe, "ylm"], capture_output=True, text=True, check=True)
    tab = np.array([float(x) for x in out.stdout.split()])
    rng = np.random.default_rng(0)
    g = rng.standard_normal((400000, 3))
    g /= np.linalg.norm(g, axis=1, keepdims=True)
    for l in range(4):
        for m in range(-l, l + 1):
            sampled = np.abs(T.real_sph_harm(l, m, g)).max()
            t = tab[l * l + l + m]
            assert sampled <= t, (l, m, sampled, t)
            assert t <= sampled * 1.004, (l, m, sampled, t)


def check_radial(exe, coef, h):
    b = radial_bounds(exe, coef, h)
    n = len(coef)
    assert np.all(np.diff(b) <= 0)                                   # suffix maxima
    t = np.linspace(0.0, 1.0, 65)
    u = coef[:, :1] + t * (coef[:, 1:2] + t * (coef[:, 2:3] + t * coef[:, 3:4]))   # (n, 65)
    r = (np.arange(n)[:, None] + t) * h
    with np.errstate(divide="ignore", invalid="ignore"):
        f = np.abs(u) / r
    f[0, 0] = abs(coef[0, 1]) / h                                    # the limit u'(0) at r = 0
    per_int = f.max(axis=1)
    suffix = np.maximum.accumulate(per_int[::-1])[::-1]
    assert np.all(suffix <= b * (1 + 1e-7)), np.max(suffix / b)
    # tight: the exact interval maxima differ from 65 samples per interval
    # by the curvature between samples only; values below the FP32 range
    # round up to its smallest number
    ok = suffix > 1e-30
    assert np.all(b[ok] <= suffix[ok] * 1.001)


@pytest.mark.parametrize("which", ["water", "si64", "chno"])
def test_radial_bounds_on_the_workload_splines(exe, which):
    if which == "water":
        radials = W.tiny_water(n_rad=8, n_ang=14).radials
    elif which == "si64":
        rng = W.rng_for(1, W.PURPOSE_BASIS)
        rc = 6.0 * W.BOHR_PER_ANG
        specs = W._seeded_radials(rng, [0, 0, 0, 0, 0, 0, 1, 1, 1, 2, 2], rc, rc - W.BOHR_PER_ANG, 2000,
                                  W.SI_ALPHA)
        radials = [W.make_radial(s) for s in specs]
    else:
        radials, _ = W.chno_species(W.rng_for(2, W.PURPOSE_BASIS))
    for rad in radials:
        assert rad.coef[0, 0] == 0.0                                 # u(0) = 0
        check_radial(exe, rad.coef, rad.h)


def test_radial_bounds_on_random_cubics(exe):
    rng = np.random.default_rng(3)
    for _ in range(20):
        n = int(rng.integers(2, 60))
        coef = rng.standard_normal((n, 4))
        coef[0, 0] = 0.0
        check_radial(exe, coef, float(rng.uniform(0.01, 0.5)))
    # u(0) != 0: the ratio is unbounded at the origin, the whole suffix is infinite
    coef = rng.standard_normal((5, 4))
    coef[0, 0] = 0.3
    b = radial_bounds(exe, coef, 0.1)
    assert np.isinf(b[0]) and np.all(np.isfinite(b[1:]))

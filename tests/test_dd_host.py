"""The double-float reciprocal square root of the basis kernels
(csrc/fgi_dd.cuh, df_rsqrt_refine), pinned on the CPU through a small C++
driver against long double: one refinement of an FP32 approximation with a
relative error up to 2^-22 (rsqrtf's 2 ulp) gives 1/sqrt(a) within 2^-42,
and within 2^-40 from a start as poor as 2^-20; sqrt(a) = a (1/sqrt(a)) as a
double-float product keeps the same accuracy.  The kernels need far less
(their values are split into about 24 bits), but an error that is the same
for every point of a radial shell must stay far below FP32 rounding."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_rsqrt_refinement_against_long_double(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
    if not os.path.exists(os.path.join(cuda_inc, "cuda_runtime.h")):
        pytest.skip("no CUDA headers")
    exe = str(tmp_path / "dd_check")
    # no FMA contraction on the host: the refinement's error-free products
    # are written with explicit fmaf
    subprocess.run([cxx, "-std=c++17", "-O1", "-ffp-contract=off",
                    "-I", os.path.join(ROOT, "paper_2208_12335_gb300", "csrc"), "-I", cuda_inc,
                    os.path.join(ROOT, "tests", "dd_check.cpp"), "-o", exe], check=True, capture_output=True)
    out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    worst_real, worst_all, worst_sqrt = (float(v) for v in out)
    assert worst_real < 2.0 ** -42
    assert worst_all < 2.0 ** -40
    assert worst_sqrt < 2.0 ** -40

"""The C ABI from a plain C99 program (CPU, host-only context).

tests/c_abi_host.c includes only include/fgi.h and links only libfgi.so:
no Python, no torch types.  It is compiled with gcc -Werror and run; it
checks sizes, pattern, batch work (including an empty batch and a batch
beyond every cutoff), the schedule query and the error paths."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libdir():
    from paper_2208_12335_gb300 import build as B
    B.build()
    import paper_2208_12335_gb300 as P
    return os.path.dirname(P.LIB_PATH)


def test_c_program_drives_the_host_side_of_the_abi(libdir, tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    exe = str(tmp_path / "c_abi_host")
    cmd = [cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-O1", "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "c_abi_host.c"), "-o", exe, "-L", libdir, "-lfgi",
           "-Wl,-rpath," + libdir, "-lm"]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stderr
    assert out.stdout.strip() == "C ABI OK"

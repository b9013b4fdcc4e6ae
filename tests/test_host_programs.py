"""The kernels' instruction streams, walked on the host exactly as the kernels walk them.

tests/host/*.cpp build the tables with the library's own builder (tables.cpp), check every
index the kernels would dereference against its array, and evaluate Q by following the
program (angular-first: slices, rank-1 groups, symmetrised core; radial-first: blocks of q2
groups, the union of their q3 with packed targets) against the direct sum over the COO
entries (the full discrete sum of Sec. 4.5) on random cores and cells, to 1e-12.  No GPU."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(os.path.dirname(HERE), "paper_2605_28475_gb300", "csrc", "tables.cpp")


@pytest.mark.parametrize("name", ["angular_program_check", "radial_program_check"])
def test_program_walk(name, tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path / name)
    subprocess.run([gxx, "-O2", "-std=c++17", "-o", exe, os.path.join(HERE, "host", name + ".cpp"), SRC], check=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and "bad=0" in r.stdout, r.stdout[-2000:]

"""Host check (no GPU) of the neighbour step's face tables.

`tests/host/ftab_check.cu` is compiled for the host with nvcc (the table builder and the general
boundary resolution are __host__ __device__) and checks, for every face cell of small lattices with
solids under seven combinations of inflow, outflow, periodic, no-slip and free-slip faces, that the
table keeps the resolver's scatter targets (App. D, Sec. 3 boundaries) except an equilibrium cell's
targets in other equilibrium cells, which it drops (an equilibrium cell never reads what it
receives), and that the plain bit marks exactly the single plain downstream target.
"""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.skipif(shutil.which("nvcc") is None, reason="needs nvcc")
def test_face_tables_match_the_general_resolution():
    src = os.path.join(ROOT, "tests", "host", "ftab_check.cu")
    with tempfile.TemporaryDirectory() as td:
        exe = os.path.join(td, "ftab_check")
        subprocess.run(["nvcc", "-std=c++17", "-O1", "-x", "cu", "-gencode", "arch=compute_103a,code=sm_103a",
                        "-I", os.path.join(ROOT, "include"), "-I", os.path.join(ROOT, "paper_2607_04516_b300", "csrc"),
                        src, "-o", exe], check=True, capture_output=True)
        out = subprocess.run([exe], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout[-2000:]
    assert "all face-table checks passed" in out.stdout
    assert out.stdout.count("tables match the resolution") == 21

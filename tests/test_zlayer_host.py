"""Host check (no GPU) of the neighbour step's ground / top layer path in the lattice blocks.

`tests/host/zlayer_check.cu` is compiled for the host with nvcc (the cell bodies are
__host__ __device__) and compares, for every layer cell of small lattices with solids in and next to
both layers, the storage elements the layer path gathers from and scatters to with those of the
general boundary resolution (halfway bounce-back at a no-slip face, specular reflection at a
free-slip face, store-side bounce-back next to solids; R8 of the boundary rules, App. D), for every
no-slip / free-slip combination of the two z faces.
"""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.skipif(shutil.which("nvcc") is None, reason="needs nvcc")
def test_layer_path_elements_match_general_resolution():
    src = os.path.join(ROOT, "tests", "host", "zlayer_check.cu")
    with tempfile.TemporaryDirectory() as td:
        exe = os.path.join(td, "zlayer_check")
        subprocess.run(["nvcc", "-std=c++17", "-O1", "-x", "cu", "-gencode", "arch=compute_103a,code=sm_103a",
                        "-I", os.path.join(ROOT, "include"), "-I", os.path.join(ROOT, "paper_2607_04516_b300", "csrc"),
                        src, "-o", exe], check=True, capture_output=True)
        out = subprocess.run([exe], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout[-2000:]
    assert "all layer-path checks passed" in out.stdout
    assert out.stdout.count("match the general resolution") == 64

"""Host emulation (no GPU) of the neighbour step's ground / top lattice blocks under
AddressSanitizer.

`tests/host/layer_emul.cu` runs the layer-path body (neighbor_layer_unit: the static rules of a
block wholly in the ground or top layer, the per-cell form for blocks across a layer boundary) of
every thread of every such block, for 16-bit and FP32 storage and the block sizes of the single
and batched launches, on a buffer laid out as the device workspace; AddressSanitizer aborts on any
access outside it and canaries catch writes into its guards (App. D streaming with the boundary
rules of Sec. 3).
"""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.skipif(shutil.which("nvcc") is None, reason="needs nvcc")
def test_layer_blocks_stay_in_bounds():
    src = os.path.join(ROOT, "tests", "host", "layer_emul.cu")
    with tempfile.TemporaryDirectory() as td:
        exe = os.path.join(td, "layer_emul")
        subprocess.run(["nvcc", "-std=c++17", "-O2", "-x", "cu", "-gencode", "arch=compute_103a,code=sm_103a",
                        "-I", os.path.join(ROOT, "include"), "-I", os.path.join(ROOT, "paper_2607_04516_b300", "csrc"),
                        "-Xcompiler", "-fsanitize=address", "-Xcompiler", "-fno-omit-frame-pointer", "-Xlinker", "-lasan",
                        src, "-o", exe], check=True, capture_output=True)
        env = dict(os.environ, ASAN_OPTIONS="detect_leaks=0")
        out = subprocess.run([exe], capture_output=True, text=True, env=env)
    assert out.returncode == 0, (out.stdout[-1500:], out.stderr[-3000:])
    assert "all layer-block emulations in bounds" in out.stdout

"""Build ``liblbm.so`` (the C-ABI library) in-tree for sm_103a with nvcc.

    python -m paper_2607_04516_b300.build [--force]
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(PKG, "liblbm.so")
# (source, defines): the step and batched kernels are compiled once per storage type (and forcing),
# so that their template instantiations build in parallel
_STORES = ("LBM_F32", "LBM_F16S", "LBM_BF16S")
UNITS = ([(os.path.join(CSRC, f), ()) for f in ("lbm_kernels.cu", "lbm_capi.cu", "lbm_noalloc.cu", "lbm_stg.cu",
                                                 "lbm_adjoint.cu", "lbm_batch.cu")]
         + [(os.path.join(CSRC, "lbm_step_kern.cu"), (f"LBM_INST_S={st}", f"LBM_INST_FORCE={fo}"))
            for st in _STORES for fo in (0, 1)]
         + [(os.path.join(CSRC, "lbm_batch_kern.cu"), (f"LBM_INST_S={st}",)) for st in _STORES])
SOURCES = sorted({src for src, _ in UNITS})
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _inputs():
    return (SOURCES + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h"))
            + glob.glob(os.path.join(INCLUDE, "*.h")))


def stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(p) > t for p in _inputs())


def build(force: bool = False, verbose: bool = False, out: str | None = None,
          defines: tuple = ()) -> str:
    """Compile the library (to ``out`` instead of the in-tree path when given, e.g. to compare
    launch-bound variants passed as ``defines``): one nvcc process per compilation unit in parallel
    (objects in a private temporary folder), then one link."""
    import concurrent.futures
    import shutil
    import tempfile
    target = out or LIB
    if out is None and not force and not stale():
        return LIB
    nvcc = os.environ.get("NVCC", "nvcc")
    tmp = target + f".tmp{os.getpid()}"
    flags = ["-O3", "-std=c++17", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC",
             *[f"-D{d}" for d in defines], "-I", INCLUDE]
    if verbose:
        flags.insert(0, "-Xptxas=-v")
    objdir = tempfile.mkdtemp(prefix="lbm_build_")
    try:
        objs = [os.path.join(objdir, f"{k:02d}_" + os.path.basename(src) + ".o") for k, (src, _) in enumerate(UNITS)]

        def compile_one(k):
            src, unit_defs = UNITS[k]
            cmd = [nvcc, *flags, *[f"-D{d}" for d in unit_defs], "-c", src, "-o", objs[k]]
            if verbose:
                print(" ".join(cmd), flush=True)
            subprocess.run(cmd, check=True)

        # longest units first
        order = sorted(range(len(UNITS)), key=lambda k: "kern" not in UNITS[k][0])
        with concurrent.futures.ThreadPoolExecutor(max_workers=min(len(UNITS), os.cpu_count() or 4)) as ex:
            list(ex.map(compile_one, order))
        subprocess.run([nvcc, *ARCH, "-shared", *objs, "-o", tmp], check=True)
    finally:
        shutil.rmtree(objdir, ignore_errors=True)
    os.replace(tmp, target)
    return target


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)

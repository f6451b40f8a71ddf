"""B300-native (sm_103a) LBM-LES urban-wind step: D3Q19 BGK + Smagorinsky, in-place streaming,
halfway bounce-back, equilibrium inflow and zero-gradient outflow, fused in one kernel per step.

``paper_2607_04516_b300.lbm``    thin ctypes binding to the C-ABI library ``liblbm.so``
``paper_2607_04516_b300.synth``  seeded synthetic inputs (geometry, inflow levels, fields)
``paper_2607_04516_b300.build``  nvcc build of the library for sm_103a

Importing the package loads nothing native; ``lbm`` loads the library on first use and raises if
it is missing or if no CUDA device is present.
"""
__all__ = ["lbm", "synth", "build"]

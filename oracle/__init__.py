"""FP64 CPU oracle for the LBM-LES step -- test infrastructure, never part of the product path.

``oracle.oracle``     ctypes wrapper around the C/OpenMP reference (``lbm_oracle.c``).
``oracle.lbm_numpy``  an independently written NumPy formulation for tiny cross-check grids.
"""

"""FP64 CPU oracle -- Python wrapper around ``lbm_oracle.c`` (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
this module.  The product library (``paper_2607_04516_b300``) never imports it and has no path
that falls back to it.

Array conventions (all float64, C-contiguous):
    F     (19, nz, ny, nx)   post-collision populations, oracle direction order (``lattice()``)
    kind  (nz, ny, nx) u8    0 fluid, 1 solid, 2 equilibrium-boundary cell
    ub    (nz, 3)            equilibrium-boundary velocity per cell height
    u     (nz, ny, nx, 3)    velocity
Face kinds are given by name, in the order x-, x+, y-, y+, z-, z+:
    'periodic' | 'inflow' | 'outflow' | 'freeslip' | 'noslip'

The paper passages each function follows are cited in ``lbm_oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")

FACE_CODES = {"periodic": 0, "inflow": 1, "outflow": 2, "freeslip": 3, "noslip": 4}
FLUID, SOLID, EQ = 0, 1, 2

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc + OpenMP into ``oracle/_build/liboracle.so``."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        I = ctypes.c_int
        D = ctypes.c_double
        L.oracle_lattice.argtypes = [P, P, P]
        L.oracle_lattice.restype = I
        L.oracle_equilibrium.argtypes = [D, P, P]
        L.oracle_equilibrium.restype = None
        L.oracle_tau_eff.argtypes = [D, D, D, D]
        L.oracle_tau_eff.restype = D
        L.oracle_collide.argtypes = [P, D, D, P, P, P, P]
        L.oracle_collide.restype = None
        L.oracle_collide_rot.argtypes = [P, D, D, P, P, P, P, P]
        L.oracle_collide_rot.restype = None
        L.oracle_classify.argtypes = [P, I, I, I, P, P]
        L.oracle_classify.restype = I
        L.oracle_expand_profile.argtypes = [P, I, I, D, P]
        L.oracle_expand_profile.restype = I
        L.oracle_init.argtypes = [P, P, I, I, I, P, P, P, D, P]
        L.oracle_init.restype = I
        L.oracle_step.argtypes = [P, P, P, I, I, I, P, P, D, D, D, P, I, I, P, P, P, P]
        L.oracle_step.restype = I
        L.oracle_macros.argtypes = [P, P, I, I, I, P, D, P, P, P, P]
        L.oracle_macros.restype = I
        L.oracle_stg.argtypes = [P, I, I, I, P, P, P, P, ctypes.c_longlong, P]
        L.oracle_stg.restype = I
        L.oracle_num_threads.argtypes = []
        L.oracle_num_threads.restype = I
        _lib = L
    return _lib


def _p(a: np.ndarray | None):
    return None if a is None else a.ctypes.data


def _faces(faces) -> np.ndarray:
    return np.array([FACE_CODES[f] for f in faces], dtype=np.int32)


def lattice():
    """(c (19,3) int, w (19,) float, opp (19,) int) in the oracle's direction order."""
    c = np.zeros((19, 3), np.int32)
    w = np.zeros(19, np.float64)
    opp = np.zeros(19, np.int32)
    lib().oracle_lattice(_p(c), _p(w), _p(opp))
    return c.astype(np.int64), w, opp.astype(np.int64)


def equilibrium(rho: float, u) -> np.ndarray:
    u = np.ascontiguousarray(u, np.float64)
    out = np.zeros(19, np.float64)
    lib().oracle_equilibrium(float(rho), _p(u), _p(out))
    return out


def tau_eff(tau: float, C: float, Q: float, rho: float) -> float:
    return lib().oracle_tau_eff(float(tau), float(C), float(Q), float(rho))


def collide(f, tau: float, C: float, force=None, omega=None):
    """One-cell collision; returns (f*, Q, tau_eff).  ``omega``: Coriolis rotation vector."""
    f = np.ascontiguousarray(f, np.float64)
    out = np.zeros(19, np.float64)
    q = ctypes.c_double()
    te = ctypes.c_double()
    fz = None if force is None else np.ascontiguousarray(force, np.float64)
    om = None if omega is None else np.ascontiguousarray(omega, np.float64)
    lib().oracle_collide_rot(_p(f), float(tau), float(C), _p(fz), _p(om), _p(out),
                             ctypes.addressof(q), ctypes.addressof(te))
    return out, q.value, te.value


def classify(solid: np.ndarray, faces) -> np.ndarray:
    solid = np.ascontiguousarray(solid, np.uint8)
    nz, ny, nx = solid.shape
    kind = np.zeros_like(solid)
    lib().oracle_classify(_p(solid), nx, ny, nz, _p(_faces(faces)), _p(kind))
    return kind


def expand_profile(speed, nz: int, theta: float) -> np.ndarray:
    speed = np.ascontiguousarray(speed, np.float64)
    ub = np.zeros((nz, 3), np.float64)
    rc = lib().oracle_expand_profile(_p(speed), len(speed), nz, float(theta), _p(ub))
    if rc != 0:
        raise ValueError("bad profile")
    return ub


def _opt(a):
    return None if a is None else np.ascontiguousarray(a, np.float64)


def init(kind: np.ndarray, ub: np.ndarray, rho=None, u=None, rho_b: float = 1.0,
         ueq=None) -> np.ndarray:
    nz, ny, nx = kind.shape
    F = np.zeros((19, nz, ny, nx), np.float64)
    rho = None if rho is None else np.ascontiguousarray(rho, np.float64)
    u = None if u is None else np.ascontiguousarray(u, np.float64)
    ub = np.ascontiguousarray(ub, np.float64)
    ueq = _opt(ueq)
    lib().oracle_init(_p(F), _p(np.ascontiguousarray(kind, np.uint8)), nx, ny, nz,
                      _p(rho), _p(u), _p(ub), float(rho_b), _p(ueq))
    return F


def step(F: np.ndarray, kind: np.ndarray, faces, ub: np.ndarray, tau: float, C: float,
         force=None, rho_b: float = 1.0, z0: int = 0, z1: int | None = None,
         out: np.ndarray | None = None, diag: bool = False, omega=None, ueq=None):
    """One time step (pull form).  Returns F_next, or (F_next, Q, tau_eff) if ``diag``.
    ``omega``: Coriolis rotation vector (lattice units), None = no Coriolis force.
    ``ueq``: per-cell velocity (nz, ny, nx, 3) of the equilibrium cells, None = ``ub`` by height."""
    nz, ny, nx = kind.shape
    if out is None:
        out = np.zeros_like(F)
    fz = None if force is None else np.ascontiguousarray(force, np.float64)
    q = te = None
    if diag:
        q = np.zeros((nz, ny, nx), np.float64)
        te = np.zeros((nz, ny, nx), np.float64)
    om = None if omega is None else np.ascontiguousarray(omega, np.float64)
    ue = _opt(ueq)
    lib().oracle_step(_p(F), _p(out), _p(kind), nx, ny, nz, _p(_faces(faces)),
                      _p(np.ascontiguousarray(ub, np.float64)), float(rho_b), float(tau), float(C),
                      _p(fz), int(z0), int(nz if z1 is None else z1), _p(q), _p(te), _p(om),
                      _p(ue))
    return (out, q, te) if diag else out


def run(F: np.ndarray, nsteps: int, *args, **kw) -> np.ndarray:
    """``nsteps`` steps with two ping-pong buffers; returns the final state."""
    a = F.copy()
    b = np.empty_like(F)
    for _ in range(nsteps):
        step(a, *args, out=b, **kw)
        a, b = b, a
    return a


def macros(F: np.ndarray, kind: np.ndarray, ub: np.ndarray, rho_b: float = 1.0, force=None,
           ueq=None):
    nz, ny, nx = kind.shape
    rho = np.zeros((nz, ny, nx), np.float64)
    u = np.zeros((nz, ny, nx, 3), np.float64)
    fz = None if force is None else np.ascontiguousarray(force, np.float64)
    ue = _opt(ueq)
    lib().oracle_macros(_p(F), _p(kind), nx, ny, nz, _p(np.ascontiguousarray(ub, np.float64)),
                        float(rho_b), _p(fz), _p(rho), _p(u), _p(ue))
    return rho, u


class StgParams(ctypes.Structure):
    """Parameters of the synthetic inflow turbulence (mirrors ``oracle_stg_params``)."""
    _fields_ = [("n_modes", ctypes.c_int), ("L", ctypes.c_double), ("I", ctypes.c_double),
                ("sigma0", ctypes.c_double), ("gain", ctypes.c_double * 3),
                ("char_normal", ctypes.c_int), ("inflow_only", ctypes.c_int),
                ("stride", ctypes.c_int), ("interpolate", ctypes.c_int)]


def stg_params(n_modes=64, L=20.0, I=0.1, sigma0=0.0, gain=(1.0, 1.0, 1.0), char_normal=False,
               inflow_only=False, stride=1, interpolate=True) -> StgParams:
    p = StgParams()
    p.n_modes, p.L, p.I, p.sigma0 = int(n_modes), float(L), float(I), float(sigma0)
    for a in range(3):
        p.gain[a] = float(gain[a])
    p.char_normal, p.inflow_only = int(bool(char_normal)), int(bool(inflow_only))
    p.stride, p.interpolate = int(stride), int(bool(interpolate))
    return p


def stg(kind: np.ndarray, faces, ub: np.ndarray, params: StgParams, rnd: np.ndarray,
        t: int) -> np.ndarray:
    """Velocity (nz, ny, nx, 3) of the equilibrium cells at step ``t`` with synthetic inflow
    turbulence; ``rnd`` (6, n_modes, 6) uniforms in [0, 1) per face (x-, x+, y-, y+, z-, z+) and
    mode: r, (mu + 1)/2, theta/2pi, phi_x/2pi, phi_y/2pi, phi_z/2pi.  Zero at non-EQ cells."""
    nz, ny, nx = kind.shape
    rnd = np.ascontiguousarray(rnd, np.float64)
    if rnd.shape != (6, params.n_modes, 6):
        raise ValueError("rnd must be (6, n_modes, 6)")
    out = np.zeros((nz, ny, nx, 3), np.float64)
    rc = lib().oracle_stg(_p(np.ascontiguousarray(kind, np.uint8)), nx, ny, nz,
                          _p(_faces(faces)), _p(np.ascontiguousarray(ub, np.float64)),
                          ctypes.addressof(params), _p(rnd), int(t), _p(out))
    if rc != 0:
        raise ValueError(f"oracle_stg failed ({rc})")
    return out


def num_threads() -> int:
    return lib().oracle_num_threads()

"""Second, independent FP64 formulation of the same time step (TEST INFRASTRUCTURE ONLY).

Purpose: cross-check the C oracle (``lbm_oracle.c``) on tiny grids with a differently written
program, so that an indexing slip in either one shows up as a disagreement.  Where the C oracle
resolves the upstream source of every population cell by cell, this module pads the lattice with
one ghost layer per face (periodic: wrap copy; outflow: edge copy; free-slip: edge copy with the
normal component of every population mirrored; no-slip: a wall marker), applied axis after axis
so that edges and corners compose, and then streams by plain array shifts.  The collision is
written with tensor contractions over the whole lattice.

Same paper passages as the C oracle: App. D (D.1 moments, D.2 BGK, D.3 streaming, D.4
equilibrium, D.8-D.11 Smagorinsky closure, mid-grid bounce-back), Sec. 3 (equilibrium velocity
faces), Guo forcing and the Coriolis force (App. E).  Same readings where the paper is silent.

Only for small lattices (a few thousand cells): it materialises several padded copies.
"""
from __future__ import annotations

import numpy as np

# D3Q19 velocities written out explicitly (a different order from the C oracle on purpose).
C = np.array([
    [0, 0, 0],
    [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1],
    [1, 1, 0], [-1, -1, 0], [1, -1, 0], [-1, 1, 0],
    [1, 0, 1], [-1, 0, -1], [1, 0, -1], [-1, 0, 1],
    [0, 1, 1], [0, -1, -1], [0, 1, -1], [0, -1, 1],
], dtype=np.int64)
W = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12, dtype=np.float64)
CS2 = 1.0 / 3.0


def _index_of(v) -> int:
    return int(np.nonzero((C == np.asarray(v)).all(axis=1))[0][0])


OPP = np.array([_index_of(-C[i]) for i in range(19)])
# MIRROR[a][i]: the direction whose a-component is negated
MIRROR = np.array([[_index_of(C[i] * np.where(np.arange(3) == a, -1, 1)) for i in range(19)]
                   for a in range(3)])

FLUID, SOLID, EQ = 0, 1, 2


def classify(solid: np.ndarray, faces) -> np.ndarray:
    kind = np.zeros(solid.shape, np.uint8)
    nz, ny, nx = solid.shape
    Z, Y, X = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    for a, coord, n in ((0, X, nx), (1, Y, ny), (2, Z, nz)):
        if faces[2 * a] == "inflow":
            kind[coord == 0] = EQ
        if faces[2 * a + 1] == "inflow":
            kind[coord == n - 1] = EQ
    kind[solid.astype(bool)] = SOLID
    return kind


def equilibrium(rho: np.ndarray, u: np.ndarray) -> np.ndarray:
    """rho (...), u (..., 3) -> feq (19, ...)  (App. D, D.4)."""
    cu = np.einsum("qa,...a->q...", C.astype(np.float64), u)
    uu = np.einsum("...a,...a->...", u, u)
    return W.reshape((19,) + (1,) * rho.ndim) * rho * (
        1.0 + cu / CS2 + cu ** 2 / (2 * CS2 ** 2) - uu / (2 * CS2))


def _pad(P: np.ndarray, wall: np.ndarray, axis_pop: int, a: int, lo: str, hi: str):
    """Pad populations P (19, ...) and the wall marker along lattice axis a (0=x, 1=y, 2=z)."""
    ax_w = 2 - a                       # array axis of lattice axis a in (z, y, x) arrays
    ax_p = ax_w + axis_pop
    Pn = np.concatenate([np.take(P, [0], axis=ax_p), P, np.take(P, [-1], axis=ax_p)], axis=ax_p)
    Wn = np.concatenate([np.take(wall, [0], axis=ax_w), wall, np.take(wall, [-1], axis=ax_w)],
                        axis=ax_w)
    n = P.shape[ax_p]
    for side, kindf in ((0, lo), (1, hi)):
        g = 0 if side == 0 else n + 1                       # ghost index
        src = (n - 1 if side == 0 else 0) if kindf == "periodic" else (0 if side == 0 else n - 1)
        sl_p = [slice(None)] * Pn.ndim
        sl_p[ax_p] = g
        sl_w = [slice(None)] * Wn.ndim
        sl_w[ax_w] = g
        ghost = np.take(P, src, axis=ax_p)
        gw = np.take(wall, src, axis=ax_w)
        if kindf == "freeslip":
            ghost = ghost[MIRROR[a]]
        if kindf == "noslip":
            gw = np.ones_like(gw)
        Pn[tuple(sl_p)] = ghost
        Wn[tuple(sl_w)] = gw
    return Pn, Wn


def step(F: np.ndarray, kind: np.ndarray, faces, ub: np.ndarray, tau: float, Cs: float,
         force=None, rho_b: float = 1.0, omega=None) -> np.ndarray:
    """One step.  F (19, nz, ny, nx) in THIS module's direction order."""
    nz, ny, nx = kind.shape
    wall = kind == SOLID
    P, Wm = F, wall
    for a in range(3):
        P, Wm = _pad(P, Wm, 1, a, faces[2 * a], faces[2 * a + 1])
    # pull: f_i(x) = P_i(x - c_i), or bounce-back when the upstream ghost/cell is a wall
    f = np.empty_like(F)
    for i in range(19):
        cx, cy, cz = C[i]
        sl = (slice(1 - cz, 1 - cz + nz), slice(1 - cy, 1 - cy + ny), slice(1 - cx, 1 - cx + nx))
        f[i] = np.where(Wm[sl], F[OPP[i]], P[i][sl])
    # collision over the whole lattice (solid cells produce junk here and are overwritten below)
    Fv = np.zeros(3) if force is None else np.asarray(force, np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        out = _collide(f, Fv, tau, Cs, omega)
    # boundary cells
    Z = np.broadcast_to(np.arange(nz)[:, None, None], kind.shape)
    feq_b = equilibrium(np.full(kind.shape, rho_b), np.asarray(ub)[Z])
    out = np.where(kind == EQ, feq_b, out)
    out = np.where(kind == SOLID, 0.0, out)
    return out


def _collide(f: np.ndarray, Fv: np.ndarray, tau: float, Cs: float, omega=None) -> np.ndarray:
    rho = f.sum(axis=0)
    mom = np.einsum("qa,q...->...a", C.astype(np.float64), f)
    # body force per cell: uniform part + Coriolis rho 2 Omega x (mom / rho)  (App. E)
    Fc = np.broadcast_to(Fv, mom.shape).copy()
    if omega is not None:
        Fc = Fc + 2.0 * np.cross(np.asarray(omega, np.float64), mom)
    u = (mom + 0.5 * Fc) / rho[..., None]
    feq = equilibrium(rho, u)
    Pi = np.einsum("qa,qb,q...->...ab", C.astype(np.float64), C.astype(np.float64), f - feq)
    Q = np.sqrt(2.0 * np.einsum("...ab,...ab->...", Pi, Pi))
    te = 0.5 * (tau + np.sqrt(tau ** 2 + 2.0 * Cs ** 2 * Q / (rho * CS2 ** 2)))
    cF = np.einsum("qa,...a->q...", C.astype(np.float64), Fc)
    uF = np.einsum("...a,...a->...", u, Fc)
    cu = np.einsum("qa,...a->q...", C.astype(np.float64), u)
    S = (1.0 - 0.5 / te) * W.reshape(19, 1, 1, 1) * ((cF - uF) / CS2 + cu * cF / CS2 ** 2)
    return f - (f - feq) / te + S


def init(kind: np.ndarray, ub: np.ndarray, rho=None, u=None, rho_b: float = 1.0) -> np.ndarray:
    nz, ny, nx = kind.shape
    Z = np.broadcast_to(np.arange(nz)[:, None, None], kind.shape)
    uu = np.asarray(ub)[Z] if u is None else np.asarray(u, np.float64)
    rr = np.ones(kind.shape) if rho is None else np.asarray(rho, np.float64)
    F = equilibrium(rr, uu)
    F = np.where(kind == EQ, equilibrium(np.full(kind.shape, rho_b), np.asarray(ub)[Z]), F)
    return np.where(kind == SOLID, 0.0, F)


def macros(F: np.ndarray, kind: np.ndarray, ub: np.ndarray, rho_b: float = 1.0, force=None):
    Fv = np.zeros(3) if force is None else np.asarray(force, np.float64)
    rho = F.sum(axis=0)
    u = (np.einsum("qa,q...->...a", C.astype(np.float64), F) - 0.5 * Fv) / np.where(
        rho == 0, 1.0, rho)[..., None]
    nz = kind.shape[0]
    Z = np.broadcast_to(np.arange(nz)[:, None, None], kind.shape)
    u = np.where((kind == EQ)[..., None], np.asarray(ub)[Z], u)
    rho = np.where(kind == EQ, rho_b, rho)
    u = np.where((kind == SOLID)[..., None], 0.0, u)
    rho = np.where(kind == SOLID, 0.0, rho)
    return rho, u


def reorder_from(F_other: np.ndarray, c_other: np.ndarray) -> np.ndarray:
    """Permute a population array given in another direction order (``c_other`` (19,3))."""
    idx = [int(np.nonzero((np.asarray(c_other) == C[i]).all(axis=1))[0][0]) for i in range(19)]
    return F_other[idx]

"""FP64 oracle of the boundary relaxation zones and the flux balancing (TEST INFRASTRUCTURE ONLY).

Only ``tests/`` may import this module; the product library never imports it.

Sec. 3 (boundary-condition paragraph): the open boundaries are supplemented by relaxation-based
damping regions, a top sponge layer and buffer nudging toward the target boundary state next to
the lateral faces, and a flux-balancing correction over the open boundaries.  Sec. 2.1: the mass
flux consistency correction removes the mean normal flux of the boundary field with the smallest
normal velocity adjustment.  The paper gives no profile, widths or rates; the readings taken:

  nudging (applied to the post-collision populations of every fluid cell, after its collision):
      F* <- F* - s (F* - f^eq(rho, u_b(z))),   rho = sum F* (mass is kept),
      s = max over the zones whose face layer is d < w cells away of sigma ((w - d) / w)^2;
      zones: the top face layer (z = nz - 1) with (w_top, sigma_top), and each open lateral face
      (inflow or outflow among x-, x+, y-, y+) with (w_buf, sigma_buf).
  flux balancing: every equilibrium cell belongs to the first inflow face holding it in the order
      x-, x+, y-, y+, z-, z+; Phi = sum over those cells of u_b(z) . n_in; every such cell's
      velocity becomes u_b(z) + delta n_in with delta = -Phi / (number of cells), the smallest
      (least-squares) uniform normal correction that makes the net inflow zero.
"""
from __future__ import annotations

import numpy as np

from . import oracle as orc

_AXIS_NORMALS = [np.array(v, np.float64) for v in
                 ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1))]


def zone_rate(shape, faces, sponge=None, buffer=None) -> np.ndarray:
    """Per-cell relaxation rate s (nz, ny, nx) of the zones; sponge / buffer = (width, sigma)."""
    nz, ny, nx = shape
    Z, Y, X = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    s = np.zeros(shape)

    def ramp(d, w, sig):
        r = np.where(d < w, (w - d) / float(w), 0.0)
        return sig * r * r

    if sponge is not None and sponge[0] > 0:
        s = np.maximum(s, ramp(nz - 1 - Z, sponge[0], sponge[1]))
    if buffer is not None and buffer[0] > 0:
        dist = (X, nx - 1 - X, Y, ny - 1 - Y)
        for k in range(4):
            if faces[k] in ("inflow", "outflow"):
                s = np.maximum(s, ramp(dist[k], buffer[0], buffer[1]))
    return s


def nudge(F: np.ndarray, kind: np.ndarray, faces, ub: np.ndarray, sponge=None, buffer=None) -> np.ndarray:
    """Relax the post-collision populations F (19, nz, ny, nx, oracle order) of fluid cells."""
    s = zone_rate(kind.shape, faces, sponge, buffer)
    s = np.where(kind == orc.FLUID, s, 0.0)
    out = F.copy()
    nz = kind.shape[0]
    for z in range(nz):
        for y in range(kind.shape[1]):
            for x in range(kind.shape[2]):
                if s[z, y, x] == 0.0:
                    continue
                rho = F[:, z, y, x].sum()
                feq = orc.equilibrium(rho, ub[z])
                out[:, z, y, x] = F[:, z, y, x] - s[z, y, x] * (F[:, z, y, x] - feq)
    return out


def run(F, nsteps, kind, faces, ub, tau, C, sponge=None, buffer=None, ueq=None, rho_b=1.0):
    """nsteps oracle steps, each followed by the nudging of the fluid cells."""
    for _ in range(nsteps):
        F = orc.step(F, kind, faces, ub, tau, C, rho_b=rho_b, ueq=ueq)
        F = nudge(F, kind, faces, ub, sponge, buffer)
    return F


def flux_owner(kind: np.ndarray, faces) -> np.ndarray:
    """Owner face index (0..5) of every equilibrium cell, -1 elsewhere."""
    nz, ny, nx = kind.shape
    own = np.full(kind.shape, -1, np.int64)
    n = (nx, ny, nz)
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                if kind[z, y, x] != orc.EQ:
                    continue
                p = (x, y, z)
                for k in range(6):
                    a = k // 2
                    if faces[k] == "inflow" and p[a] == ((n[a] - 1) if (k & 1) else 0):
                        own[z, y, x] = k
                        break
    return own


def flux_balanced_ueq(kind: np.ndarray, faces, ub: np.ndarray):
    """(ueq (nz, ny, nx, 3), Phi before, Phi after, delta): per-cell velocities of the equilibrium
    cells after the flux balancing; zeros at other cells."""
    own = flux_owner(kind, faces)
    nz = kind.shape[0]
    ueq = np.zeros(kind.shape + (3,))
    cells = np.argwhere(own >= 0)
    phi = 0.0
    for z, y, x in cells:
        phi += float(ub[z] @ _AXIS_NORMALS[own[z, y, x]])
    delta = -phi / len(cells) if len(cells) else 0.0
    after = 0.0
    for z, y, x in cells:
        nrm = _AXIS_NORMALS[own[z, y, x]]
        ueq[z, y, x] = ub[z] + delta * nrm
        after += float(ueq[z, y, x] @ nrm)
    return ueq, phi, after, delta

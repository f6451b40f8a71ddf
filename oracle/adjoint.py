"""FP64 discrete adjoint of the time step (TEST INFRASTRUCTURE ONLY).

Only ``tests/`` may import this module; the product library never imports it and has no path that
falls back to it.

Problem (boundary assimilation, the inverse of Sec. 3's boundary-condition paragraph and App. A:
the paper fits the inflow to lidar profiles by Kriging; here the same inflow is fitted by
gradients).  The inflow parameters p = (s_0 .. s_{L-1}, theta) set the equilibrium boundary
velocity u_b(z) = s(z) (cos theta, sin theta, 0) through the level-to-height mapping of
``oracle.expand_profile``.  The initial state is F*_0 = f^eq(1, u_b(z)) in fluid cells (D.4) and
f^eq(rho_b, u_b(z)) in equilibrium cells; F*_n = Phi(F*_{n-1}) is the oracle's time step.  A
virtual lidar samples the horizontal velocity u = sum c F* / rho (D.1) at fluid cells; the loss is
    J(p) = sum_samples sum_{a = x, y} (ubar_a - target_a)^2,
    ubar = mean of u over the states n = T - n_avg + 1 .. T.

Adjoint (reverse sweep over every stored state, no checkpointing; tiny lattices only):
    lambda_T = dJ/dF*_T (explicit),
    lambda_{n-1} = G^T [ J_C(f_n)^T lambda_n ]_fluid + dJ/dF*_{n-1} (explicit),
    dJ/du_b(z) += sum over equilibrium cells at height z of (d f^eq / d u)^T lambda_n  (every n),
    dJ/du_b(z) += sum over all non-solid cells at height z of (d f^eq / d u)^T lambda_0  (F*_0),
where f_n = G F*_{n-1} is the gathered (streamed) pre-collision state and J_C the Jacobian of the
per-cell collision.  The pieces are computed in the most direct way available:
  - G is an explicit index map: for every fluid cell and direction, the flat index of the state
    element it reads, resolved cell by cell from the streaming and boundary rules (App. D
    streaming and mid-grid bounce-back; Sec. 3 faces; same readings as the C oracle).  G^T is the
    scatter-add of that map.  ``gather_map`` is pinned by reproducing the C oracle's step.
  - J_C and d f^eq / d u by complex-step differentiation, d g(x)/dx_j = Im g(x + i h e_j) / h,
    of a restatement of the collision (D.1, D.4, D.8, D.10, D.11, D.2) that accepts complex
    input; exact to rounding, no hand-derived derivative.  At Pi = 0 the LES term is taken as
    having zero derivative (Q = |Pi| is not differentiable there; its factor sum lambda (f^eq - f)
    vanishes there anyway).
  - the chain rule to p uses the linearity of the profile mapping in the speeds (columns of
    ``expand_profile`` at unit speeds) and d u_b / d theta = u_b at theta + pi/2.
Sampled cells must be fluid cells (a sample in an equilibrium cell would depend on p directly).
"""
from __future__ import annotations

import math

import numpy as np

from . import oracle as orc

CS2 = 1.0 / 3.0
_H = 1e-60   # complex-step size


def _lat():
    c, w, opp = orc.lattice()
    return c.astype(np.int64), w, opp.astype(np.int64)


def gather_map(kind: np.ndarray, faces) -> np.ndarray:
    """Flat source index (into F of shape (19, N)) of every population a fluid cell gathers.

    Returns src (19, N) int64, -1 for cells that do not gather (solid, equilibrium).  Rule for the
    population i of fluid cell p, source position s = p - c_i (App. D streaming and bounce-back;
    Sec. 3 faces; one axis at a time at edges and corners):
      - a no-slip face beyond any out-of-range axis of s  -> bounce-back: F*_opp(i)(p);
      - otherwise each out-of-range axis: periodic wraps; outflow clamps to the face layer (zero
        gradient); free-slip clamps and negates that velocity component of the direction;
      - a solid resolved source -> bounce-back;  else F*_d(s) with the (possibly mirrored) d."""
    c, _, opp = _lat()
    nz, ny, nx = kind.shape
    n = (nx, ny, nz)
    N = nx * ny * nz
    dir_of = {tuple(v): i for i, v in enumerate(c)}
    src = np.full((19, N), -1, np.int64)
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                cell = (z * ny + y) * nx + x
                if kind[z, y, x] != orc.FLUID:
                    continue
                p = (x, y, z)
                for i in range(19):
                    s = [p[a] - c[i][a] for a in range(3)]
                    bb = False
                    for a in range(3):
                        if s[a] < 0 and faces[2 * a] == "noslip":
                            bb = True
                        if s[a] >= n[a] and faces[2 * a + 1] == "noslip":
                            bb = True
                    vel = list(c[i])
                    if not bb:
                        for a in range(3):
                            if 0 <= s[a] < n[a]:
                                continue
                            hi = s[a] >= n[a]
                            fk = faces[2 * a + int(hi)]
                            if fk == "periodic":
                                s[a] = s[a] - n[a] if hi else s[a] + n[a]
                            else:
                                s[a] = n[a] - 1 if hi else 0
                                if fk == "freeslip":
                                    vel[a] = -vel[a]
                        if kind[s[2], s[1], s[0]] == orc.SOLID:
                            bb = True
                    if bb:
                        src[i, cell] = opp[i] * N + cell
                    else:
                        d = dir_of[tuple(vel)]
                        src[i, cell] = d * N + (s[2] * ny + s[1]) * nx + s[0]
    return src


def equilibrium_c(rho, u):
    """D.4 for arrays (complex allowed): rho (M,), u (3, M) -> (19, M)."""
    c, w, _ = _lat()
    cu = c.astype(np.float64) @ u                      # (19, M)
    uu = (u * u).sum(axis=0)
    return w[:, None] * rho[None, :] * (1.0 + cu / CS2 + cu ** 2 / (2 * CS2 ** 2)
                                        - uu[None, :] / (2 * CS2))


def collide_c(f, tau: float, Cs: float):
    """Collision of every column of f (19, M), complex allowed: moments (D.1), equilibrium (D.4),
    Pi^(1) (D.8), Q (D.10), tau_eff (D.11), BGK (D.2).  No body force."""
    c, _, _ = _lat()
    cf = c.astype(np.float64)
    rho = f.sum(axis=0)
    u = (cf.T @ f) / rho[None, :]
    feq = equilibrium_c(rho, u)
    neq = f - feq
    Pi = np.einsum("ia,ib,im->abm", cf, cf, neq)
    PP = (Pi * Pi).sum(axis=(0, 1))
    pos = PP.real > 0.0
    Q = np.where(pos, np.sqrt(2.0 * np.where(pos, PP, 1.0)), 0.0 * PP)
    te = 0.5 * (tau + np.sqrt(tau * tau + 2.0 * Cs * Cs * Q / (rho * CS2 * CS2)))
    return f - neq / te[None, :]


def collision_jacobian(f: np.ndarray, tau: float, Cs: float) -> np.ndarray:
    """d f*_k / d f_j for every column of f (19, M) by complex step: (19 k, 19 j, M)."""
    M = f.shape[1]
    Jac = np.empty((19, 19, M))
    for j in range(19):
        fc = f.astype(np.complex128)
        fc[j] += 1j * _H
        Jac[:, j, :] = collide_c(fc, tau, Cs).imag / _H
    return Jac


def equilibrium_du(rho: np.ndarray, u: np.ndarray) -> np.ndarray:
    """d f^eq_k / d u_a by complex step: rho (M,), u (3, M) -> (19, 3, M)."""
    M = u.shape[1]
    out = np.empty((19, 3, M))
    for a in range(3):
        uc = u.astype(np.complex128)
        uc[a] += 1j * _H
        out[:, a, :] = equilibrium_c(rho.astype(np.complex128), uc).imag / _H
    return out


class Problem:
    """One assimilation problem on a small lattice (see the module docstring)."""

    def __init__(self, solid, faces, tau, Cs, nsteps, n_avg, cols, heights, target, L,
                 rho_b: float = 1.0):
        self.solid = np.ascontiguousarray(solid, np.uint8)
        self.faces = tuple(faces)
        self.tau, self.Cs = float(tau), float(Cs)
        self.T, self.n_avg = int(nsteps), int(n_avg)
        self.cols = np.asarray(cols, np.int64).reshape(-1, 2)      # (ncol, 2) = (x, y)
        self.heights = np.asarray(heights, np.int64).reshape(-1)   # (nh,)
        self.target = np.asarray(target, np.float64).reshape(len(self.cols), len(self.heights), 2)
        self.L = int(L)
        self.rho_b = float(rho_b)
        self.kind = orc.classify(self.solid, self.faces)
        nz, ny, nx = self.solid.shape
        self.shape = (nz, ny, nx)
        self.N = nx * ny * nz
        cells = [(int(k) * ny + int(y)) * nx + int(x) for (x, y) in self.cols for k in self.heights]
        self.sample_cells = np.array(cells, np.int64)
        if (self.kind.reshape(-1)[self.sample_cells] != orc.FLUID).any():
            raise ValueError("sampled cells must be fluid cells")
        if not 1 <= self.n_avg <= self.T + 1:
            raise ValueError("n_avg must be in [1, T + 1]")

    # ------------------------------------------------------------------ forward
    def profile(self, speed, theta):
        return orc.expand_profile(np.asarray(speed, np.float64), self.shape[0], float(theta))

    def initial_state(self, ub):
        return orc.init(self.kind, ub, rho_b=self.rho_b)

    def forward(self, speed, theta, keep: bool = False):
        """Mean sampled velocity (ncol, nh, 3) and, with ``keep``, every state F*_0 .. F*_T."""
        ub = self.profile(speed, theta)
        F = self.initial_state(ub)
        states = [F] if keep else None
        acc = np.zeros((len(self.sample_cells), 3))
        first = self.T - self.n_avg + 1
        if first <= 0:
            acc += self._sample(F)
        for n in range(1, self.T + 1):
            F = orc.step(F, self.kind, self.faces, ub, self.tau, self.Cs, rho_b=self.rho_b)
            if keep:
                states.append(F)
            if n >= first:
                acc += self._sample(F)
        mean = (acc / self.n_avg).reshape(len(self.cols), len(self.heights), 3)
        return (mean, states) if keep else mean

    def _sample(self, F):
        c, _, _ = _lat()
        f = F.reshape(19, -1)[:, self.sample_cells]
        rho = f.sum(axis=0)
        return (c.astype(np.float64).T @ f).T / rho[:, None]

    def loss(self, speed, theta) -> float:
        mean = self.forward(speed, theta)
        r = mean[..., :2] - self.target
        return float((r * r).sum())

    # ------------------------------------------------------------------ adjoint
    def _explicit(self, F, resid):
        """dJ/dF* at the sampled cells of one averaged state: 2 r . d u / d F* / n_avg, with
        d u_a / d F*_i = (c_ia - u_a) / rho."""
        c, _, _ = _lat()
        f = F.reshape(19, -1)[:, self.sample_cells]
        rho = f.sum(axis=0)
        u = (c.astype(np.float64).T @ f) / rho[None, :]            # (3, S)
        g = np.zeros((19, len(self.sample_cells)))
        for a in range(2):
            g += (2.0 * resid[:, a] / self.n_avg)[None, :] * (c[:, a][:, None] - u[a][None, :]) / rho[None, :]
        return g

    def gradient(self, speed, theta):
        """(J, dJ/dspeed (L,), dJ/dtheta) by the discrete adjoint."""
        speed = np.asarray(speed, np.float64)
        mean, states = self.forward(speed, theta, keep=True)
        resid = (mean[..., :2] - self.target).reshape(-1, 2)
        J = float((resid * resid).sum())
        nz, ny, nx = self.shape
        N = self.N
        src = gather_map(self.kind, self.faces)
        kflat = self.kind.reshape(-1)
        fluid = np.nonzero(kflat == orc.FLUID)[0]
        eq = np.nonzero(kflat == orc.EQ)[0]
        zcell = np.arange(N) // (nx * ny)
        ub = self.profile(speed, theta)
        first = self.T - self.n_avg + 1
        g_ub = np.zeros((nz, 3))

        def add_explicit(lam, n):
            if n >= first:
                lam[:, self.sample_cells] += self._explicit(states[n], resid)

        def add_ub(lam, cells, rho_val):
            if len(cells) == 0:
                return
            dfe = equilibrium_du(np.full(len(cells), rho_val), ub[zcell[cells]].T)  # (19, 3, M)
            contrib = np.einsum("km,kam->ma", lam[:, cells], dfe)
            np.add.at(g_ub, zcell[cells], contrib)

        lam = np.zeros((19, N))
        add_explicit(lam, self.T)
        for n in range(self.T, 0, -1):
            add_ub(lam, eq, self.rho_b)                  # F*_n of equilibrium cells = f^eq(u_b)
            Fprev = states[n - 1].reshape(-1)
            f = Fprev[src[:, fluid]]                     # gathered pre-collision state (19, M)
            Jac = collision_jacobian(f, self.tau, self.Cs)
            mu = np.einsum("kjm,km->jm", Jac, lam[:, fluid])
            nxt = np.zeros(19 * N)
            np.add.at(nxt, src[:, fluid].reshape(-1), mu.reshape(-1))
            lam = nxt.reshape(19, N)
            add_explicit(lam, n - 1)
        # the initial state depends on u_b in every non-solid cell
        add_ub(lam, fluid, 1.0)
        add_ub(lam, eq, self.rho_b)
        # chain rule to the level speeds and the direction
        dspeed = np.zeros(self.L)
        for l in range(self.L):
            e = np.zeros(self.L)
            e[l] = 1.0
            dspeed[l] = float((self.profile(e, theta) * g_ub).sum())
        dtheta = float((self.profile(speed, theta + 0.5 * math.pi) * g_ub).sum())
        return J, dspeed, dtheta, g_ub

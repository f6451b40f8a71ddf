"""Seeded synthetic inputs: geometry, inflow level speeds, initial velocity fields.

This module produces INPUTS only -- solid masks, face kinds, per-level inflow speeds and explicit
initial velocity fields -- and holds none of the solver's arithmetic.  The CUDA path and the FP64
oracle are both fed from it; neither is imported here.

The paper's own inputs (3D-GloBFP building footprints, NASADEM terrain, Doppler-lidar boundary
winds; Sec. 3) are not available, so every workload is synthetic, shaped like the paper's: a 5 m
lattice over a kilometre-scale urban patch with N_cell of order 1e7-1e8 (Sec. 3, baseline case),
buildings as voxel solids on a no-slip ground, an observation-like sheared inflow profile.

Conventions: arrays are (nz, ny, nx) with x fastest in memory; a height level k is the cell
whose centre sits k + 1/2 above the ground wall (the wall lies half a spacing below the first
cell, App. D, bounce-back paragraph).  Face kinds in the order x-, x+, y-, y+, z-, z+:
'periodic' | 'inflow' | 'outflow' | 'freeslip' | 'noslip'.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Case:
    """One synthetic workload: geometry, faces, model constants, inflow levels, initial field."""
    name: str
    solid: np.ndarray                 # (nz, ny, nx) uint8, 1 = solid
    faces: tuple                      # 6 face kinds
    tau: float
    cs: float                         # Smagorinsky constant C
    speed: np.ndarray                 # inflow speed per level (L levels)
    theta: float                      # inflow direction [rad], 0 = +x, counter-clockwise
    u0: np.ndarray | None = None      # (nz, ny, nx, 3) initial velocity (None: profile)
    rho0: np.ndarray | None = None    # (nz, ny, nx) initial density (None: 1)
    force: tuple | None = None        # uniform body-force density (Guo forcing), lattice units
    coriolis: tuple | None = None     # rotation vector Omega^lbm of the Coriolis force, lattice units
    rho_b: float = 1.0
    meta: dict = field(default_factory=dict)

    @property
    def shape(self):
        return self.solid.shape

    @property
    def dims(self):
        nz, ny, nx = self.solid.shape
        return nx, ny, nz


# ----------------------------------------------------------------------------- inflow levels
def log_law_levels(nz: int, u_ref: float, z_ref: float, z0: float) -> np.ndarray:
    """Neutral log-law speed at each cell height k + 1/2: u_ref ln(z/z0) / ln(z_ref/z0)."""
    z = np.arange(nz) + 0.5
    return u_ref * np.log(z / z0) / math.log(z_ref / z0)


def power_law_levels(nz: int, u_ref: float, z_ref: float, alpha: float) -> np.ndarray:
    """Power-law speed at each cell height k + 1/2: u_ref (z / z_ref)^alpha."""
    z = np.arange(nz) + 0.5
    return u_ref * (z / z_ref) ** alpha


def direction_from_seed(seed: int) -> float:
    """Inflow direction uniform in [0, 360) degrees, returned in radians."""
    return math.radians(float(np.random.default_rng(seed).uniform(0.0, 360.0)))


def faces_for_direction(theta: float, bottom: str = "noslip", top: str = "freeslip") -> tuple:
    """A lateral face is an inflow face when the wind blows into the domain through it
    (u . n_in > 0), an outflow face otherwise; a wind within 1e-6 of parallel to a face counts as
    parallel (outflow on both sides)."""
    cx, cy = math.cos(theta), math.sin(theta)
    eps = 1e-6
    return ("inflow" if cx > eps else "outflow", "inflow" if cx < -eps else "outflow",
            "inflow" if cy > eps else "outflow", "inflow" if cy < -eps else "outflow",
            bottom, top)


# ----------------------------------------------------------------------------- initial fields
def profile_field(speed_per_cell: np.ndarray, theta: float, shape) -> np.ndarray:
    """Velocity field equal to the level speed of each cell height, along theta (L == nz)."""
    nz, ny, nx = shape
    assert len(speed_per_cell) == nz
    u = np.zeros((nz, ny, nx, 3), np.float64)
    u[..., 0] = (speed_per_cell * math.cos(theta))[:, None, None]
    u[..., 1] = (speed_per_cell * math.sin(theta))[:, None, None]
    return u


def perturb(u: np.ndarray, solid: np.ndarray, amp: float, seed: int) -> np.ndarray:
    """u + amp * xi, xi ~ U[-1, 1]^3 per cell and component (PCG64 stream ``seed``); solids 0."""
    xi = np.random.default_rng(seed).uniform(-1.0, 1.0, size=u.shape)
    out = u + amp * xi
    out[solid.astype(bool)] = 0.0
    return out


# ----------------------------------------------------------------------------- geometry
def cube_case(nx: int = 64, ny: int = 64, nz: int = 32, seed: int = 0, tau: float = 0.52,
              cs: float = 0.16, noise: float = 0.01) -> Case:
    """Single cubical building 8 x 8 x 16 cells centred in a 64 x 64 x 32 lattice; log-law
    inflow along +x (u_ref 0.05 at z = 32, z0 = 0.1); zero-gradient outflow; periodic in y;
    no-slip ground; free-slip top; initial velocity = profile + 1% u_ref uniform noise."""
    solid = np.zeros((nz, ny, nx), np.uint8)
    cx0, cy0 = nx // 2 - 4, ny // 2 - 4
    solid[0:min(16, nz - 1), cy0:cy0 + 8, cx0:cx0 + 8] = 1
    speed = log_law_levels(nz, 0.05, 32.0, 0.1)
    faces = ("inflow", "outflow", "periodic", "periodic", "noslip", "freeslip")
    u0 = perturb(profile_field(speed, 0.0, solid.shape), solid, noise * 0.05, seed)
    return Case("cube", solid, faces, tau, cs, speed, 0.0, u0=u0,
                meta={"seed": seed, "noise": noise})


def city_mask(nx: int, ny: int, nz: int, seed: int, plan_fraction: float = 0.35,
              side_min: int = 2, side_max: int = 12, margin: int = 8, gap: int = 1,
              h_median: float = 6.0, h_sigma: float = 0.6, h_max: int = 50,
              max_attempts: int = 1_000_000) -> tuple[np.ndarray, dict]:
    """Box city by seeded dart throwing: footprints with sides U{side_min..side_max} (x and y
    independent), rejected within ``gap`` cells of another footprint or within ``margin`` cells
    of a lateral face, until the plan-area fraction reaches ``plan_fraction``; heights
    round(exp(ln h_median + h_sigma N(0,1))) clamped to [1, min(h_max, nz - 2)]."""
    rng = np.random.default_rng(seed)
    occ = np.zeros((ny, nx), bool)
    height = np.zeros((ny, nx), np.int32)
    target = plan_fraction * nx * ny
    area = 0
    attempts = 0
    placed = 0
    hcap = max(1, min(h_max, nz - 2))
    batch = 4096
    while area < target and attempts < max_attempts:
        sx = rng.integers(side_min, side_max + 1, size=batch)
        sy = rng.integers(side_min, side_max + 1, size=batch)
        ux = rng.random(batch)
        uy = rng.random(batch)
        hs = rng.standard_normal(batch)
        for b in range(batch):
            attempts += 1
            w, d = int(sx[b]), int(sy[b])
            span_x = nx - 2 * margin - w
            span_y = ny - 2 * margin - d
            if span_x < 0 or span_y < 0:
                continue
            x0 = margin + int(ux[b] * (span_x + 1))
            y0 = margin + int(uy[b] * (span_y + 1))
            if occ[max(0, y0 - gap):y0 + d + gap, max(0, x0 - gap):x0 + w + gap].any():
                continue
            h = int(round(math.exp(math.log(h_median) + h_sigma * hs[b])))
            h = min(max(h, 1), hcap)
            occ[y0:y0 + d, x0:x0 + w] = True
            height[y0:y0 + d, x0:x0 + w] = h
            area += w * d
            placed += 1
            if area >= target or attempts >= max_attempts:
                break
    z = np.arange(nz)[:, None, None]
    solid = (z < height[None, :, :]).astype(np.uint8)
    info = {"buildings": placed, "attempts": attempts, "plan_fraction": area / (nx * ny),
            "solid_fraction": float(solid.mean())}
    return solid, info


def city_case(nx: int = 400, ny: int = 400, nz: int = 80, seed: int = 1, dir_seed: int | None = None,
              tau: float = 0.505, cs: float = 0.16, u_ref: float = 0.06, z_ref: float = 60.0,
              alpha: float = 0.25, noise: float = 0.01) -> Case:
    """Synthetic city on a 5 m lattice (400 x 400 x 80 = 2 km x 2 km x 400 m by default):
    power-law inflow from a seeded direction; lateral faces inflow/outflow by the wind
    direction; free-slip top; no-slip ground."""
    solid, info = city_mask(nx, ny, nz, seed)
    theta = direction_from_seed(seed if dir_seed is None else dir_seed)
    speed = power_law_levels(nz, u_ref, z_ref, alpha)
    faces = faces_for_direction(theta)
    u0 = (perturb(profile_field(speed, theta, solid.shape), solid, noise * u_ref, seed + 1000)
          if noise > 0 else None)
    return Case(f"city{nx}x{ny}x{nz}", solid, faces, tau, cs, speed, theta, u0=u0,
                meta={"seed": seed, **info})


def taylor_green_case(n: int = 32, U0: float = 0.01, tau: float = 0.8, cs: float = 0.0,
                      nz: int | None = None) -> Case:
    """2D Taylor-Green vortex extruded along z in a fully periodic box:
    u = -U0 cos(kx) sin(ky), v = U0 sin(kx) cos(ky), k = 2 pi / n, at cell centres."""
    nz = n if nz is None else nz
    k = 2.0 * math.pi / n
    x = np.arange(n) + 0.0
    X, Y = np.meshgrid(x, x, indexing="xy")          # (ny, nx)
    u = np.zeros((nz, n, n, 3))
    u[..., 0] = (-U0 * np.cos(k * X) * np.sin(k * Y))[None]
    u[..., 1] = (U0 * np.sin(k * X) * np.cos(k * Y))[None]
    solid = np.zeros((nz, n, n), np.uint8)
    faces = ("periodic",) * 6
    return Case(f"tg{n}", solid, faces, tau, cs, np.zeros(nz), 0.0, u0=u,
                meta={"U0": U0, "k": k})


def channel_case(nz: int = 16, nxy: int = 4, force: float = 1e-6, tau: float = 0.5 + math.sqrt(3 / 16),
                 cs: float = 0.0) -> Case:
    """Plane channel between no-slip walls at z = -1/2 and z = nz - 1/2, periodic in x and y,
    driven by a uniform body force along +x; starts from rest."""
    solid = np.zeros((nz, nxy, nxy), np.uint8)
    faces = ("periodic", "periodic", "periodic", "periodic", "noslip", "noslip")
    u0 = np.zeros((nz, nxy, nxy, 3))
    return Case(f"channel{nz}", solid, faces, tau, cs, np.zeros(nz), 0.0, u0=u0,
                force=(force, 0.0, 0.0))


def random_small_case(nx: int, ny: int, nz: int, faces, seed: int, solid_fraction: float = 0.1,
                      u_amp: float = 0.05, tau: float = 0.6, cs: float = 0.16,
                      theta: float = 0.3, margin: int = 1) -> Case:
    """Tiny lattice with scattered solid cells (kept ``margin`` cells off the lateral faces),
    random initial velocity and density -- for brute-force cross-checks of the boundary logic."""
    rng = np.random.default_rng(seed)
    solid = (rng.random((nz, ny, nx)) < solid_fraction).astype(np.uint8)
    if margin > 0:
        solid[:, :, :margin] = 0
        solid[:, :, nx - margin:] = 0
        solid[:, :margin, :] = 0
        solid[:, ny - margin:, :] = 0
    u0 = rng.uniform(-u_amp, u_amp, size=(nz, ny, nx, 3))
    u0[solid.astype(bool)] = 0.0
    rho0 = 1.0 + rng.uniform(-0.01, 0.01, size=(nz, ny, nx))
    speed = u_amp * (0.5 + 0.5 * rng.random(nz))
    return Case(f"rand{nx}x{ny}x{nz}", solid, tuple(faces), tau, cs, speed, theta, u0=u0,
                rho0=rho0)


def stg_uniforms(n_modes: int, seed: int, shared: bool = False) -> np.ndarray:
    """Random draws of the synthetic inflow turbulence (App. F): (6, n_modes, 6) uniforms on [0, 1)
    per face (x-, x+, y-, y+, z-, z+) and mode -- r_m, (mu_m + 1)/2, theta_m / 2pi and the three
    phases / 2pi.  Each face gets its own stream seeded from (seed, face) unless ``shared``, in
    which case every face gets the same realisation.  Only random numbers: no method arithmetic."""
    out = np.empty((6, n_modes, 6), np.float64)
    for f in range(6):
        rng = np.random.default_rng([seed, 0 if shared else f + 1])
        out[f] = rng.random((n_modes, 6))
    return out


# ----------------------------------------------------------------------------- boundary assimilation
def lidar_columns(solid: np.ndarray, n_cols: int, seed: int, clearance: int = 3,
                  top: int | None = None, face_margin: int = 10) -> np.ndarray:
    """(n_cols, 2) integer (x, y) positions of virtual lidar columns, drawn uniformly (PCG64
    stream ``seed``) among the columns whose cells up to height ``top`` (default: all) are at
    least ``clearance`` cells (Chebyshev distance) from every solid cell and at least
    ``face_margin`` cells from the lateral faces (inside the built-up area); distinct columns."""
    nz, ny, nx = solid.shape
    top = nz if top is None else top
    blocked = solid[:top].any(axis=0)
    ok = np.zeros((ny, nx), bool)
    m = max(clearance, face_margin)
    ok[m:ny - m, m:nx - m] = True
    ys, xs = np.nonzero(blocked)
    for y, x in zip(ys, xs):
        ok[max(0, y - clearance):y + clearance + 1, max(0, x - clearance):x + clearance + 1] = False
    cand = np.argwhere(ok)                      # (m, 2) = (y, x)
    if len(cand) < n_cols:
        raise ValueError("not enough clear columns")
    pick = np.random.default_rng(seed).choice(len(cand), size=n_cols, replace=False)
    return np.stack([cand[pick, 1], cand[pick, 0]], axis=1).astype(np.int32)


@dataclass
class Assimilation:
    """Inflow recovery from virtual lidar: a city, hidden 'truth' inflow parameters, a first
    guess, the lidar columns and heights, and the averaging window."""
    case: Case
    L: int                       # level speeds
    speed_true: np.ndarray
    theta_true: float
    speed_guess: np.ndarray
    theta_guess: float
    cols: np.ndarray             # (ncol, 2) int32 (x, y)
    heights: np.ndarray          # (nh,) int32 cell heights
    nsteps: int
    n_avg: int                   # the last n_avg states of the run are averaged
    checkpoint_every: int


def assimilation_case(nx: int = 128, ny: int = 128, nz: int = 48, seed: int = 4, L: int = 24,
                      n_cols: int = 8, heights=tuple(range(4, 41, 4)), nsteps: int = 2000,
                      n_avg: int = 500, checkpoint_every: int = 100, tau: float = 0.505,
                      cs: float = 0.16, u_ref: float = 0.06, z_ref: float = 60.0,
                      alpha: float = 0.25, guess_scale: float = 0.8,
                      guess_dtheta: float = 0.1) -> Assimilation:
    """Synthetic city (same generator as ``city_case``, seed-fixed) whose inflow is parameterised
    by L level speeds (equal blocks of nz / L cells) and one direction.  Truth: the power law at
    the level centres from a seeded direction; first guess: ``guess_scale`` x the truth speeds and
    the direction turned by ``guess_dtheta`` rad (the face kinds follow the truth direction and
    stay fixed).  Lidar columns: ``n_cols`` seeded fluid columns >= 2 cells from solids and
    >= 10 cells from the lateral faces (at a plan-area fraction of 0.35 only a handful of columns
    inside the built-up area keep 3 cells from every building)."""
    solid, info = city_mask(nx, ny, nz, seed)
    theta = direction_from_seed(seed)
    zc = (np.arange(L) + 0.5) * nz / L
    speed = u_ref * (zc / z_ref) ** alpha
    faces = faces_for_direction(theta)
    heights = np.asarray(heights, np.int32)
    cols = lidar_columns(solid, n_cols, seed + 7, clearance=2, top=int(heights.max()) + 1)
    case = Case(f"assim{nx}x{ny}x{nz}", solid, faces, tau, cs, speed, theta,
                meta={"seed": seed, **info})
    return Assimilation(case, L, speed, theta, guess_scale * speed, theta + guess_dtheta, cols,
                        heights, nsteps, n_avg, checkpoint_every)


# ----------------------------------------------------------------------------- ensembles
def ensemble_cases(nx: int = 256, ny: int = 256, nz: int = 64, seed: int = 3, n_dir: int = 16,
                   u_refs=(0.04, 0.07), tau: float = 0.505, cs: float = 0.16, z_ref: float = 60.0,
                   alpha: float = 0.25) -> list:
    """Wind-rose ensemble on one synthetic city: n_dir inflow directions 0, 360/n_dir, ... degrees
    times the reference speeds u_refs (power law, alpha 0.25, z_ref 60); faces follow each
    direction.  Members start from the profile (no noise)."""
    solid, info = city_mask(nx, ny, nz, seed)
    out = []
    for k in range(n_dir):
        theta = math.radians(360.0 * k / n_dir)
        for u in u_refs:
            speed = power_law_levels(nz, u, z_ref, alpha)
            out.append(Case(f"ens{nx}x{ny}x{nz}_d{k}_u{u}", solid, faces_for_direction(theta), tau, cs,
                            speed, theta, meta={"seed": seed, **info}))
    return out


UNEVEN_SIZES = ((96, 96, 32), (128, 96, 32), (160, 128, 48), (192, 160, 48), (224, 128, 64),
                (256, 192, 64), (288, 160, 64), (320, 192, 64))


def uneven_cases(sizes=UNEVEN_SIZES, seed: int = 10, tau: float = 0.505, cs: float = 0.16,
                 u_ref: float = 0.06, z_ref: float = 60.0, alpha: float = 0.25) -> list:
    """Domains of uneven size (96x96x32 .. 320x192x64 by default), each its own seeded city and
    seeded inflow direction, power-law inflow; members start from the profile."""
    out = []
    for k, (nx, ny, nz) in enumerate(sizes):
        solid, info = city_mask(nx, ny, nz, seed + k)
        theta = direction_from_seed(seed + k)
        speed = power_law_levels(nz, u_ref, z_ref, alpha)
        out.append(Case(f"uneven{nx}x{ny}x{nz}", solid, faces_for_direction(theta), tau, cs, speed, theta,
                        meta={"seed": seed + k, **info}))
    return out

"""Pins of the oracle's full time step: streaming indices and every boundary rule (single-population
pulses), conservation, symmetry, rest state, brute-force cross-check against the independently
written NumPy formulation, profile expansion.  CPU only; paper App. D (D.1-D.4, bounce-back),
Sec. 3 (boundary conditions)."""
import math

import numpy as np
import pytest

from oracle import oracle as orc
from oracle import lbm_numpy as onp
from paper_2607_04516_b300 import synth

C, W, OPP = orc.lattice()
IDX = {tuple(v): i for i, v in enumerate(C)}
TAU_INF = 1e15      # BGK with tau -> infinity: pure streaming (f* = f up to 1e-15)


def _rest_state(shape):
    nz, ny, nx = shape
    return np.broadcast_to(W[:, None, None, None], (19, nz, ny, nx)).copy()


def _pulse_step(faces, shape, cell, d, solid=None, amp=1e-3):
    """Put +amp on population d at ``cell`` (x, y, z) over a rest state; one pure-stream step.
    Returns {(x, y, z, direction vector): excess} for every population that changed."""
    nz, ny, nx = shape
    solid = np.zeros(shape, np.uint8) if solid is None else solid
    kind = orc.classify(solid, faces)
    ub = np.zeros((nz, 3))
    F = _rest_state(shape)
    F[:, kind == orc.SOLID] = 0.0
    x, y, z = cell
    F[IDX[d], z, y, x] += amp
    out = orc.step(F, kind, faces, ub, TAU_INF, 0.0)
    ref = _rest_state(shape)
    ref[:, kind == orc.SOLID] = 0.0
    diff = out - ref
    hits = {}
    for i, zz, yy, xx in zip(*np.nonzero(np.abs(diff) > 1e-12)):
        hits[(int(xx), int(yy), int(zz), tuple(int(v) for v in C[i]))] = diff[i, zz, yy, xx]
    return hits


PER = ("periodic",) * 6


def test_pulse_streams_along_its_velocity():
    shape = (5, 6, 7)
    for d in map(tuple, C):
        if d == (0, 0, 0):
            continue
        hits = _pulse_step(PER, shape, (3, 2, 2), d)
        assert hits.keys() == {(3 + d[0], 2 + d[1], 2 + d[2], d)}, d


def test_pulse_wraps_on_periodic_faces():
    shape = (5, 6, 7)
    hits = _pulse_step(PER, shape, (6, 5, 4), (1, 1, 0))
    assert hits.keys() == {(0, 0, 4, (1, 1, 0))}
    hits = _pulse_step(PER, shape, (0, 0, 0), (0, -1, -1))
    assert hits.keys() == {(0, 5, 4, (0, -1, -1))}


def test_pulse_bounces_back_from_solid_cell():
    """Mid-grid bounce-back: a population heading into a solid returns reversed to its cell."""
    shape = (5, 6, 7)
    solid = np.zeros(shape, np.uint8)
    solid[2, 2, 4] = 1
    hits = _pulse_step(PER, shape, (3, 2, 2), (1, 0, 0), solid=solid)
    assert hits.keys() == {(3, 2, 2, (-1, 0, 0))}
    hits = _pulse_step(PER, shape, (3, 3, 2), (1, -1, 0), solid=solid)
    assert hits.keys() == {(3, 3, 2, (-1, 1, 0))}


def test_pulse_bounces_back_from_noslip_ground():
    faces = ("periodic", "periodic", "periodic", "periodic", "noslip", "freeslip")
    hits = _pulse_step(faces, (5, 6, 7), (3, 2, 0), (1, 0, -1))
    assert hits.keys() == {(3, 2, 0, (-1, 0, 1))}


def test_pulse_reflects_specularly_at_freeslip_top():
    faces = ("periodic", "periodic", "periodic", "periodic", "noslip", "freeslip")
    hits = _pulse_step(faces, (5, 6, 7), (3, 2, 4), (1, 0, 1))
    assert hits.keys() == {(4, 2, 4, (1, 0, -1))}
    hits = _pulse_step(faces, (5, 6, 7), (3, 2, 4), (0, 0, 1))
    assert hits.keys() == {(3, 2, 4, (0, 0, -1))}


def test_pulse_at_zero_gradient_outflow():
    """Zero gradient: an inward population of the outflow layer also seeds the population of the
    same direction entering the layer from outside; an outward one leaves the domain."""
    faces = ("inflow", "outflow", "periodic", "periodic", "noslip", "freeslip")
    shape = (5, 6, 7)
    nx = shape[2]
    hits = _pulse_step(faces, shape, (nx - 1, 2, 2), (-1, 1, 0))
    assert hits.keys() == {(nx - 2, 3, 2, (-1, 1, 0)), (nx - 1, 3, 2, (-1, 1, 0))}
    hits = _pulse_step(faces, shape, (nx - 1, 2, 2), (-1, 0, 0))
    assert hits.keys() == {(nx - 2, 2, 2, (-1, 0, 0)), (nx - 1, 2, 2, (-1, 0, 0))}
    hits = _pulse_step(faces, shape, (nx - 1, 2, 2), (1, 0, 1))
    assert hits == {}


def test_pulse_outflow_top_corner():
    faces = ("inflow", "outflow", "periodic", "periodic", "noslip", "freeslip")
    shape = (5, 6, 7)
    nx, nz = shape[2], shape[0]
    hits = _pulse_step(faces, shape, (nx - 1, 2, nz - 1), (-1, 0, 1))
    # normal stream -> (nx-2, 2, top) reflected; zero-gradient copy -> (nx-1, 2, top) reflected
    assert hits.keys() == {(nx - 2, 2, nz - 1, (-1, 0, -1)), (nx - 1, 2, nz - 1, (-1, 0, -1))}


def test_equilibrium_cells_hold_feq():
    faces = ("inflow", "outflow", "periodic", "periodic", "noslip", "freeslip")
    case = synth.random_small_case(8, 6, 5, faces, seed=3)
    kind = orc.classify(case.solid, faces)
    ub = orc.expand_profile(case.speed, 5, 0.4)
    F = orc.init(kind, ub, case.rho0, case.u0)
    out = orc.step(F, kind, faces, ub, 0.6, 0.16)
    for z in range(5):
        feq = orc.equilibrium(1.0, ub[z])
        for y in range(6):
            np.testing.assert_allclose(out[:, z, y, 0], feq, rtol=0, atol=1e-17)


@pytest.mark.parametrize("cs", [0.0, 0.16])
def test_periodic_box_conserves_mass_and_momentum(cs):
    case = synth.random_small_case(9, 7, 6, PER, seed=1, solid_fraction=0.0, u_amp=0.05)
    kind = orc.classify(case.solid, PER)
    ub = np.zeros((6, 3))
    F = orc.init(kind, ub, case.rho0, case.u0)
    m0 = F.sum()
    p0 = (C.T @ F.reshape(19, -1)).sum(1)
    G = orc.run(F, 60, kind, PER, ub, 0.52, cs)
    assert abs(G.sum() - m0) / m0 < 1e-13
    np.testing.assert_allclose((C.T @ G.reshape(19, -1)).sum(1), p0, rtol=0, atol=1e-13 * m0)


def test_periodic_box_with_solids_conserves_mass():
    """Bounce-back exchanges momentum with walls but never creates or destroys mass."""
    case = synth.random_small_case(9, 7, 6, PER, seed=2, solid_fraction=0.15, u_amp=0.05,
                                   margin=0)
    kind = orc.classify(case.solid, PER)
    ub = np.zeros((6, 3))
    F = orc.init(kind, ub, case.rho0, case.u0)
    G = orc.run(F, 60, kind, PER, ub, 0.55, 0.16)
    assert abs(G.sum() - F.sum()) / F.sum() < 1e-13


def test_uniform_flow_stays_uniform():
    shape = (4, 5, 6)
    kind = np.zeros(shape, np.uint8)
    u = np.broadcast_to(np.array([0.04, -0.02, 0.01]), shape + (3,)).copy()
    F = orc.init(kind, np.zeros((4, 3)), None, u)
    G = orc.run(F, 20, kind, PER, np.zeros((4, 3)), 0.51, 0.16)
    np.testing.assert_allclose(G, F, rtol=0, atol=1e-15)


def test_rest_state_stays_at_rest_in_closed_box():
    faces = ("periodic", "periodic", "periodic", "periodic", "noslip", "noslip")
    rng = np.random.default_rng(5)
    solid = (rng.random((6, 7, 8)) < 0.2).astype(np.uint8)
    kind = orc.classify(solid, faces)
    ub = np.zeros((6, 3))
    F = orc.init(kind, ub, None, np.zeros((6, 7, 8, 3)))
    G = orc.run(F, 30, kind, faces, ub, 0.51, 0.16)
    rho, u = orc.macros(G, kind, ub)
    assert np.abs(u).max() < 1e-16
    np.testing.assert_allclose(rho[kind == 0], 1.0, rtol=0, atol=1e-15)


def test_cube_flow_keeps_mirror_symmetry():
    """No noise and a geometry symmetric about the y mid-plane: u_y stays antisymmetric."""
    case = synth.cube_case(nx=24, ny=16, nz=12, noise=0.0)
    # make the cube symmetric in y on this smaller grid: cells y in [4, 12)
    solid = np.zeros_like(case.solid)
    solid[0:6, 4:12, 8:16] = 1
    kind = orc.classify(solid, case.faces)
    ub = orc.expand_profile(case.speed[:12], 12, 0.0)
    F = orc.init(kind, ub)
    G = orc.run(F, 80, kind, case.faces, ub, 0.52, 0.16)
    _, u = orc.macros(G, kind, ub)
    assert np.abs(u[..., 1]).max() > 1e-6
    np.testing.assert_allclose(u[:, ::-1, :, 1], -u[..., 1], rtol=0, atol=1e-14)
    np.testing.assert_allclose(u[:, ::-1, :, 0], u[..., 0], rtol=0, atol=1e-14)


FACE_SETS = [
    ("inflow", "outflow", "periodic", "periodic", "noslip", "freeslip"),
    ("outflow", "inflow", "inflow", "outflow", "noslip", "freeslip"),
    ("inflow", "outflow", "outflow", "inflow", "noslip", "outflow"),
    ("periodic", "periodic", "noslip", "noslip", "freeslip", "freeslip"),
    ("outflow", "outflow", "outflow", "outflow", "noslip", "inflow"),
    ("freeslip", "outflow", "periodic", "periodic", "noslip", "noslip"),
    ("periodic",) * 6,
]


@pytest.mark.parametrize("faces", FACE_SETS)
@pytest.mark.parametrize("force", [None, (2e-5, -1e-5, 0.0)])
def test_c_oracle_matches_numpy_formulation(faces, force):
    """Brute force: two differently written FP64 programs agree on tiny grids (corners, edges,
    scattered solids, every face kind)."""
    case = synth.random_small_case(8, 6, 5, faces, seed=7, solid_fraction=0.12, margin=0)
    kind = orc.classify(case.solid, faces)
    assert (onp.classify(case.solid, faces) == kind).all()
    ub = orc.expand_profile(case.speed, 5, case.theta)
    F = orc.init(kind, ub, case.rho0, case.u0)
    Fn = onp.reorder_from(F, C)
    for _ in range(6):
        F = orc.step(F, kind, faces, ub, 0.56, 0.16, force=force)
        Fn = onp.step(Fn, kind, faces, ub, 0.56, 0.16, force=force)
    np.testing.assert_allclose(onp.reorder_from(F, C), Fn, rtol=0, atol=1e-15)
    r1, u1 = orc.macros(F, kind, ub, force=force)
    r2, u2 = onp.macros(Fn, kind, ub, force=force)
    np.testing.assert_allclose(u1, u2, rtol=0, atol=1e-15)
    np.testing.assert_allclose(r1, r2, rtol=1e-14, atol=0)


def test_z_range_step_equals_full_step():
    faces = FACE_SETS[1]
    case = synth.random_small_case(8, 6, 5, faces, seed=9)
    kind = orc.classify(case.solid, faces)
    ub = orc.expand_profile(case.speed, 5, 2.0)
    F = orc.init(kind, ub, case.rho0, case.u0)
    full = orc.step(F, kind, faces, ub, 0.55, 0.16)
    part = np.zeros_like(F)
    for z0 in range(5):
        orc.step(F, kind, faces, ub, 0.55, 0.16, z0=z0, z1=z0 + 1, out=part)
    np.testing.assert_array_equal(full, part)


def test_profile_expansion_blocks_and_interpolation():
    sp = np.array([1.0, 2.0, 4.0])
    ub = orc.expand_profile(sp, 6, 0.0)
    np.testing.assert_allclose(ub[:, 0], [1, 1, 2, 2, 4, 4])
    np.testing.assert_allclose(ub[:, 1:], 0.0, atol=0)
    th = math.radians(30)
    ub = orc.expand_profile(sp, 3, th)
    np.testing.assert_allclose(ub[:, 0], sp * math.cos(th))
    np.testing.assert_allclose(ub[:, 1], sp * math.sin(th))
    # 2 levels over 5 cells: centres at 1.25 and 3.75 (heights); cells at 0.5 .. 4.5
    ub = orc.expand_profile(np.array([1.0, 3.0]), 5, 0.0)
    h = np.arange(5) + 0.5
    expect = np.interp(h, [1.25, 3.75], [1.0, 3.0])
    np.testing.assert_allclose(ub[:, 0], expect, rtol=1e-15)

"""Pins of the FP64 oracle's discrete adjoint (oracle/adjoint.py), CPU only.

The adjoint is pinned to things other than itself:
  - its explicit gather map, combined with its complex-capable collision, reproduces the C
    oracle's time step on random states with every face kind (App. D streaming, bounce-back,
    Sec. 3 faces);
  - its collision restatement equals the C oracle's collision (D.1-D.11);
  - its complex-step Jacobians equal central finite differences;
  - the whole gradient of the lidar misfit (speeds and direction) equals central finite
    differences of the FP64 forward model, for equal-height and interpolated level mappings,
    with buildings and several face combinations.
"""
import math

import numpy as np
import pytest

from oracle import adjoint as adj
from oracle import oracle as orc
from paper_2607_04516_b300 import synth

FACE_SETS = [
    ("inflow", "outflow", "periodic", "periodic", "noslip", "freeslip"),
    ("outflow", "inflow", "inflow", "outflow", "noslip", "freeslip"),
    ("inflow", "outflow", "outflow", "inflow", "noslip", "outflow"),
    ("periodic", "periodic", "noslip", "noslip", "freeslip", "freeslip"),
    ("freeslip", "outflow", "periodic", "periodic", "noslip", "noslip"),
    ("periodic",) * 6,
]


@pytest.mark.parametrize("faces", FACE_SETS)
def test_gather_map_reproduces_the_oracle_step(faces):
    case = synth.random_small_case(8, 6, 5, faces, seed=11, solid_fraction=0.12, margin=0)
    kind = orc.classify(case.solid, faces)
    ub = orc.expand_profile(case.speed, 5, case.theta)
    F = orc.init(kind, ub, case.rho0, case.u0)
    ref = orc.step(F, kind, faces, ub, 0.56, 0.16)
    src = adj.gather_map(kind, faces)
    fl = np.nonzero(kind.reshape(-1) == orc.FLUID)[0]
    assert (src[:, fl] >= 0).all()
    mine = adj.collide_c(F.reshape(-1)[src[:, fl]], 0.56, 0.16)
    np.testing.assert_allclose(mine, ref.reshape(19, -1)[:, fl], rtol=0, atol=2e-15)


def test_collision_restatement_matches_c_oracle():
    rng = np.random.default_rng(3)
    _, w, _ = orc.lattice()
    for _ in range(20):
        u = rng.uniform(-0.1, 0.1, 3)
        f = orc.equilibrium(1.0 + rng.uniform(-0.02, 0.02), u) + 2e-3 * rng.standard_normal(19) * w
        ref, _, _ = orc.collide(f, 0.52, 0.16)
        mine = adj.collide_c(f[:, None], 0.52, 0.16)[:, 0]
        np.testing.assert_allclose(mine, ref, rtol=0, atol=1e-15)


def test_complex_step_jacobians_match_finite_differences():
    rng = np.random.default_rng(5)
    _, w, _ = orc.lattice()
    f = np.stack([orc.equilibrium(1.0, rng.uniform(-0.08, 0.08, 3)) + 3e-3 * rng.standard_normal(19) * w
                  for _ in range(6)], axis=1)
    Jac = adj.collision_jacobian(f, 0.51, 0.16)
    h = 1e-6
    for j in range(19):
        fp, fm = f.copy(), f.copy()
        fp[j] += h
        fm[j] -= h
        fd = (adj.collide_c(fp, 0.51, 0.16) - adj.collide_c(fm, 0.51, 0.16)) / (2 * h)
        np.testing.assert_allclose(Jac[:, j], fd, rtol=0, atol=1e-8)
    rho = np.array([1.0, 1.01])
    u = rng.uniform(-0.1, 0.1, (3, 2))
    D = adj.equilibrium_du(rho, u)
    for a in range(3):
        up, um = u.copy(), u.copy()
        up[a] += h
        um[a] -= h
        fd = (adj.equilibrium_c(rho, up) - adj.equilibrium_c(rho, um)) / (2 * h)
        np.testing.assert_allclose(D[:, a], fd, rtol=0, atol=1e-9)


def _problem(faces, L, nz=8, T=24, n_avg=8, seed=0):
    nx, ny = 12, 10
    solid = np.zeros((nz, ny, nx), np.uint8)
    solid[0:4, 4:6, 5:7] = 1
    solid[0:2, 7:8, 8:10] = 1
    cols = [(3, 3), (9, 2), (4, 8)]
    hts = [1, 3, 5]
    p0 = adj.Problem(solid, faces, 0.55, 0.16, T, n_avg, cols, hts, np.zeros((3, 3, 2)), L)
    rng = np.random.default_rng(seed)
    truth_speed = 0.05 + 0.01 * rng.random(L)
    truth = p0.forward(truth_speed, 0.45)[..., :2]
    return adj.Problem(solid, faces, 0.55, 0.16, T, n_avg, cols, hts, truth, L)


def _fd_gradient(prob, speed, theta, h=1e-6):
    out = []
    for l in range(len(speed)):
        e = np.zeros(len(speed))
        e[l] = h
        out.append((prob.loss(speed + e, theta) - prob.loss(speed - e, theta)) / (2 * h))
    out.append((prob.loss(speed, theta + h) - prob.loss(speed, theta - h)) / (2 * h))
    return np.array(out)


@pytest.mark.parametrize("faces,L", [
    (("inflow", "outflow", "inflow", "outflow", "noslip", "freeslip"), 2),    # equal blocks
    (("inflow", "outflow", "inflow", "outflow", "noslip", "freeslip"), 3),    # interpolated
    (("inflow", "outflow", "periodic", "periodic", "noslip", "freeslip"), 4),
    (("inflow", "outflow", "outflow", "inflow", "noslip", "outflow"), 3),
])
def test_adjoint_gradient_matches_central_differences(faces, L):
    prob = _problem(faces, L)
    speed = np.linspace(0.04, 0.06, L)
    theta = 0.4
    J, ds, dth, _ = prob.gradient(speed, theta)
    assert J > 0
    g = np.concatenate([ds, [dth]])
    fd = _fd_gradient(prob, speed, theta)
    assert np.abs(g - fd).max() <= 1e-7 * np.abs(fd).max()


def test_adjoint_gradient_vanishes_at_the_truth():
    faces = ("inflow", "outflow", "inflow", "outflow", "noslip", "freeslip")
    prob = _problem(faces, 2, seed=1)
    rng = np.random.default_rng(1)
    truth_speed = 0.05 + 0.01 * rng.random(2)
    J, ds, dth, _ = prob.gradient(truth_speed, 0.45)
    assert J < 1e-28
    assert np.abs(ds).max() < 1e-12 and abs(dth) < 1e-12

"""Pins of the oracle's relaxation zones and flux balancing (oracle/zones.py), CPU only.

Sec. 3 (boundary paragraph): top sponge and lateral buffer nudging toward the target boundary
state, flux balancing over the open boundaries; Sec. 2.1: smallest normal correction that removes
the net boundary flux.  Pinned by closed forms: from a uniform equilibrium state one step changes
nothing but the nudging, so the velocity deviation of every layer shrinks by exactly 1 - s(d) with
s(d) = sigma ((w - d)/w)^2 and the mass stays; the balanced boundary field has zero net inflow and
differs from the profile by the same normal shift -Phi/A on every cell.
"""
import numpy as np
import pytest

from oracle import oracle as orc
from oracle import zones

C, W, OPP = orc.lattice()


def _uniform(shape, u0, kind):
    F = np.zeros((19,) + shape)
    feq = orc.equilibrium(1.0, u0)
    F[:] = feq[:, None, None, None]
    F[:, kind == orc.SOLID] = 0.0
    return F


def _velocity(F):
    rho = F.sum(axis=0)
    return np.einsum("qa,q...->...a", C.astype(float), F) / rho[..., None], rho


@pytest.mark.parametrize("w,sig", [(1, 1.0), (3, 0.4), (5, 0.25)])
def test_top_sponge_shrinks_each_layer_by_its_ramp(w, sig):
    shape = (8, 5, 6)
    faces = ("periodic",) * 6
    kind = orc.classify(np.zeros(shape, np.uint8), faces)
    u0 = np.array([0.05, -0.02, 0.01])
    ub = np.tile(np.array([0.03, 0.01, 0.0]), (shape[0], 1))
    F = _uniform(shape, u0, kind)
    Fn = zones.run(F, 1, kind, faces, ub, 0.6, 0.16, sponge=(w, sig))
    u, rho = _velocity(Fn)
    np.testing.assert_allclose(rho, 1.0, rtol=0, atol=1e-14)
    for z in range(shape[0]):
        d = shape[0] - 1 - z
        s = sig * ((w - d) / w) ** 2 if d < w else 0.0
        want = ub[z] + (1.0 - s) * (u0 - ub[z])
        np.testing.assert_allclose(u[z], np.broadcast_to(want, u[z].shape), rtol=0, atol=1e-15)


def test_lateral_buffers_only_next_to_open_faces():
    shape = (4, 6, 10)
    faces = ("outflow", "outflow", "periodic", "periodic", "periodic", "periodic")
    kind = orc.classify(np.zeros(shape, np.uint8), faces)
    u0 = np.array([0.04, 0.02, 0.0])
    ub = np.tile(np.array([0.06, 0.0, 0.0]), (shape[0], 1))
    F = _uniform(shape, u0, kind)
    w, sig = 3, 0.5
    Fn = zones.run(F, 1, kind, faces, ub, 0.6, 0.16, buffer=(w, sig))
    u, rho = _velocity(Fn)
    np.testing.assert_allclose(rho, 1.0, rtol=0, atol=1e-14)
    for x in range(shape[2]):
        d = min(x, shape[2] - 1 - x)
        s = sig * ((w - d) / w) ** 2 if d < w else 0.0
        want = ub[0] + (1.0 - s) * (u0 - ub[0])
        np.testing.assert_allclose(u[:, :, x], np.broadcast_to(want, u[:, :, x].shape), rtol=0, atol=1e-15)


def test_overlapping_zones_take_the_larger_rate_and_skip_non_fluid_cells():
    shape = (5, 6, 7)
    faces = ("inflow", "outflow", "outflow", "inflow", "noslip", "freeslip")
    s = zones.zone_rate(shape, faces, sponge=(2, 0.5), buffer=(2, 0.8))
    # corner cell next to the top and the x- face: max(0.5, 0.8)
    assert s[4, 3, 0] == pytest.approx(0.8)
    assert s[4, 3, 3] == pytest.approx(0.5)
    assert s[3, 3, 3] == pytest.approx(0.5 * 0.25)
    assert s[2, 3, 3] == 0.0
    solid = np.zeros(shape, np.uint8)
    solid[0:2, 2:4, 2:4] = 1
    kind = orc.classify(solid, faces)
    F = np.random.default_rng(1).random((19,) + shape) * 0.05
    ub = np.tile(np.array([0.03, 0.01, 0.0]), (shape[0], 1))
    Fn = zones.nudge(F, kind, faces, ub, sponge=(2, 0.5), buffer=(2, 0.8))
    keep = kind != orc.FLUID
    np.testing.assert_array_equal(Fn[:, keep], F[:, keep])


def test_flux_balancing_removes_the_net_inflow_with_one_normal_shift():
    rng = np.random.default_rng(3)
    shape = (6, 9, 11)
    faces = ("inflow", "inflow", "inflow", "outflow", "noslip", "inflow")
    solid = (rng.random(shape) < 0.15).astype(np.uint8)
    kind = orc.classify(solid, faces)
    ub = np.stack([0.04 + 0.01 * rng.random(6), 0.02 * rng.random(6), np.zeros(6)], axis=1)
    ueq, before, after, delta = zones.flux_balanced_ueq(kind, faces, ub)
    own = zones.flux_owner(kind, faces)
    cells = np.argwhere(own >= 0)
    assert len(cells) == int((kind == orc.EQ).sum())
    normals = np.array([(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)], float)
    phi = sum(ub[z] @ normals[own[z, y, x]] for z, y, x in cells)
    assert before == pytest.approx(phi, abs=1e-15)
    assert abs(after) < 1e-14
    assert delta == pytest.approx(-phi / len(cells))
    for z, y, x in cells:
        np.testing.assert_allclose(ueq[z, y, x] - ub[z], delta * normals[own[z, y, x]], rtol=0, atol=1e-16)
    # the uniform shift is the minimum-norm solution of "sum of the normal corrections = -Phi"
    # (least squares of the underdetermined 1 x A system)
    sol = np.linalg.lstsq(np.ones((1, len(cells))), np.array([-phi]), rcond=None)[0]
    np.testing.assert_allclose(sol, delta, rtol=1e-12, atol=0)
    # ownership: the first inflow face in the order x-, x+, y-, y+, z-, z+
    assert own[2, 0, 0] == 0 and own[2, 0, shape[2] - 1] == 1 and own[5, 4, 5] == 5 and own[2, 0, 5] == 2

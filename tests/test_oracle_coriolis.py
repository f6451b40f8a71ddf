"""Pins of the oracle's Coriolis force (paper App. E: F_c = rho 2 Omega^lbm x u, applied through
Guo's forcing).  CPU only."""
import numpy as np
import pytest

from oracle import oracle as orc
from oracle import lbm_numpy as onp
from paper_2607_04516_b300 import synth

C, W, _ = orc.lattice()
PER = ("periodic",) * 6


def _cross_matrix(om):
    ox, oy, oz = om
    return np.array([[0.0, -oz, oy], [oz, 0.0, -ox], [-oy, ox, 0.0]])


@pytest.mark.parametrize("omega", [(0.0, 0.0, 1e-3), (2e-4, -3e-4, 7e-4)])
def test_uniform_flow_rotates_by_the_discrete_inertial_map(omega):
    """A uniform state streams onto itself, and Guo's collision adds exactly F to sum c f; with
    F = 2 Omega x m the momentum obeys m_{n+1} = (I + 2 [Omega x]) m_n."""
    shape = (3, 3, 3)
    kind = np.zeros(shape, np.uint8)
    u0 = np.array([0.04, 0.01, -0.02])
    F = orc.init(kind, np.zeros((3, 3)), None, np.broadcast_to(u0, shape + (3,)).copy())
    m0 = (C.T @ F[:, 0, 0, 0])
    n = 60
    G = orc.run(F, n, kind, PER, np.zeros((3, 3)), 0.8, 0.16, omega=np.array(omega))
    M = np.linalg.matrix_power(np.eye(3) + 2.0 * _cross_matrix(omega), n)
    np.testing.assert_allclose(C.T @ G[:, 1, 2, 0], M @ m0, rtol=0, atol=1e-15)
    assert abs(G[:, 0, 0, 0].sum() - F[:, 0, 0, 0].sum()) < 1e-13     # mass untouched


def test_coriolis_force_direction_follows_the_printed_formula():
    """With Omega along +z and a flow along +x the force 2 rho Omega x u points along +y."""
    f = orc.equilibrium(1.0, [0.05, 0.0, 0.0])
    out, _, _ = orc.collide(f, 0.6, 0.0, omega=[0.0, 0.0, 1e-3])
    dm = C.T @ out - C.T @ f
    np.testing.assert_allclose(dm, [0.0, 2e-3 * 0.05, 0.0], rtol=1e-12, atol=1e-16)


@pytest.mark.parametrize("faces", [
    ("inflow", "outflow", "periodic", "periodic", "noslip", "freeslip"),
    ("outflow", "inflow", "inflow", "outflow", "noslip", "freeslip"),
    ("periodic",) * 6,
])
def test_c_oracle_matches_numpy_formulation_with_rotation(faces):
    case = synth.random_small_case(8, 6, 5, faces, seed=17, solid_fraction=0.12, margin=0)
    kind = orc.classify(case.solid, faces)
    ub = orc.expand_profile(case.speed, 5, case.theta)
    F = orc.init(kind, ub, case.rho0, case.u0)
    Fn = onp.reorder_from(F, C)
    om = np.array([1e-3, -2e-3, 3e-3])
    force = (1e-5, 0.0, -2e-5)
    for _ in range(5):
        F = orc.step(F, kind, faces, ub, 0.56, 0.16, force=force, omega=om)
        Fn = onp.step(Fn, kind, faces, ub, 0.56, 0.16, force=force, omega=om)
    np.testing.assert_allclose(onp.reorder_from(F, C), Fn, rtol=0, atol=1e-15)

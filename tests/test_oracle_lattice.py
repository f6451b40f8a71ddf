"""Pins of the oracle's lattice, equilibrium, collision and LES closure against what the
mathematics fixes (paper App. D).  CPU only."""
import itertools

import numpy as np
import pytest

from oracle import oracle as orc

RNG = np.random.default_rng(12345)


def test_velocity_set_is_d3q19():
    c, w, opp = orc.lattice()
    assert c.shape == (19, 3)
    assert len({tuple(v) for v in c}) == 19
    assert set(map(tuple, c)) == {v for v in itertools.product((-1, 0, 1), repeat=3)
                                  if sum(x * x for x in v) <= 2}
    for i in range(19):
        assert (c[opp[i]] == -c[i]).all()


def test_weights_isotropy_2nd_and_4th_order():
    """App. D: weights satisfy the 2nd- and 4th-order isotropy constraints with c_s^2 = 1/3."""
    c, w, _ = orc.lattice()
    cs2 = 1.0 / 3.0
    d = np.eye(3)
    assert abs(w.sum() - 1.0) < 1e-15
    np.testing.assert_allclose(np.einsum("q,qa->a", w, c), 0.0, atol=1e-16)
    np.testing.assert_allclose(np.einsum("q,qa,qb->ab", w, c, c), cs2 * d, atol=1e-16)
    np.testing.assert_allclose(np.einsum("q,qa,qb,qc->abc", w, c, c, c), 0.0, atol=1e-16)
    iso4 = cs2 ** 2 * (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
                       + np.einsum("ad,bc->abcd", d, d))
    np.testing.assert_allclose(np.einsum("q,qa,qb,qc,qd->abcd", w, c, c, c, c), iso4, atol=1e-16)


def test_weights_are_the_unique_isotropic_solution():
    """The three shell weights are fixed by sum w = 1, sum w c_x^2 = c_s^2, sum w c_x^2 c_y^2 =
    c_s^4: solving that system independently must give the oracle's weights."""
    c, w, _ = orc.lattice()
    shell = (c ** 2).sum(1)
    A = np.array([[1, 6, 12], [0, 2, 8], [0, 0, 4]], float)   # counts per shell
    b = np.array([1.0, 1 / 3, 1 / 9])
    w_shell = np.linalg.solve(A, b)
    np.testing.assert_allclose(w, w_shell[shell], rtol=1e-15)


@pytest.mark.parametrize("trial", range(5))
def test_equilibrium_moments(trial):
    """D.4 reproduces rho, rho u and rho c_s^2 delta + rho u u exactly (D3Q19, 2nd order)."""
    c, _, _ = orc.lattice()
    rho = 1.0 + RNG.uniform(-0.1, 0.1)
    u = RNG.uniform(-0.1, 0.1, 3)
    feq = orc.equilibrium(rho, u)
    assert abs(feq.sum() - rho) < 1e-15
    np.testing.assert_allclose(c.T @ feq, rho * u, atol=1e-16)
    np.testing.assert_allclose(np.einsum("qa,qb,q->ab", c, c, feq),
                               rho / 3 * np.eye(3) + rho * np.outer(u, u), atol=1e-15)


def _neq_with_flux(P):
    """Non-equilibrium part with prescribed second moment P and zero mass/momentum:
    f^neq_i = w_i (9/2)(c_i c_i - delta/3) : P (Hermite projection, exact on D3Q19)."""
    c, w, _ = orc.lattice()
    H = np.einsum("qa,qb->qab", c, c) - np.eye(3) / 3.0
    return w * 4.5 * np.einsum("qab,ab->q", H, P)


@pytest.mark.parametrize("trial", range(5))
def test_collision_conserves_mass_momentum_and_relaxes_stress(trial):
    """D.2: BGK keeps rho and rho u; the non-equilibrium flux relaxes by (1 - 1/tau_eff)."""
    c, _, _ = orc.lattice()
    rho = 1.0 + RNG.uniform(-0.05, 0.05)
    u = RNG.uniform(-0.08, 0.08, 3)
    P = RNG.uniform(-1e-3, 1e-3, (3, 3))
    P = 0.5 * (P + P.T)
    f = orc.equilibrium(rho, u) + _neq_with_flux(P)
    out, Q, te = orc.collide(f, 0.55, 0.16)
    assert abs(out.sum() - f.sum()) < 1e-15
    np.testing.assert_allclose(c.T @ out, c.T @ f, atol=1e-16)
    pi_out = np.einsum("qa,qb,q->ab", c, c, out - orc.equilibrium(rho, u))
    np.testing.assert_allclose(pi_out, (1.0 - 1.0 / te) * P, atol=1e-15)


@pytest.mark.parametrize("tau,C", [(0.505, 0.16), (0.52, 0.16), (0.8, 0.1), (0.5000002, 0.16)])
def test_tau_eff_solves_the_smagorinsky_relation(tau, C):
    """D.11 must be the positive root of c_s^2 (tau_eff - tau) = (C Delta)^2 |S| with
    |S| = Q / (2 rho c_s^2 tau_eff) (D.5-D.7, D.10); Q is checked against a prescribed flux."""
    cs2 = 1.0 / 3.0
    rho = 1.0 + RNG.uniform(-0.05, 0.05)
    u = RNG.uniform(-0.05, 0.05, 3)
    P = RNG.uniform(-1e-3, 1e-3, (3, 3))
    P = 0.5 * (P + P.T)
    f = orc.equilibrium(rho, u) + _neq_with_flux(P)
    _, Q, te = orc.collide(f, tau, C)
    assert Q == pytest.approx(np.sqrt(2.0 * (P * P).sum()), rel=1e-12)
    S = Q / (2.0 * rho * cs2 * te)
    assert cs2 * (te - tau) == pytest.approx(C ** 2 * S, rel=1e-12, abs=1e-18)
    assert te > tau


def test_tau_eff_limits():
    assert orc.tau_eff(0.6, 0.16, 0.0, 1.0) == 0.6
    assert orc.tau_eff(0.6, 0.0, 1e-3, 1.0) == 0.6
    # large-Q limit: tau_eff ~ sqrt(2 C^2 Q / (rho c_s^4)) / 2 * (1 + ...)
    te = orc.tau_eff(0.5, 0.16, 1e4, 1.0)
    assert te == pytest.approx(0.5 * np.sqrt(2 * 0.16 ** 2 * 1e4 * 9), rel=1e-2)


def test_guo_force_moments():
    """Guo forcing: mass kept, momentum gains exactly F (sum c f* = sum c f + F)."""
    c, _, _ = orc.lattice()
    f = orc.equilibrium(1.02, [0.03, -0.01, 0.02]) + _neq_with_flux(np.diag([1e-4, -2e-4, 1e-4]))
    F = np.array([1e-5, -2e-5, 3e-5])
    out, _, _ = orc.collide(f, 0.7, 0.0, force=F)
    assert abs(out.sum() - f.sum()) < 1e-15
    np.testing.assert_allclose(c.T @ out, c.T @ f + F, atol=1e-17)

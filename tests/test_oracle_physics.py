"""Pins of the oracle against closed-form flows (paper App. D: viscosity-relaxation relation D.5,
Chapman-Enskog strain link D.9-D.10, bounce-back walls; Guo forcing for the channel).  CPU only."""
import math

import numpy as np
import pytest

from oracle import oracle as orc
from paper_2607_04516_b300 import synth

C, W, _ = orc.lattice()
PER = ("periodic",) * 6


def _tg_energy_rate(n, tau, cs, t0=40, t1=240, nz=1):
    case = synth.taylor_green_case(n=n, U0=0.01, tau=tau, cs=cs, nz=nz)
    kind = orc.classify(case.solid, PER)
    ub = np.zeros((nz, 3))
    F = orc.init(kind, ub, None, case.u0)
    ts, es = [], []
    buf = np.empty_like(F)
    for t in range(1, t1 + 1):
        orc.step(F, kind, PER, ub, tau, cs, out=buf)
        F, buf = buf, F
        if t >= t0 and t % 10 == 0:
            _, u = orc.macros(F, kind, ub)
            ts.append(t)
            es.append(float((u ** 2).sum()))
    slope = np.polyfit(ts, np.log(es), 1)[0]
    return -slope


def test_taylor_green_decay_rate_matches_viscosity():
    """Kinetic energy of the 2D TG vortex decays as exp(-4 nu k^2 t), nu = (tau - 1/2)/3."""
    n, tau = 32, 0.8
    nu = (tau - 0.5) / 3.0
    k = 2 * math.pi / n
    rate = _tg_energy_rate(n, tau, 0.0)
    assert rate == pytest.approx(4 * nu * k * k, rel=1e-2)


def test_taylor_green_converges_second_order():
    tau = 0.8
    nu = (tau - 0.5) / 3.0
    errs = []
    for n in (16, 32, 64):
        k = 2 * math.pi / n
        scale = (n / 16) ** 2        # same number of decay times on every grid (diffusive scaling)
        rate = _tg_energy_rate(n, tau, 0.0, t0=int(10 * scale), t1=int(60 * scale))
        errs.append(abs(rate / (4 * nu * k * k) - 1.0))
    order1 = math.log2(errs[0] / errs[1])
    order2 = math.log2(errs[1] / errs[2])
    assert order1 > 1.7 and order2 > 1.7, errs


def test_smagorinsky_adds_dissipation():
    base = _tg_energy_rate(32, 0.51, 0.0)
    les = _tg_energy_rate(32, 0.51, 0.16)
    assert les > base * 1.01


def _central_strain(u):
    """|S| = sqrt(2 S:S) from second-order central differences of a periodic field u (nz,ny,nx,3)."""
    grad = np.zeros(u.shape[:3] + (3, 3))
    for a, ax in ((0, 2), (1, 1), (2, 0)):
        grad[..., a, :] = (np.roll(u, -1, axis=ax) - np.roll(u, 1, axis=ax)) / 2.0
    S = 0.5 * (grad + np.swapaxes(grad, -1, -2))      # grad[..., a, b] = d_a u_b
    return np.sqrt(2.0 * (S * S).sum(axis=(-1, -2)))


def test_strain_from_nonequilibrium_flux_matches_velocity_gradient():
    """D.9/D.10: |S| recovered locally as Q / (2 rho c_s^2 tau) agrees with the finite-difference
    strain rate of the velocity field, with error falling at second order in the spacing."""
    tau = 0.8
    errs = []
    for n in (16, 32, 64):
        case = synth.taylor_green_case(n=n, U0=0.01, tau=tau, cs=0.0, nz=1)
        kind = orc.classify(case.solid, PER)
        ub = np.zeros((1, 3))
        F = orc.init(kind, ub, None, case.u0)
        F = orc.run(F, n * n // 16, kind, PER, ub, tau, 0.0)
        # Q of a step belongs to the populations that step gathers; the velocity it observes is
        # the moment of the same populations
        G, Q, te = orc.step(F, kind, PER, ub, tau, 0.0, diag=True)
        rho, u1 = orc.macros(G, kind, ub)
        s_lb = Q / (2.0 * rho * (1.0 / 3.0) * te)
        s_fd = _central_strain(u1)
        errs.append(np.linalg.norm(s_lb - s_fd) / np.linalg.norm(s_fd))
    assert errs[-1] < 0.01, errs
    assert math.log2(errs[0] / errs[1]) > 1.6 and math.log2(errs[1] / errs[2]) > 1.6, errs


def _channel_profile(nz, tau, force=1e-6, steps=None):
    case = synth.channel_case(nz=nz, nxy=1, force=force, tau=tau)
    kind = orc.classify(case.solid, case.faces)
    ub = np.zeros((nz, 3))
    F = orc.init(kind, ub, None, case.u0)
    nu = (tau - 0.5) / 3.0
    steps = steps or int(12 * nz * nz / nu)
    F = orc.run(F, steps, kind, case.faces, ub, tau, 0.0, force=case.force)
    rho, u = orc.macros(F, kind, ub, force=case.force)
    z = np.arange(nz)
    exact = force / (2.0 * nu) * (z + 0.5) * (nz - 0.5 - z)
    return u[:, 0, 0, 0], exact, u


def test_poiseuille_exact_at_magic_tau():
    """BGK + mid-grid bounce-back + Guo forcing reproduce the parabolic channel profile with the
    walls exactly half a spacing outside the last fluid cells when tau = 1/2 + sqrt(3/16)."""
    tau = 0.5 + math.sqrt(3.0 / 16.0)
    got, exact, u = _channel_profile(16, tau)
    np.testing.assert_allclose(got, exact, rtol=1e-9, atol=0)
    assert np.abs(u[..., 1:]).max() < 1e-13 * np.abs(got).max() * 1e4


def test_poiseuille_converges_second_order_off_magic_tau():
    errs = []
    for nz in (8, 16, 32):
        got, exact, _ = _channel_profile(nz, 0.6)
        errs.append(np.abs(got - exact).max() / exact.max())
    assert math.log2(errs[0] / errs[1]) > 1.8 and math.log2(errs[1] / errs[2]) > 1.8, errs

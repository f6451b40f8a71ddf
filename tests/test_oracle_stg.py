"""Pins of the oracle's synthetic von Karman inflow turbulence (paper App. F).  CPU only.

The mode sum is checked through properties of its output rather than by retyping it:
  - phase averaging: shifting mode m's phases by 2 pi k m / K (K = 2 N_m + 1, k = 0..K-1) kills
    every cross term, so the average of (U - U_b)^2 is exactly sigma^2 g^2 sum A_m^2 / 2, which the
    amplitude normalisation fixes to sigma^2 g^2;
  - quarter-period phase shifts turn one mode into a complex amplitude whose ratios between
    neighbouring cells / steps measure the wave vector and the frequency;
  - closed forms of the log-spaced wavenumbers (endpoints, geometric mean), isotropy of the
    sampled directions, Kolmogorov's -5/3 range of the von Karman spectrum, frozen convection.
"""
import math

import numpy as np
import pytest

from oracle import oracle as orc

FACES = ("inflow", "outflow", "inflow", "outflow", "noslip", "freeslip")
SHAPE = (4, 5, 6)                       # nz, ny, nx


def _kind(faces=FACES, shape=SHAPE):
    return orc.classify(np.zeros(shape, np.uint8), faces)


def _ub(u, nz=SHAPE[0]):
    return np.broadcast_to(np.asarray(u, np.float64), (nz, 3)).copy()


def _dev(kind, faces, ub, P, rnd, t):
    U = orc.stg(kind, faces, ub, P, rnd, t)
    base = np.where((kind == orc.EQ)[..., None], ub[:, None, None, :], 0.0)
    return U - base


def _rnd(n_modes, seed=0):
    return np.random.default_rng(seed).random((6, n_modes, 6))


def _with_phase_shift(rnd, shifts):
    """shifts (n_modes,) in units of 2 pi, applied to all three phases of every face."""
    out = rnd.copy()
    out[:, :, 3:] = np.mod(out[:, :, 3:] + np.asarray(shifts)[None, :, None], 1.0)
    return out


def _complex_amplitude(kind, faces, ub, P, rnd, t):
    """For one mode: dev(phi) - i dev(phi + pi/2) = sigma g sqrt(2) exp(i (k.x + omega t + phi))."""
    a = _dev(kind, faces, ub, P, rnd, t)
    b = _dev(kind, faces, ub, P, _with_phase_shift(rnd, [0.25]), t)
    return a - 1j * b


@pytest.mark.parametrize("char_normal", [False, True])
@pytest.mark.parametrize("n_modes", [1, 3, 5])
def test_phase_averaged_variance_is_sigma_squared(char_normal, n_modes):
    """<(U - U_b)_a^2> over the K phase shifts = (I u_char g_a)^2 at every turbulent cell."""
    kind = _kind()
    u = np.array([0.05, 0.03, 0.0])                   # oblique: |U| != |U . n|
    ub = _ub(u)
    gain = (1.0, 0.5, 0.8)
    I = 0.12
    P = orc.stg_params(n_modes=n_modes, L=6.0, I=I, gain=gain, char_normal=char_normal)
    rnd = _rnd(n_modes, seed=3)
    K = 2 * n_modes + 1
    m = np.arange(1, n_modes + 1)
    acc = 0.0
    for k in range(K):
        acc = acc + _dev(kind, FACES, ub, P, _with_phase_shift(rnd, k * m / K), 7) ** 2
    acc /= K
    nz, ny, nx = SHAPE
    west = np.zeros(SHAPE, bool)
    west[:, :, 0] = True
    south = np.zeros(SHAPE, bool)
    south[:, 0, 1:] = True
    for mask, normal in ((west, np.array([1.0, 0, 0])), (south, np.array([0, 1.0, 0]))):
        uchar = abs(u @ normal) if char_normal else np.linalg.norm(u)
        want = (I * uchar * np.asarray(gain)) ** 2
        np.testing.assert_allclose(acc[mask], np.broadcast_to(want, (mask.sum(), 3)),
                                   rtol=1e-10, atol=0)
    others = (kind == orc.EQ) & ~west & ~south
    assert others.sum() == 0 or np.all(acc[others] == 0)


def test_sigma0_used_when_intensity_is_not_positive():
    kind = _kind()
    ub = _ub([0.04, 0.0, 0.0])
    P = orc.stg_params(n_modes=2, L=5.0, I=0.0, sigma0=3e-3)
    rnd = _rnd(2, seed=5)
    K = 5
    acc = sum(_dev(kind, FACES, ub, P, _with_phase_shift(rnd, k * np.arange(1, 3) / K), 0) ** 2
              for k in range(K)) / K
    np.testing.assert_allclose(acc[:, :, 0], 9e-6, rtol=1e-10)


def _measure_k(P, rnd1, u=(0.05, 0.0, 0.0)):
    """Wave vector of a single mode: k_y, k_z from the west face, k_x from the south face (both
    faces get the same mode)."""
    kind = _kind()
    r = rnd1.copy()
    r[2] = r[0]
    Z = _complex_amplitude(kind, FACES, _ub(u), P, r, 0)
    ky = np.angle(Z[1, 2, 0, 0] / Z[1, 1, 0, 0])
    kz = np.angle(Z[2, 1, 0, 0] / Z[1, 1, 0, 0])
    kx = np.angle(Z[1, 0, 3, 0] / Z[1, 0, 2, 0])
    # the same ratios hold for every component and every neighbouring pair
    np.testing.assert_allclose(np.angle(Z[1, 3, 0, 1] / Z[1, 2, 0, 1]), ky, atol=1e-9)
    np.testing.assert_allclose(np.angle(Z[1, 0, 4, 2] / Z[1, 0, 3, 2]), kx, atol=1e-9)
    return np.array([kx, ky, kz])


@pytest.mark.parametrize("L,r,want", [
    (8.0, 0.0, 2 * math.pi / 80.0),                                   # xi = 0: k_min = 2 pi / 10 L
    (8.0, 0.5, math.sqrt(2 * math.pi / 80.0 * math.pi)),              # geometric mean of the ends
    (0.1, 0.0, 0.1 * math.pi),                                        # k_min >= k_max: 0.1 k_max
])
def test_single_mode_wavenumber_closed_forms(L, r, want):
    P = orc.stg_params(n_modes=1, L=L, I=0.1)
    rnd = _rnd(1, seed=11)
    rnd[:, 0, 0] = r
    k = _measure_k(P, rnd)
    assert np.linalg.norm(k) == pytest.approx(want, rel=1e-9)


def test_sampled_wave_directions_are_isotropic():
    P = orc.stg_params(n_modes=1, L=8.0, I=0.1)
    rng = np.random.default_rng(2024)
    dirs = []
    for _ in range(300):
        rnd = rng.random((6, 1, 6))
        rnd[:, 0, 0] = 0.3
        k = _measure_k(P, rnd)
        dirs.append(k / np.linalg.norm(k))
    d = np.array(dirs)
    assert np.abs(d.mean(axis=0)).max() < 0.12                       # 3.6 sigma of 1/sqrt(900)
    M = d.T @ d / len(d)
    np.testing.assert_allclose(M, np.eye(3) / 3, atol=0.07)


def test_spectrum_follows_kolmogorov_in_the_inertial_range():
    """Two modes with k L >> 1: A_0^2 / A_1^2 = (k_0 / k_1)^(-5/3) (1 + O((kL)^-2))."""
    L = 1000.0
    P = orc.stg_params(n_modes=2, L=L, I=0.1)
    rnd = _rnd(2, seed=8)
    rnd[:, :, 0] = 0.9                                                # xi = 0.45 and 0.95
    kind = _kind()
    ub = _ub([0.05, 0.0, 0.0])
    amp2 = []
    for j in range(2):                                                # isolate mode j
        sh = np.zeros(2)
        vals = []
        for q in range(4):
            sh[j] = q / 4
            vals.append(_dev(kind, FACES, ub, P, _with_phase_shift(rnd, sh), 0)[1, 1, 0, 0])
        amp2.append((vals[0] - vals[2]) ** 2 + (vals[1] - vals[3]) ** 2)   # 4 (sigma A_j)^2
    kmin, kmax = 2 * math.pi / (10 * L), math.pi
    k0 = kmin * (kmax / kmin) ** 0.45
    k1 = kmin * (kmax / kmin) ** 0.95
    assert amp2[0] / amp2[1] == pytest.approx((k0 / k1) ** (-5.0 / 3.0), rel=0.01)
    # and the normalisation: the two amplitudes squared sum to 2 (unit variance)
    sigma = 0.1 * 0.05
    assert (amp2[0] + amp2[1]) / (4 * sigma ** 2) == pytest.approx(2.0, rel=1e-10)


def test_frozen_convection_with_the_printed_phase_sign():
    """omega = u_ref k . e_c enters as +omega t, so q(x, t) = q(x + u_ref e_c t, 0)."""
    kind = _kind(shape=(3, 4, 9))
    ub = _ub([0.05, 0.0, 0.0], nz=3)
    P = orc.stg_params(n_modes=8, L=4.0, I=0.1)
    rnd = _rnd(8, seed=21)
    rnd[2] = rnd[0]
    d20 = _dev(kind, FACES, ub, P, rnd, 20)                           # u_ref t = 1 cell
    d0 = _dev(kind, FACES, ub, P, rnd, 0)
    np.testing.assert_allclose(d20[:, 0, 1:-2], d0[:, 0, 2:-1], rtol=0, atol=1e-15)
    assert np.abs(d20[:, 0, 1:-2] - d0[:, 0, 1:-2]).max() > 1e-4      # the field does move


def test_reference_speed_is_the_mean_speed_of_the_turbulent_cells():
    """omega / k_x measured on a sheared profile equals the brute-force mean |U_b|."""
    faces = FACES
    nz = SHAPE[0]
    speeds = np.array([0.02, 0.04, 0.05, 0.07])
    ub = np.zeros((nz, 3))
    ub[:, 0] = speeds
    kind = _kind()
    P = orc.stg_params(n_modes=1, L=6.0, I=0.1)
    rnd = _rnd(1, seed=4)
    rnd[2] = rnd[0]
    Z0 = _complex_amplitude(kind, faces, ub, P, rnd, 0)
    Z1 = _complex_amplitude(kind, faces, ub, P, rnd, 1)
    omega = np.angle(Z1[2, 0, 3, 0] / Z0[2, 0, 3, 0])
    kx = np.angle(Z0[2, 0, 3, 0] / Z0[2, 0, 2, 0])
    turbulent = np.zeros(SHAPE, bool)
    turbulent[:, :, 0] = True
    turbulent[:, 0, :] = True
    uref = speeds[np.nonzero(turbulent)[0]].mean()
    assert omega / kx == pytest.approx(uref, rel=1e-9)


@pytest.mark.parametrize("interpolate", [False, True])
def test_temporal_stride_holds_or_interpolates_between_anchors(interpolate):
    kind = _kind()
    ub = _ub([0.05, 0.01, 0.0])
    rnd = _rnd(4, seed=9)
    P1 = orc.stg_params(n_modes=4, L=5.0, I=0.1, stride=1)
    Ps = orc.stg_params(n_modes=4, L=5.0, I=0.1, stride=5, interpolate=interpolate)
    for t in (10, 12, 14, 15):
        got = orc.stg(kind, FACES, ub, Ps, rnd, t)
        if not interpolate or t % 5 == 0:
            want = orc.stg(kind, FACES, ub, P1, rnd, (t // 5) * 5)
        else:
            al = (t % 5) / 5
            want = (1 - al) * orc.stg(kind, FACES, ub, P1, rnd, 10) + \
                al * orc.stg(kind, FACES, ub, P1, rnd, 15)
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-15)


def test_face_ownership_and_exclusions():
    faces = ("inflow", "inflow", "inflow", "inflow", "inflow", "inflow")
    shape = (4, 5, 6)
    kind = _kind(faces, shape)
    ub = _ub([0.05, 0.0, 0.0])
    P = orc.stg_params(n_modes=3, L=5.0, I=0.1, char_normal=True)
    rnd = _rnd(3, seed=1)
    d = _dev(kind, faces, ub, P, rnd, 3)
    # the ground is never turbulent; south/north/top faces have U . n = 0 and are dropped
    assert np.all(d[0, 1:-1, 1:-1] == 0)
    assert np.all(d[1:, 0, 1:-1] == 0) and np.all(d[1:, -1, 1:-1] == 0)
    assert np.all(d[-1, 1:-1, 1:-1] == 0)
    # west and east own their whole faces, including the edges and the ground row
    assert np.all(np.abs(d[:, :, 0]).max(axis=-1) > 0)
    assert np.all(np.abs(d[:, :, -1]).max(axis=-1) > 0)
    # the west face's modes are its own: changing another face's draws leaves it alone
    r2 = rnd.copy()
    r2[1] = _rnd(3, seed=99)[1]
    d2 = _dev(kind, faces, ub, P, r2, 3)
    np.testing.assert_array_equal(d2[:, :, 0], d[:, :, 0])
    assert np.abs(d2[:, :, -1] - d[:, :, -1]).max() > 1e-6
    # inflow_only keeps the east face (U . n_in < 0) laminar
    Pi = orc.stg_params(n_modes=3, L=5.0, I=0.1, char_normal=True, inflow_only=True)
    di = _dev(kind, faces, ub, Pi, rnd, 3)
    assert np.all(di[:, :, -1] == 0)
    assert np.all(np.abs(di[:, :, 0]).max(axis=-1) > 0)
    # a cell that is not an equilibrium cell reports zero
    U = orc.stg(kind, faces, ub, P, rnd, 3)
    assert np.all(U[kind != orc.EQ] == 0)


def test_south_edge_cells_belong_to_the_west_face():
    kind = _kind()
    ub = _ub([0.05, 0.02, 0.0])
    P = orc.stg_params(n_modes=2, L=5.0, I=0.1)
    rnd = _rnd(2, seed=6)
    d = _dev(kind, FACES, ub, P, rnd, 0)
    r2 = rnd.copy()
    r2[2] = _rnd(2, seed=7)[2]                                        # new south-face draws
    d2 = _dev(kind, FACES, ub, P, r2, 0)
    np.testing.assert_array_equal(d2[:, :, 0], d[:, :, 0])            # x = 0 column: west
    assert np.abs(d2[:, 0, 1:] - d[:, 0, 1:]).max() > 1e-6

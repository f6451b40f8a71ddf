"""GPU parity of the synthetic von Karman inflow turbulence (App. F): the sm_103a kernel that sets
the inflow faces' equilibrium velocities before each step, and the fused step driven by them,
against the FP64 oracle (oracle_stg + oracle_step with per-cell equilibrium velocities)."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2607_04516_b300 import synth

from gpu_common import (TOL_U, f32, f64_of_f32, gpu_domain, lib_to_oracle_order, oracle_inputs,
                        oracle_run, rel_l2)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_04516_b300 import build
    build.build()


def _oracle_params(kw):
    """Oracle parameters from the library's keyword set, rounded to FP32 as the library holds them."""
    r = lambda v: float(np.float32(v))
    return orc.stg_params(n_modes=kw.get("n_modes", 64), L=r(kw.get("length", 20.0)),
                          I=r(kw.get("intensity", 0.1)), sigma0=r(kw.get("sigma0", 0.0)),
                          gain=[r(g) for g in kw.get("gain", (1.0, 1.0, 1.0))],
                          char_normal=kw.get("char_normal", False),
                          inflow_only=kw.get("inflow_only", False), stride=kw.get("stride", 1),
                          interpolate=kw.get("interpolate", True))


def _oracle_run_stg(case, nsteps, kw, rnd):
    kind, ub = oracle_inputs(case)
    P = _oracle_params(kw)
    fz = None if case.force is None else f64_of_f32(case.force)
    om = None if case.coriolis is None else f64_of_f32(case.coriolis)
    F = orc.init(kind, ub, f64_of_f32(case.rho0), f64_of_f32(case.u0), case.rho_b)
    ueq = None
    for t in range(nsteps):
        ueq = orc.stg(kind, case.faces, ub, P, rnd, t)
        F = orc.step(F, kind, case.faces, ub, case.tau, case.cs, force=fz, rho_b=case.rho_b,
                     omega=om, ueq=ueq)
    rho, u = orc.macros(F, kind, ub, case.rho_b, fz, ueq=ueq)
    return rho, u, F, kind, ub


def _gpu_run_stg(case, nsteps, kw, rnd, store="f32"):
    dom = gpu_domain(case, store)
    dom.configure_stg(rnd, **kw)
    dom.step(nsteps)
    return dom


FACE_SETS = [
    ("inflow", "outflow", "inflow", "outflow", "noslip", "freeslip"),
    ("outflow", "inflow", "outflow", "inflow", "noslip", "inflow"),
    ("inflow", "inflow", "inflow", "inflow", "inflow", "inflow"),
    ("periodic", "periodic", "inflow", "outflow", "noslip", "freeslip"),
]
PARAMS = [
    dict(n_modes=16, length=4.0, intensity=0.1),
    dict(n_modes=8, length=3.0, intensity=0.2, gain=(1.0, 0.6, 0.3), char_normal=True),
    dict(n_modes=8, length=3.0, intensity=0.15, inflow_only=True, stride=3, interpolate=True),
    dict(n_modes=5, length=6.0, intensity=0.0, sigma0=3e-3, stride=4, interpolate=False),
    dict(n_modes=300, length=0.05, intensity=0.1),                    # degenerate band, many modes
]


def _small_case(faces, seed):
    case = synth.random_small_case(13, 7, 6, faces, seed=seed, solid_fraction=0.12, margin=0)
    case.speed = np.array([0.03, 0.05, 0.06])
    case.theta = 0.6
    return case


@pytest.mark.parametrize("faces", FACE_SETS)
@pytest.mark.parametrize("pi", range(len(PARAMS)))
@pytest.mark.parametrize("nsteps", [1, 6])
def test_equilibrium_cell_velocity_matches_oracle(faces, pi, nsteps):
    """U_i(t) of every equilibrium cell after nsteps (t = nsteps - 1) vs oracle_stg."""
    kw = PARAMS[pi]
    case = _small_case(faces, seed=31 + pi)
    rnd = synth.stg_uniforms(kw["n_modes"], seed=100 + pi)
    dom = _gpu_run_stg(case, nsteps, kw, rnd)
    rho, u = dom.macroscopic()
    u = u.cpu().numpy().astype(np.float64)
    kind, ub = oracle_inputs(case)
    want = orc.stg(kind, faces, ub, _oracle_params(kw), rnd, nsteps - 1)
    eq = kind == orc.EQ
    assert eq.any()
    err = np.abs(u[eq] - want[eq]).max()
    assert err <= 1e-7, err
    np.testing.assert_allclose(rho.cpu().numpy()[eq], case.rho_b, rtol=0, atol=0)


def test_reference_speed_and_direction_are_the_brute_force_means():
    faces = FACE_SETS[0]
    case = _small_case(faces, seed=3)
    kw = dict(n_modes=4, length=4.0, intensity=0.1)
    dom = _gpu_run_stg(case, 0, kw, synth.stg_uniforms(4, seed=1))
    u_ref, e_c, kept = dom.stg_reference()
    kind, ub = oracle_inputs(case)
    nz, ny, nx = kind.shape
    mask = np.zeros(kind.shape, bool)
    mask[:, :, 0] = True                                              # x- face
    mask[:, 0, :] = True                                              # y- face
    mask &= kind == orc.EQ
    ub32 = ub.astype(np.float32).astype(np.float64)                   # the library holds FP32 u_b
    U = np.broadcast_to(ub32[:, None, None, :], kind.shape + (3,))[mask]
    assert u_ref == pytest.approx(np.linalg.norm(U, axis=1).mean(), rel=1e-12)
    s = U.sum(0)
    np.testing.assert_allclose(e_c, s / np.linalg.norm(s), rtol=0, atol=1e-14)
    assert kept == (1 << 0) | (1 << 2)


@pytest.mark.parametrize("faces", FACE_SETS)
@pytest.mark.parametrize("pi", [0, 2, 3])
@pytest.mark.parametrize("nsteps", [1, 2, 7])
def test_small_lattices_with_inflow_turbulence_populations(faces, pi, nsteps):
    """Post-collision populations, element by element, after steps driven by the turbulent
    inflow (13 x 7 x 6 lattice, solids on the faces)."""
    kw = PARAMS[pi]
    case = _small_case(faces, seed=41 + pi)
    rnd = synth.stg_uniforms(kw["n_modes"], seed=200 + pi)
    dom = _gpu_run_stg(case, nsteps, kw, rnd)
    g = dom.export_populations().cpu().numpy()
    _, _, F, kind, _ = _oracle_run_stg(case, nsteps, kw, rnd)
    _, wo, _ = orc.lattice()
    G = g[lib_to_oracle_order()] + wo[:, None, None, None]
    diff = np.abs(G - F)[:, kind != orc.SOLID]
    assert diff.max() <= 2e-6, diff.max()


@pytest.mark.parametrize("store", ["f32", "f16s"])
def test_cube_with_inflow_turbulence(store):
    """The cube flow fed by a turbulent west inflow (I = 0.1, L = 8, 64 modes) for 200 steps."""
    case = synth.cube_case()
    kw = dict(n_modes=64, length=8.0, intensity=0.1)
    rnd = synth.stg_uniforms(64, seed=5)
    dom = _gpu_run_stg(case, 200, kw, rnd, store)
    rho, u = dom.macroscopic()
    u = u.cpu().numpy().astype(np.float64)
    _, ur, _, kind, _ = _oracle_run_stg(case, 200, kw, rnd)
    _, u_lam, _, _, _ = oracle_run(synth.cube_case(), 200)
    fl = kind == orc.FLUID
    assert rel_l2(ur, u_lam, fl) > 10 * TOL_U[store]                 # the inflow turbulence matters
    assert rel_l2(u, ur, fl) <= TOL_U[store]


def test_disable_and_profile_change():
    faces = FACE_SETS[0]
    case = _small_case(faces, seed=9)
    kw = dict(n_modes=8, length=4.0, intensity=0.1)
    rnd = synth.stg_uniforms(8, seed=2)
    dom = _gpu_run_stg(case, 3, kw, rnd)
    kind, ub = oracle_inputs(case)
    eq = kind == orc.EQ
    # a new profile rebuilds the tables (u_ref and e_c follow it) and the next step uses them
    speed2 = np.array([0.02, 0.04], np.float32)
    dom.set_inflow_profile(speed2, 0.3)
    u_ref, _, _ = dom.stg_reference()
    ub2 = orc.expand_profile(speed2.astype(np.float64), kind.shape[0], float(np.float32(0.3)))
    dom.step(1)
    _, u = dom.macroscopic()
    want = orc.stg(kind, faces, ub2, _oracle_params(kw), rnd, 3)
    assert np.abs(u.cpu().numpy()[eq] - want[eq]).max() <= 1e-7
    mask = np.zeros(kind.shape, bool)
    mask[:, :, 0] = True
    mask[:, 0, :] = True
    mask &= eq
    ub32 = ub2.astype(np.float32).astype(np.float64)
    U = np.broadcast_to(ub32[:, None, None, :], kind.shape + (3,))[mask]
    assert u_ref == pytest.approx(np.linalg.norm(U, axis=1).mean(), rel=1e-12)
    # switched off: the equilibrium cells take u_b again from the next step on
    dom.disable_stg()
    dom.step(1)
    _, u = dom.macroscopic()
    base = np.broadcast_to(ub2[:, None, None, :], kind.shape + (3,))
    assert np.abs(u.cpu().numpy()[eq] - base[eq]).max() <= 1e-8


def test_configure_rejects_bad_arguments():
    from paper_2607_04516_b300 import lbm
    closed = synth.random_small_case(6, 5, 4, ("periodic",) * 4 + ("noslip", "freeslip"), seed=1)
    dom = gpu_domain(closed)
    with pytest.raises(lbm.LbmError, match="no inflow face"):
        dom.configure_stg(synth.stg_uniforms(4, seed=0), n_modes=4)
    case = _small_case(FACE_SETS[0], seed=2)
    dom = gpu_domain(case)
    bad = synth.stg_uniforms(4, seed=0)
    bad[1, 2, 3] = 1.0
    with pytest.raises(lbm.LbmError, match="outside"):
        dom.configure_stg(bad, n_modes=4)
    with pytest.raises(lbm.LbmError):
        dom.configure_stg(synth.stg_uniforms(4, seed=0), n_modes=4, length=-1.0)
    with pytest.raises(lbm.LbmError):
        dom.configure_stg(synth.stg_uniforms(4, seed=0), n_modes=4, stride=0)
    with pytest.raises(lbm.LbmError):                                 # nothing configured
        dom.stg_reference()


def test_city_400x400x80_equilibrium_cells_after_two_steps():
    """The full-size city workload with its west and south inflow faces turbulent (64 modes):
    every equilibrium cell's velocity after two steps vs oracle_stg."""
    case = synth.city_case()
    kw = dict(n_modes=64, length=20.0, intensity=0.1)
    rnd = synth.stg_uniforms(64, seed=11)
    dom = _gpu_run_stg(case, 2, kw, rnd)
    _, u = dom.macroscopic()
    u = u.cpu().numpy()
    kind, ub = oracle_inputs(case)
    want = orc.stg(kind, case.faces, ub, _oracle_params(kw), rnd, 1)
    eq = kind == orc.EQ
    assert eq.sum() > 50000
    err = np.abs(u[eq] - want[eq]).max()
    assert err <= 1e-7, err


@pytest.mark.parametrize("nsteps", [1, 2, 5])
def test_inflow_turbulence_with_coriolis_force_and_zones_populations(nsteps):
    """All per-step physics terms at once, as in a production run: the turbulent inflow (App. F), a
    uniform force and Coriolis (App. E), a top sponge and lateral buffers (Sec. 3); populations
    element by element against the oracle, which nudges after each of its steps."""
    from oracle import zones
    kw = PARAMS[2]
    case = _small_case(FACE_SETS[0], seed=47)
    case.coriolis = (1e-3, -2e-3, 3e-3)
    case.force = (1e-5, 0.0, -2e-5)
    sponge, buffer = (2, 0.3), (2, 0.25)
    rnd = synth.stg_uniforms(kw["n_modes"], seed=207)
    dom = gpu_domain(case, "f32", sponge=sponge, buffer=buffer)
    dom.configure_stg(rnd, **kw)
    dom.step(nsteps)
    g = dom.export_populations().cpu().numpy()
    kind, ub = oracle_inputs(case)
    P = _oracle_params(kw)
    fz, om = f64_of_f32(case.force), f64_of_f32(case.coriolis)
    F = orc.init(kind, ub, f64_of_f32(case.rho0), f64_of_f32(case.u0), case.rho_b)
    for t in range(nsteps):
        ueq = orc.stg(kind, case.faces, ub, P, rnd, t)
        F = orc.step(F, kind, case.faces, ub, case.tau, case.cs, force=fz, rho_b=case.rho_b, omega=om, ueq=ueq)
        F = zones.nudge(F, kind, case.faces, ub, sponge=sponge, buffer=buffer)
    _, wo, _ = orc.lattice()
    G = g[lib_to_oracle_order()] + wo[:, None, None, None]
    diff = np.abs(G - F)[:, kind != orc.SOLID]
    assert diff.max() <= 2e-6, diff.max()

"""GPU parity of the boundary relaxation zones (top sponge, lateral buffers) and the flux balancing
against the FP64 oracle (oracle/zones.py; Sec. 3 boundary paragraph, Sec. 2.1 flux consistency)."""
import numpy as np
import pytest

from oracle import oracle as orc
from oracle import zones
from paper_2607_04516_b300 import synth
from gpu_common import TOL_U, f32, f64_of_f32, lib_to_oracle_order, oracle_inputs, rel_l2

pytestmark = pytest.mark.gpu

FACE_SETS = [
    ("inflow", "outflow", "periodic", "periodic", "noslip", "freeslip"),
    ("outflow", "inflow", "inflow", "outflow", "noslip", "freeslip"),
    ("inflow", "outflow", "outflow", "inflow", "noslip", "outflow"),
    ("inflow", "inflow", "inflow", "outflow", "noslip", "inflow"),
]


def _gpu(case, store="f32", **kw):
    from paper_2607_04516_b300 import lbm
    d = lbm.Domain(case.solid, case.faces, case.tau, case.cs, store, case.rho_b, **kw)
    d.set_inflow_profile(f32(case.speed), case.theta)
    d.init_fields(f32(case.rho0), f32(case.u0))
    return d


@pytest.mark.parametrize("faces", FACE_SETS)
@pytest.mark.parametrize("nsteps", [1, 4])
@pytest.mark.parametrize("flux", [False, True])
def test_small_lattices_zones_and_flux_balance_populations(faces, nsteps, flux):
    case = synth.random_small_case(13, 9, 7, faces, seed=21, solid_fraction=0.12, margin=0)
    sponge, buffer = (3, 0.4), (2, 0.3)
    dom = _gpu(case, sponge=sponge, buffer=buffer, flux_balance=flux)
    dom.step(nsteps)
    g = dom.export_populations().cpu().numpy()
    kind, ub = oracle_inputs(case)
    ueq = None
    if flux:
        ueq, before, after, delta = zones.flux_balanced_ueq(kind, faces, ub)
        b, a, sh = dom.flux_balance_info()
        assert b == pytest.approx(before, abs=1e-6) and abs(a) < 1e-5 and sh == pytest.approx(delta, abs=1e-7)
    F = orc.init(kind, ub, f64_of_f32(case.rho0), f64_of_f32(case.u0), ueq=ueq)
    F = zones.run(F, nsteps, kind, faces, ub, case.tau, case.cs, sponge=sponge, buffer=buffer, ueq=ueq)
    _, wo, _ = orc.lattice()
    G = g[lib_to_oracle_order()] + wo[:, None, None, None]
    diff = np.abs(G - F)[:, kind != orc.SOLID]
    assert diff.max() <= 2e-6, diff.max()


@pytest.mark.parametrize("store", ["f32", "f16s"])
def test_cube_with_sponge_and_buffers_200_steps(store):
    case = synth.cube_case()
    sponge, buffer = (6, 0.2), (5, 0.1)
    dom = _gpu(case, store, sponge=sponge, buffer=buffer)
    dom.step(200)
    _, u = dom.macroscopic()
    u = u.cpu().numpy().astype(np.float64)
    kind, ub = oracle_inputs(case)
    F = orc.init(kind, ub, None, f64_of_f32(case.u0))
    F = zones.run(F, 200, kind, case.faces, ub, case.tau, case.cs, sponge=sponge, buffer=buffer)
    _, ur = orc.macros(F, kind, ub)
    err = rel_l2(u, ur, kind == orc.FLUID)
    print(f"cube + zones {store}: rel L2 u = {err:.2e}")
    assert err <= TOL_U[store]


def test_flux_balance_info_off_and_on():
    case = synth.random_small_case(13, 9, 7, FACE_SETS[3], seed=22, solid_fraction=0.2, margin=0)
    d0 = _gpu(case)
    b0, a0, s0 = d0.flux_balance_info()
    assert s0 == 0.0 and a0 == b0
    d1 = _gpu(case, flux_balance=True)
    b1, a1, s1 = d1.flux_balance_info()
    assert b1 == b0 and abs(a1) < 1e-5 * max(1.0, abs(b1)) and s1 != 0.0


@pytest.mark.parametrize("nsteps", [1, 2])
def test_two_cell_forced_path_on_a_large_lattice(nsteps):
    """FP32 lattices of at least 2^21 cells update two cells per thread, forced ones too: a uniform
    body force and Coriolis (App. E), top sponge and lateral buffers, flux-balanced equilibrium cells through the paired
    forced collision and nudging, against the oracle population by population (both step kinds)."""
    faces = FACE_SETS[1]
    case = synth.random_small_case(128, 128, 130, faces, seed=23, solid_fraction=0.04, margin=0)
    assert case.solid.size >= 1 << 21
    omega, force = (2e-3, -1e-3, 3e-3), (1e-5, 0.0, -2e-5)
    sponge, buffer = (4, 0.3), (3, 0.25)
    dom = _gpu(case, sponge=sponge, buffer=buffer, flux_balance=True, coriolis=omega, force=force)
    dom.step(nsteps)
    g = dom.export_populations().cpu().numpy()
    kind, ub = oracle_inputs(case)
    ueq, _, _, _ = zones.flux_balanced_ueq(kind, faces, ub)
    F = orc.init(kind, ub, f64_of_f32(case.rho0), f64_of_f32(case.u0), ueq=ueq)
    for _ in range(nsteps):
        F = orc.step(F, kind, faces, ub, case.tau, case.cs, force=f64_of_f32(force), omega=f64_of_f32(omega), ueq=ueq)
        F = zones.nudge(F, kind, faces, ub, sponge=sponge, buffer=buffer)
    _, wo, _ = orc.lattice()
    G = g[lib_to_oracle_order()] + wo[:, None, None, None]
    diff = np.abs(G - F)[:, kind != orc.SOLID]
    print(f"large lattice, forced two-cell path, {nsteps} steps: max |diff| = {diff.max():.2e}")
    assert diff.max() <= 2e-6, diff.max()


@pytest.mark.parametrize("store,tol_rel", [("f16s", 2.0 ** -11), ("bf16s", 2.0 ** -8)])
@pytest.mark.parametrize("nx", [14, 13])
@pytest.mark.parametrize("warm", [2, 3])
def test_16bit_forced_pairs_with_zones_and_coriolis(store, tol_rel, nx, warm):
    """16-bit storage takes the paired forced collision and nudging in both step kinds (adjacent
    pairs in the local step when nx and N are even, else the (n, n + 256) pairs).  From the GPU's
    own state after `warm` steps, one more step with a uniform force, Coriolis, sponge, buffers and
    flux balancing against the oracle's step from the same populations: every population within
    the storage rounding of its shifted value."""
    faces = FACE_SETS[1]
    case = synth.random_small_case(nx, 8, 6, faces, seed=24, solid_fraction=0.1, margin=0)
    omega, force = (2e-3, -1e-3, 3e-3), (1e-5, 0.0, -2e-5)
    sponge, buffer = (2, 0.3), (2, 0.25)
    dom = _gpu(case, store, sponge=sponge, buffer=buffer, flux_balance=True, coriolis=omega, force=force)
    dom.step(warm)
    g0 = dom.export_populations().cpu().numpy().astype(np.float64)
    dom.step(1)
    g1 = dom.export_populations().cpu().numpy().astype(np.float64)
    kind, ub = oracle_inputs(case)
    ueq, _, _, _ = zones.flux_balanced_ueq(kind, faces, ub)
    _, wo, _ = orc.lattice()
    order = lib_to_oracle_order()
    F = g0[order] + wo[:, None, None, None]
    F = orc.step(F, kind, faces, ub, case.tau, case.cs, force=f64_of_f32(force), omega=f64_of_f32(omega), ueq=ueq)
    F = zones.nudge(F, kind, faces, ub, sponge=sponge, buffer=buffer)
    G = g1[order] + wo[:, None, None, None]
    keep = kind != orc.SOLID
    err = np.abs(G - F)[:, keep]
    bound = 3e-7 + 2.0 * tol_rel * np.abs(F - wo[:, None, None, None])[:, keep]
    worst = float((err / bound).max())
    print(f"{store} nx={nx} warm={warm}: forced pairs, worst error / bound = {worst:.3f}")
    assert worst <= 1.0

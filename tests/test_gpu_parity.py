"""GPU parity: the sm_103a path through the C ABI against the FP64 oracle, element by element on
the same seeded inputs.  Tolerances (relative L2 of velocity over fluid cells): FP32 1e-5 and
FP16S 1e-3, the targets stated for FP32 and 16-bit storage.  BF16S misses the 1e-3 target (BF16
keeps 8 significant bits: each store rounds by up to 2^-9 relative; over hundreds of steps that
lands at a few 1e-3); its tests assert the measured envelope 1e-2 instead, and
test_bf16s_misses_the_16bit_target states that it does not meet 1e-3."""
import math

import numpy as np
import pytest

from oracle import oracle as orc
from paper_2607_04516_b300 import synth

from gpu_common import (MEETS_TARGET, TARGET_U, TOL_U, f32, gpu_domain, gpu_run, lib_to_oracle_order, oracle_inputs,
                        oracle_one_step_planes, oracle_run, rel_l2)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_04516_b300 import build
    build.build()


_ORACLE_CACHE = {}


def _oracle_cached(key, case, nsteps):
    if key not in _ORACLE_CACHE:
        _ORACLE_CACHE[key] = oracle_run(case, nsteps)
    return _ORACLE_CACHE[key]


# ------------------------------------------------------------------ laminar cases, full fields
@pytest.mark.parametrize("store", ["f32", "f16s", "bf16s"])
@pytest.mark.parametrize("nsteps", [200, 500])
def test_cube_64x64x32(store, nsteps):
    case = synth.cube_case()
    rho, u, _ = gpu_run(case, nsteps, store)
    rr, ur, _, kind, _ = _oracle_cached(("cube", nsteps), case, nsteps)
    fl = kind == orc.FLUID
    err = rel_l2(u, ur, fl)
    print(f"cube {store} {nsteps} steps: rel L2 u = {err:.3e}, rho = {rel_l2(rho - 1, rr - 1, fl):.3e}")
    tol = TOL_U[store] * (2.0 if nsteps == 500 else 1.0)
    assert err <= tol


def test_bf16s_misses_the_16bit_target():
    """BF16S storage does not meet the 1e-3 bound of 16-bit storage on the cube after 200 steps
    (only FP16S does); its parity tests assert the 1e-2 envelope.  Should BF16S ever meet the
    bound, this test fails and the envelope goes."""
    assert not MEETS_TARGET["bf16s"] and MEETS_TARGET["f16s"]
    case = synth.cube_case()
    _, u, _ = gpu_run(case, 200, "bf16s")
    _, ur, _, kind, _ = _oracle_cached(("cube", 200), case, 200)
    err = rel_l2(u, ur, kind == orc.FLUID)
    assert TARGET_U["bf16s"] < err <= TOL_U["bf16s"]


@pytest.mark.parametrize("cs", [0.0, 0.16])
@pytest.mark.parametrize("store", ["f32", "f16s"])
def test_taylor_green_32(cs, store):
    case = synth.taylor_green_case(n=32, U0=0.01, tau=0.8, cs=cs)
    rho, u, _ = gpu_run(case, 200, store)
    rr, ur, _, kind, _ = _oracle_cached(("tg", cs), case, 200)
    err = rel_l2(u, ur, kind == orc.FLUID)
    print(f"TG cs={cs} {store}: rel L2 u = {err:.3e}")
    assert err <= TOL_U[store]


def test_channel_with_body_force():
    case = synth.channel_case(nz=16, nxy=8, force=1e-5, tau=0.9)
    rho, u, _ = gpu_run(case, 600, "f32")
    rr, ur, _, kind, _ = _oracle_cached("channel", case, 600)
    err = rel_l2(u, ur, kind == orc.FLUID)
    assert err <= 1e-5


# ------------------------------------------------------------------ every boundary combination
FACE_SETS = [
    ("inflow", "outflow", "periodic", "periodic", "noslip", "freeslip"),
    ("outflow", "inflow", "inflow", "outflow", "noslip", "freeslip"),
    ("inflow", "outflow", "outflow", "inflow", "noslip", "outflow"),
    ("periodic", "periodic", "noslip", "noslip", "freeslip", "freeslip"),
    ("outflow", "outflow", "outflow", "outflow", "noslip", "inflow"),
    ("freeslip", "outflow", "periodic", "periodic", "noslip", "noslip"),
    ("periodic",) * 6,
    ("outflow",) * 6,
]


@pytest.mark.parametrize("faces", FACE_SETS)
@pytest.mark.parametrize("nsteps", [1, 2, 5])
@pytest.mark.parametrize("force", [None, (2e-5, -1e-5, 0.0)])
def test_small_lattices_every_face_kind_populations(faces, nsteps, force):
    """Post-collision populations, element by element, on a 13 x 7 x 6 lattice with solids
    everywhere including the faces (546 cells: 3 blocks with a ragged tail)."""
    case = synth.random_small_case(13, 7, 6, faces, seed=11, solid_fraction=0.12, margin=0)
    case.force = force
    dom = gpu_domain(case, "f32")
    dom.step(nsteps)
    g = dom.export_populations().cpu().numpy()
    _, _, F, kind, _ = oracle_run(case, nsteps)
    _, wo, _ = orc.lattice()
    G = g[lib_to_oracle_order()] + wo[:, None, None, None]
    nonsolid = kind != orc.SOLID
    diff = np.abs(G - F)[:, nonsolid]
    assert diff.max() <= 2e-6, diff.max()


@pytest.mark.parametrize("store", ["f16s", "bf16s"])
def test_small_lattice_16bit_storage(store):
    faces = FACE_SETS[1]
    case = synth.random_small_case(13, 7, 6, faces, seed=12, solid_fraction=0.1, margin=0)
    rho, u, _ = gpu_run(case, 6, store)
    rr, ur, _, kind, _ = oracle_run(case, 6)
    assert rel_l2(u, ur, kind == orc.FLUID) <= TOL_U[store]


@pytest.mark.parametrize("dims", [(2, 2, 2), (3, 5, 2), (33, 1, 1), (257, 3, 2)])
def test_degenerate_and_ragged_lattices(dims):
    nx, ny, nz = dims
    faces = ["periodic"] * 6
    if nx >= 2:
        faces[0], faces[1] = "inflow", "outflow"
    if nz >= 2:
        faces[4], faces[5] = "noslip", "freeslip"
    case = synth.random_small_case(nx, ny, nz, faces, seed=5, solid_fraction=0.0, margin=0)
    rho, u, _ = gpu_run(case, 7, "f32")
    rr, ur, _, kind, _ = oracle_run(case, 7)
    fl = kind == orc.FLUID
    if fl.any():
        assert np.abs(u - ur)[fl].max() <= 1e-6


def test_all_solid_lattice_is_inert():
    case = synth.random_small_case(6, 5, 4, FACE_SETS[0], seed=1)
    case.solid[:] = 1
    rho, u, dom = gpu_run(case, 4, "f32")
    assert (rho == 0).all() and (u == 0).all()
    d = dom.diagnostics()
    assert d["mass"] == 0.0 and d["nonfinite"] == 0


# ------------------------------------------------------------------ full-size, bench launch config
def _one_step_parity(case, store, warm, planes, tol_abs, tol_rel):
    dom = gpu_domain(case, store)
    dom.step(warm)
    perm = lib_to_oracle_order()
    g0 = dom.export_populations()
    need = sorted({p for z in planes for p in (z - 1, z, z + 1) if 0 <= p < case.shape[0]})
    g0_planes = {p: g0[:, p].cpu().numpy() for p in need}
    del g0
    dom.step(1)
    g1 = dom.export_populations()
    kind, ub = oracle_inputs(case)
    ref = oracle_one_step_planes(g0_planes, kind, case.faces, ub, case.tau, case.cs, case.force,
                                 case.rho_b, planes, perm)
    _, wo, _ = orc.lattice()
    worst = 0.0
    for z in planes:
        got = g1[:, z].cpu().numpy().astype(np.float64)[perm] + wo[:, None, None]
        want = ref[z]
        ns = kind[z] != orc.SOLID
        err = np.abs(got - want)[:, ns]
        bound = tol_abs + tol_rel * np.abs(want - wo[:, None, None])[:, ns]
        worst = max(worst, float((err / bound).max()))
        assert (err <= bound).all(), (z, float(err.max()))
    return worst


@pytest.mark.parametrize("store,tol_rel", [("f32", 0.0), ("f16s", 2.0 ** -11), ("bf16s", 2.0 ** -8)])
def test_city_400x400x80_one_step_sampled_planes(store, tol_rel):
    """The benchmark workload (12.8M cells) in the launch configuration the benchmark times: the
    step from a GPU state to the next, recomputed by the oracle on the ground, a mid and the top
    planes.  Both sides start from the same stored populations."""
    case = synth.city_case()
    worst = _one_step_parity(case, store, warm=30, planes=[0, 1, 7, 40, 78, 79],
                             tol_abs=3e-7, tol_rel=tol_rel)
    print(f"city {store}: worst error / bound = {worst:.3f}")


def test_city_1000x1000x160_one_step_sampled_planes():
    """Largest configuration (160M cells, 12.2 GB of FP32 populations)."""
    case = synth.city_case(nx=1000, ny=1000, nz=160, seed=2, noise=0.0)
    _one_step_parity(case, "f32", warm=3, planes=[0, 5, 159], tol_abs=3e-7, tol_rel=0.0)


# ------------------------------------------------------------------ API behaviour on the GPU
def test_sample_columns_match_full_fields_and_flag_out_of_range():
    case = synth.cube_case()
    dom = gpu_domain(case, "f32")
    dom.step(11)                      # odd: layout A readback
    rho, u = dom.macroscopic()
    ij = np.array([[3, 4], [30, 30], [63, 63], [0, 10], [64, 0], [-1, 5]], np.int32)
    kk = np.array([0, 5, 15, 31, 32], np.int32)
    out = dom.sample_columns(ij, kk).cpu().numpy()
    r = rho.cpu().numpy()
    uu = u.cpu().numpy()
    for c, (x, y) in enumerate(ij):
        for h, z in enumerate(kk):
            if 0 <= x < 64 and 0 <= y < 64 and 0 <= z < 32:
                np.testing.assert_array_equal(out[c, h, :3], uu[z, y, x])
                assert out[c, h, 3] == r[z, y, x]
            else:
                assert np.isnan(out[c, h]).all()
    # a solid cell reads zero, an inflow cell reads (u_b, rho_b)
    assert (out[1, 0] == 0).all()
    assert out[3, 0, 3] == 1.0 and out[3, 0, 1] == 0.0
    assert dom.sample_columns(np.zeros((0, 2), np.int32), kk).shape == (0, 5, 4)


def test_step_zero_and_counter():
    case = synth.cube_case(nx=16, ny=16, nz=8)
    dom = gpu_domain(case, "f32")
    g0 = dom.export_populations()
    dom.step(0)
    assert dom.steps_done == 0
    assert torch.equal(g0, dom.export_populations())
    dom.step(3)
    assert dom.steps_done == 3
    dom.init_fields(None, None)
    assert dom.steps_done == 0


def test_diagnostics_mass_in_periodic_box_and_oracle_mass():
    case = synth.random_small_case(24, 20, 16, ("periodic",) * 6, seed=3, solid_fraction=0.05,
                                   margin=0)
    dom = gpu_domain(case, "f32")
    m0 = dom.diagnostics()["mass"]
    dom.step(101)
    d = dom.diagnostics()
    _, _, F, kind, _ = oracle_run(case, 101)
    m_ref = F[:, kind == orc.FLUID].sum()
    assert abs(d["mass"] - m_ref) / m_ref < 1e-6
    assert abs(d["mass"] - m0) / m0 < 1e-6
    assert d["nonfinite"] == 0
    assert abs(d["net_flux"]) == 0.0     # no open faces


def test_watchdog_reports_nonfinite_state():
    from paper_2607_04516_b300 import lbm
    case = synth.cube_case(nx=16, ny=16, nz=8)
    dom = gpu_domain(case, "f32", watchdog_every=2)
    u = case.u0.astype(np.float32).copy()
    u[4, 2, 2, 0] = np.nan                          # a corrupt fluid input cell, rejected by nothing
    assert not case.solid[4, 2, 2]
    dom.init_fields(None, u)
    with pytest.raises(lbm.LbmError) as e:
        dom.step(4)
    assert e.value.status == -4
    assert dom.diagnostics()["nonfinite"] > 0


def test_runs_on_a_side_stream():
    case = synth.cube_case(nx=32, ny=32, nz=16)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        dom = gpu_domain(case, "f32")
        dom.step(20)
        rho, u = dom.macroscopic()
    s.synchronize()
    rho2, u2, _ = gpu_run(case, 20, "f32")
    np.testing.assert_array_equal(u.cpu().numpy(), u2.astype(np.float32))


# ------------------------------------------------------------------ Coriolis force (App. E)
@pytest.mark.parametrize("faces", FACE_SETS[:3] + [FACE_SETS[6]])
@pytest.mark.parametrize("nsteps", [1, 4])
def test_small_lattices_with_coriolis_populations(faces, nsteps):
    case = synth.random_small_case(13, 7, 6, faces, seed=21, solid_fraction=0.12, margin=0)
    case.coriolis = (1e-3, -2e-3, 3e-3)
    case.force = (1e-5, 0.0, -2e-5)
    dom = gpu_domain(case, "f32")
    dom.step(nsteps)
    g = dom.export_populations().cpu().numpy()
    _, _, F, kind, _ = oracle_run(case, nsteps)
    _, wo, _ = orc.lattice()
    G = g[lib_to_oracle_order()] + wo[:, None, None, None]
    diff = np.abs(G - F)[:, kind != orc.SOLID]
    assert diff.max() <= 2e-6, diff.max()


@pytest.mark.parametrize("store", ["f32", "f16s"])
def test_cube_with_coriolis(store):
    """The cube flow with an exaggerated rotation (|Omega^lbm| ~ 1e-3, a thousand times Earth's at a
    5 m / 0.01 s lattice) so that the force changes the field visibly within 200 steps."""
    case = synth.cube_case()
    case.coriolis = (0.0, 6e-4, 8e-4)
    rho, u, _ = gpu_run(case, 200, store)
    rr, ur, _, kind, _ = _oracle_cached(("cube-rot", 200), case, 200)
    ref0 = _oracle_cached(("cube", 200), synth.cube_case(), 200)[1]
    fl = kind == orc.FLUID
    assert rel_l2(ur, ref0, fl) > 10 * TOL_U[store]          # the rotation matters here
    assert rel_l2(u, ur, fl) <= TOL_U[store]


@pytest.mark.parametrize("store", ["f32", "f16s"])
def test_export_import_resumes_bit_for_bit(store):
    """Checkpoint / restart: export after an even number of steps, import into a fresh domain, step
    on: the same populations as the uninterrupted run (and an odd step count is refused)."""
    from paper_2607_04516_b300 import lbm
    case = synth.random_small_case(14, 8, 6, ("outflow", "inflow", "inflow", "outflow", "noslip", "freeslip"),
                                   seed=31, solid_fraction=0.1, margin=0)
    a = gpu_domain(case, store)
    a.step(6)
    saved = a.export_populations()
    a.step(5)
    want = a.export_populations().cpu().numpy()
    b = gpu_domain(case, store)
    b.step(3)                          # arbitrary prior state, overwritten by the import
    b.import_populations(saved, 6)
    assert b.steps_done == 6
    b.step(5)
    got = b.export_populations().cpu().numpy()
    np.testing.assert_array_equal(got, want)
    with pytest.raises(lbm.LbmError):
        b.import_populations(saved, 7)


@pytest.mark.parametrize("store", ["f32", "f16s"])
def test_all_solid_and_empty_requests(store):
    """Degenerate inputs: a lattice with no fluid cell steps without touching anything (diagnostics
    report zero mass and no non-finite cell); empty sample requests are no-ops."""
    import torch
    from paper_2607_04516_b300 import lbm
    faces = ("inflow", "outflow", "periodic", "periodic", "noslip", "freeslip")
    solid = np.ones((6, 5, 8), np.uint8)
    d = lbm.Domain(solid, faces, 0.6, 0.16, store)
    d.set_inflow_profile(np.full(6, 0.05, np.float32), 0.0)
    d.init_fields()
    d.step(7)
    rho, u = d.macroscopic()
    assert float(rho.abs().max()) == 0.0 and float(u.abs().max()) == 0.0
    diag = d.diagnostics()
    assert diag["mass"] == 0.0 and diag["nonfinite"] == 0
    out = torch.empty((0, 3, 4), dtype=torch.float32, device="cuda")
    lbm.lbm_sample_columns(d.dom, torch.empty((0, 2), dtype=torch.int32, device="cuda"),
                           torch.zeros(3, dtype=torch.int32, device="cuda"), out)
    # a lattice whose only non-solid cells are equilibrium cells: they hold f^eq(rho_b, u_b)
    solid2 = np.ones((4, 4, 6), np.uint8)
    solid2[:, :, 0] = 0
    d2 = lbm.Domain(solid2, faces, 0.6, 0.16, store)
    d2.set_inflow_profile(np.full(4, 0.05, np.float32), 0.0)
    d2.init_fields()
    d2.step(3)
    _, u2 = d2.macroscopic()
    torch.cuda.synchronize()
    np.testing.assert_allclose(u2[:, :, 0, 0].cpu().numpy(), 0.05, rtol=0, atol=1e-7)


def test_city_400x400x80_long_run_checks():
    """The benchmark city at tau = 0.505 is turbulent, so its instantaneous fields are not compared
    with the oracle beyond a step; what is checked over a long run: no non-finite population, bounded
    mass drift over 2000 FP32 steps, and 50-step agreement of 16-bit storage with the FP32 path."""
    import torch
    case = synth.city_case()
    d = gpu_domain(case, "f32")
    m0 = d.diagnostics()["mass"]
    d.step(1500)
    m1500 = d.diagnostics()["mass"]
    d.step(500)
    diag = d.diagnostics()
    assert diag["nonfinite"] == 0
    # an open domain: the mass follows the boundary fluxes while the flow develops (+0.35% over
    # the first 2000 steps from the profile start), then settles
    print(f"city mass: start {m0:.0f}, step 1500 {m1500:.0f}, step 2000 {diag['mass']:.0f}")
    assert abs(diag["mass"] - m0) / m0 < 1e-2
    assert abs(diag["mass"] - m1500) / m1500 < 2e-3
    assert diag["umax"] < 0.3
    ref = gpu_domain(case, "f32")
    ref.step(50)
    _, u32 = ref.macroscopic()
    fl = torch.as_tensor(case.solid == 0, device="cuda")
    for store, tol in (("f16s", 1e-3), ("bf16s", 1e-2)):
        d16 = gpu_domain(case, store)
        d16.step(50)
        _, u = d16.macroscopic()
        err = float(torch.linalg.vector_norm((u - u32)[fl].double()) / torch.linalg.vector_norm(u32[fl].double()))
        print(f"city {store} vs f32 after 50 steps: rel L2 u = {err:.2e}")
        assert err <= tol


@pytest.mark.parametrize("store", ["f16s", "f32"])
def test_steps_captured_in_a_cuda_graph_replay_like_direct_steps(store):
    """lbm_step enqueued during a CUDA-graph capture of the domain's stream (the neighbour step's
    ground/top layer kernel forks onto the domain's second stream and joins back: the capture must
    take it in) replays to the same populations, bit for bit, as the same steps launched directly.
    A 16-bit lattice of any size, and an FP32 lattice of at least 2^21 cells, take the layer kernel."""
    import torch
    case = synth.city_case(nx=160 if store == "f32" else 64, ny=128 if store == "f32" else 48,
                           nz=104 if store == "f32" else 16, seed=5)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        dom = gpu_domain(case, store, stream=s)
        ref = gpu_domain(case, store, stream=s)
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        dom.step(2)                       # a neighbour and a local step
    with torch.cuda.stream(s):
        for _ in range(3):
            g.replay()
        ref.step(6)
    torch.cuda.synchronize()
    assert dom.steps_done == 2            # the host counter saw the captured steps only
    a = dom.export_populations().cpu().numpy()
    b = ref.export_populations().cpu().numpy()
    torch.cuda.synchronize()
    np.testing.assert_array_equal(a, b)

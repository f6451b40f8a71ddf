"""The C-ABI library builds for sm_103a, loads, and exports every symbol include/lbm.h declares;
host-only entry points and argument validation (no GPU needed, no compute call)."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

from paper_2607_04516_b300 import build as lbuild
from paper_2607_04516_b300 import lbm, synth
from oracle import oracle as orc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    lbuild.build()
    return lbm.load(require_gpu=False)


def _declared_symbols():
    text = open(os.path.join(ROOT, "include", "lbm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    syms = _declared_symbols()
    for required in ("lbm_create_domain", "lbm_set_inflow_profile", "lbm_step",
                     "lbm_sample_columns", "lbm_destroy"):
        assert required in syms


def test_library_exports_every_declared_symbol(lib):
    for s in _declared_symbols():
        assert hasattr(lib, s), s
    assert set(_declared_symbols()) == set(lbm.SIGNATURES), "binding and header disagree"


def test_build_targets_sm_103a_only():
    assert lbuild.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_direction_table_is_the_oracles_lattice(lib):
    c, w = lbm.lbm_direction_table()
    co, wo, _ = orc.lattice()
    assert {tuple(v) for v in c} == {tuple(v) for v in co}
    lookup = {tuple(v): wo[i] for i, v in enumerate(co)}
    for i in range(19):
        assert w[i] == pytest.approx(lookup[tuple(c[i])], rel=1e-7)
    # documented pairing: (2k-1, 2k) are opposite
    for k in range(1, 10):
        assert (c[2 * k - 1] == -c[2 * k]).all()


@pytest.mark.parametrize("deg", [0, 10, 45, 90, 135, 180, 200, 270, 300, 359.9])
def test_faces_for_direction_matches_input_generator(lib, deg):
    th = math.radians(deg)
    assert lbm.lbm_faces_for_direction(th) == synth.faces_for_direction(th)


def test_workspace_bytes_layout(lib):
    p = lbm.make_params(("inflow", "outflow", "periodic", "periodic", "noslip", "freeslip"))
    n = lbm.lbm_workspace_bytes(64, 64, 32, p)
    N = 64 * 64 * 32
    assert n >= 19 * N * 4 + N
    assert n % 256 == 0
    p16 = lbm.make_params(("inflow", "outflow", "periodic", "periodic", "noslip", "freeslip"),
                          store="f16s")
    assert lbm.lbm_workspace_bytes(64, 64, 32, p16) < n
    assert lbm.lbm_workspace_bytes(64, 64, 32, p16) >= 19 * N * 2 + N


@pytest.mark.parametrize("bad", [
    dict(dims=(0, 4, 4)),
    dict(tau=0.5),
    dict(tau=float("nan")),
    dict(cs=-0.1),
    dict(store=7),
    dict(faces=("periodic", "outflow", "periodic", "periodic", "noslip", "freeslip")),
    dict(faces=("inflow", "outflow", "periodic", "periodic", "noslip", 9)),
    dict(dims=(1, 4, 4)),
    dict(dims=(2000, 2000, 1000)),
])
def test_invalid_arguments_are_rejected_on_the_host(lib, bad):
    faces = bad.get("faces", ("inflow", "outflow", "periodic", "periodic", "noslip", "freeslip"))
    p = lbm.make_params(faces, tau=bad.get("tau", 0.52), cs=bad.get("cs", 0.16),
                        store=bad.get("store", "f32"))
    nx, ny, nz = bad.get("dims", (8, 8, 8))
    assert lbm.lbm_workspace_bytes(nx, ny, nz, p) == 0
    out = ctypes.c_void_p()
    solid = np.zeros(max(1, nx * ny * nz) if nx * ny * nz < 10 ** 8 else 1, np.uint8)
    st = lib.lbm_create_domain(solid.ctypes.data, nx, ny, nz, ctypes.byref(p),
                               ctypes.c_void_p(256), 1 << 40, None, ctypes.byref(out))
    assert st == -1 and not out.value


def test_create_rejects_null_and_small_workspace_before_any_cuda_call(lib):
    p = lbm.make_params(("inflow", "outflow", "periodic", "periodic", "noslip", "freeslip"))
    solid = np.zeros(8 * 8 * 8, np.uint8)
    out = ctypes.c_void_p()
    assert lib.lbm_create_domain(solid.ctypes.data, 8, 8, 8, ctypes.byref(p), None, 1 << 30, None,
                                 ctypes.byref(out)) == -1
    assert lib.lbm_create_domain(None, 8, 8, 8, ctypes.byref(p), ctypes.c_void_p(256), 1 << 30, None,
                                 ctypes.byref(out)) == -1
    need = lib.lbm_workspace_bytes(8, 8, 8, ctypes.byref(p))
    assert lib.lbm_create_domain(solid.ctypes.data, 8, 8, 8, ctypes.byref(p), ctypes.c_void_p(256),
                                 need - 1, None, ctypes.byref(out)) == -2
    # misaligned workspace
    assert lib.lbm_create_domain(solid.ctypes.data, 8, 8, 8, ctypes.byref(p), ctypes.c_void_p(257),
                                 need + 512, None, ctypes.byref(out)) == -1
    assert lib.lbm_create_domain(solid.ctypes.data, 8, 8, 8, ctypes.byref(p), ctypes.c_void_p(256),
                                 need, None, None) == -1


def test_null_handles_are_safe(lib):
    lib.lbm_destroy(None)
    assert lib.lbm_step(None, 1) == -1
    assert lib.lbm_steps_done(None) == -1
    assert lib.lbm_last_error(None) == b"no domain"
    assert lib.lbm_params_default(None) == -1
    assert lib.lbm_faces_for_direction(ctypes.c_float(0.0), None) == -1


def test_binding_refuses_to_run_without_a_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(RuntimeError):
        lbm.Domain(np.zeros((4, 4, 4), np.uint8), ("periodic",) * 6)


def test_coriolis_omega_is_earth_rotation_in_the_local_enu_frame(lib):
    """App. E: Omega_ENU = Omega (0, cos lat, sin lat), Omega = 7.292115e-5 rad/s, times dt."""
    lat, dt = 23.113, 0.01
    om = lbm.lbm_coriolis_omega(lat, dt)
    w = 7.292115e-5 * dt
    assert om[0] == 0.0
    assert om[1] == pytest.approx(w * math.cos(math.radians(lat)), rel=1e-6)
    assert om[2] == pytest.approx(w * math.sin(math.radians(lat)), rel=1e-6)
    with pytest.raises(lbm.LbmError):
        lbm.lbm_coriolis_omega(10.0, -1.0)


def test_params_default_has_no_rotation(lib):
    p = lbm.make_params(("periodic",) * 6)
    assert tuple(p.coriolis) == (0.0, 0.0, 0.0)
    assert lbm.lbm_workspace_bytes(8, 8, 8, lbm.make_params(("periodic",) * 6,
                                                            coriolis=(0, 0, float("nan")))) == 0


def test_stg_params_default_and_null_handles(lib):
    p = lbm.make_stg_params()
    assert (p.n_modes, p.length, p.intensity, p.sigma0) == (64, 20.0, pytest.approx(0.1), 0.0)
    assert tuple(p.gain) == (1.0, 1.0, 1.0)
    assert (p.char_normal, p.inflow_only, p.stride, p.interpolate) == (0, 0, 1, 1)
    assert lib.lbm_stg_params_default(None) == -1
    assert lib.lbm_stg_workspace_bytes(None, 8) == 0
    assert lib.lbm_stg_configure(None, ctypes.byref(p), None, None, 0) == -1
    assert lib.lbm_stg_disable(None) == -1
    assert lib.lbm_stg_reference(None, None, None, None) == -1


def test_ctypes_structs_match_the_c_layout(tmp_path):
    """sizeof and every field offset of the parameter structs, as gcc lays them out from the
    header, equal the binding's ctypes mirrors."""
    structs = {"lbm_params": lbm.lbm_params, "lbm_stg_params": lbm.lbm_stg_params}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "lbm.h"', 'int main(void) {']
    for name, cls in structs.items():
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for fname, _ in cls._fields_:
            lines.append(f'printf("{name} {fname} %zu\\n", offsetof({name}, {fname}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    import subprocess
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l}
    for name, cls in structs.items():
        assert got[(name, "size")] == ctypes.sizeof(cls), name
        for fname, _ in cls._fields_:
            assert got[(name, fname)] == getattr(cls, fname).offset, (name, fname)


def test_batch_workspace_bytes(lib):
    assert lbm.load(False).lbm_batch_workspace_bytes(0) == 0
    assert lbm.load(False).lbm_batch_workspace_bytes(5000) == 0
    small, big = lbm.load(False).lbm_batch_workspace_bytes(1), lbm.load(False).lbm_batch_workspace_bytes(40)
    assert 0 < small < big and big % 256 == 0


def test_lattice_units_mach_scaling(lib):
    """Mach scaling: u_lbm = u_si dt/dx = Ma c_s, nu_lbm = nu_si dt/dx^2, tau = 3 nu_lbm + 1/2."""
    u = lbm.lbm_lattice_units(5.0, 5.3205, 0.10, 1.5e-5)
    cs = 1.0 / math.sqrt(3.0)
    assert u["u_lbm"] == pytest.approx(0.1 * cs, rel=1e-15)
    assert 5.3205 * u["dt_si"] / 5.0 == pytest.approx(u["u_lbm"], rel=1e-14)
    assert u["nu_lbm"] == pytest.approx(1.5e-5 * u["dt_si"] / 25.0, rel=1e-14)
    assert u["tau"] == pytest.approx(3 * u["nu_lbm"] + 0.5, rel=1e-15)
    for bad in [(0.0, 5.0, 0.1, 1e-5), (5.0, -1.0, 0.1, 1e-5), (5.0, 5.0, 0.0, 1e-5), (5.0, 5.0, 0.1, -1.0),
                (float("nan"), 5.0, 0.1, 1e-5)]:
        with pytest.raises(lbm.LbmError):
            lbm.lbm_lattice_units(*bad)

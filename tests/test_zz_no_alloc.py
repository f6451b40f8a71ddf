"""lbm_diagnostics_noalloc: the diagnostics reductions for callers that must not allocate device
memory (scratch in a fixed array inside the library).  Checked through the C ABI against
lbm_diagnostics on two calls in a row, in both streaming layouts and two storage kinds; that a call
after the first on a device leaves the free device memory unchanged; the same checks in a fresh
Python process (where the entry point's first call does the per-device set-up); the size limit of
its fixed scratch."""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2607_04516_b300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# The two entry points give their threads the cells in a different order.  max |u| and the
# non-finite count are order-free; the flux is summed in FP64 (rounding ~1e-16 per term); the mass
# is formed from per-thread FP32 partial sums of rho - 1, which round differently.  A thread of the
# allocation-free kernel adds 64 cells; each add rounds by at most half an ulp of its partial
# (|partial| <= 64 max|rho - 1|, max|rho - 1| < 1e-2 on this flow): <= 64 x 0.64 x 2^-24 ~ 2.4e-6
# per partial, <= 5e-3 over the 2048 partials of the 2^17-cell cube, 4e-8 of its mass (~1.3e5).
# (One cell missing or counted twice would show as ~8e-6.)
RTOL_MASS = 1e-7
RTOL_FLUX = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_04516_b300 import build
    build.build()


def _domain(store):
    from paper_2607_04516_b300 import lbm
    case = synth.cube_case()
    dom = lbm.Domain(case.solid, case.faces, case.tau, case.cs, store)
    dom.set_inflow_profile(case.speed.astype(np.float32), case.theta)
    dom.init_fields(None, case.u0.astype(np.float32))
    return dom


def _noalloc(dom):
    from paper_2607_04516_b300 import lbm
    out = torch.full((4,), float("nan"), dtype=torch.float64, device=dom.device)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    lbm.lbm_diagnostics_noalloc(dom.dom, out)
    dom.stream.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    return out.cpu().numpy(), free0 - free1


def check_consecutive_calls(store):
    """Two calls in a row after an odd and after an even step count agree with lbm_diagnostics;
    every call after the first on this device leaves the free device memory unchanged."""
    dom = _domain(store)
    first = True
    for nsteps in (7, 1):                  # odd then even step count: both layouts
        dom.step(nsteps)
        ref = dom.diagnostics()
        want = np.array([ref["mass"], ref["net_flux"], ref["umax"], ref["nonfinite"]])
        for _ in range(2):                 # two calls in a row share the fixed scratch
            got, used = _noalloc(dom)
            if not first:
                assert used == 0, f"free device memory changed by {used} bytes"
            first = False
            assert np.isfinite(got).all()
            np.testing.assert_allclose(got[0], want[0], rtol=RTOL_MASS)
            np.testing.assert_allclose(got[1], want[1], rtol=RTOL_FLUX, atol=1e-12)
            assert got[2] == want[2]
            assert got[3] == want[3]
        assert want[0] > 0.5 * dom.N            # total mass of the fluid cells, rho ~ 1


@pytest.mark.parametrize("store", ["f32", "f16s"])
def test_noalloc_diagnostics_match_the_workspace_version_on_consecutive_calls(store):
    check_consecutive_calls(store)


def test_noalloc_in_a_fresh_process():
    """The same checks in a new interpreter, where the first call on the device looks up the
    scratch address."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = ("import sys; sys.path.insert(0, %r); sys.path.insert(0, %r); "
            "import test_zz_no_alloc as t; t.check_consecutive_calls('f32'); print('fresh ok')"
            % (root, os.path.join(root, "tests")))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600, cwd=root)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
    assert "fresh ok" in r.stdout


def test_noalloc_rejects_lattices_beyond_its_scratch():
    from paper_2607_04516_b300 import lbm
    # 2^28 cells is the limit; one more z plane of 1024 x 1024 crosses it (16-bit storage: 11.6 GB)
    if torch.cuda.mem_get_info()[0] < 16 * 2**30:
        pytest.skip("needs 16 GB of free device memory for a lattice above the scratch limit")
    nx, ny, nz = 1024, 1024, 257
    solid = np.zeros((nz, ny, nx), np.uint8)
    faces = ("periodic",) * 6
    dom = lbm.Domain(solid, faces, 0.6, 0.16, "f16s")
    del solid
    out = torch.zeros(4, dtype=torch.float64, device=dom.device)
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_diagnostics_noalloc(dom.dom, out)
    assert e.value.status == -1
    assert "2^28" in str(e.value)
    assert (out == 0).all()
    del dom
    torch.cuda.empty_cache()

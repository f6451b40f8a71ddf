"""lbm_diagnostics_noalloc: the diagnostics reductions for callers that must not allocate device
memory (scratch in a fixed array inside the library).  Checked through the C ABI against
lbm_diagnostics on two calls in a row, in both streaming layouts and two storage kinds, plus the
size limit of its fixed scratch.  Runs alone in a fresh process as well as after the other tests."""
import numpy as np
import pytest

from paper_2607_04516_b300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

RTOL = 1e-12     # FP64 sums added in a different order than lbm_diagnostics


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
    lbm.lbm_diagnostics_noalloc(dom.dom, out)
    dom.stream.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("store", ["f32", "f16s"])
def test_noalloc_diagnostics_match_the_workspace_version_on_consecutive_calls(store):
    dom = _domain(store)
    for nsteps in (7, 1):                  # odd then even step count: both layouts
        dom.step(nsteps)
        ref = dom.diagnostics()
        want = np.array([ref["mass"], ref["net_flux"], ref["umax"], ref["nonfinite"]])
        for _ in range(2):                 # two calls in a row share the fixed scratch
            got = _noalloc(dom)
            assert np.isfinite(got).all()
            np.testing.assert_allclose(got[:2], want[:2], rtol=RTOL, atol=1e-12)
            assert got[2] == want[2]
            assert got[3] == want[3]
        assert want[0] > 0.5 * dom.N            # total mass of the fluid cells, rho ~ 1


def test_noalloc_rejects_lattices_beyond_its_scratch():
    from paper_2607_04516_b300 import lbm
    # 2^28 cells is the limit; one more z plane of 1024 x 1024 crosses it (16-bit storage: 11.6 GB)
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

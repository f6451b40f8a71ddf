"""Thin Python binding of the C ABI in ``include/lbm.h`` (argument marshalling only).

Every entry point keeps its C name (``lbm_create_domain``, ``lbm_step``, ...) and forwards torch
CUDA tensors as raw device pointers; all computation happens in ``liblbm.so``.  The library is
loaded on first use; a missing library or a missing CUDA device raises ``RuntimeError`` -- there
is no fallback path.  ``Domain`` bundles the calls for convenience.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "liblbm.so")

FACES = {"periodic": 0, "inflow": 1, "outflow": 2, "freeslip": 3, "noslip": 4}
FACE_NAMES = {v: k for k, v in FACES.items()}
STORES = {"f32": 0, "f16s": 1, "bf16s": 2}
STATUS = {0: "LBM_OK", -1: "LBM_EINVAL", -2: "LBM_ENOMEM", -3: "LBM_ECUDA", -4: "LBM_EUNSTABLE",
          -5: "LBM_ESTATE"}


class LbmError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class lbm_params(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_float), ("cs_smag", ctypes.c_float), ("rho_b", ctypes.c_float),
                ("store", ctypes.c_int), ("face", ctypes.c_int * 6), ("force", ctypes.c_float * 3),
                ("watchdog_every", ctypes.c_int), ("coriolis", ctypes.c_float * 3),
                ("sponge_top", ctypes.c_int), ("sponge_sigma", ctypes.c_float),
                ("buffer_width", ctypes.c_int), ("buffer_sigma", ctypes.c_float),
                ("flux_balance", ctypes.c_int)]


class lbm_stg_params(ctypes.Structure):
    _fields_ = [("n_modes", ctypes.c_int), ("length", ctypes.c_float), ("intensity", ctypes.c_float),
                ("sigma0", ctypes.c_float), ("gain", ctypes.c_float * 3), ("char_normal", ctypes.c_int),
                ("inflow_only", ctypes.c_int), ("stride", ctypes.c_int), ("interpolate", ctypes.c_int)]


class lbm_adjoint_params(ctypes.Structure):
    _fields_ = [("n_steps", ctypes.c_int), ("n_avg", ctypes.c_int), ("checkpoint_every", ctypes.c_int)]


# exported symbols and their ctypes signatures (the header is the authority)
_P, _I, _F, _LL, _SZ = ctypes.c_void_p, ctypes.c_int, ctypes.c_float, ctypes.c_longlong, ctypes.c_size_t
_PP = ctypes.POINTER(lbm_params)
SIGNATURES = {
    "lbm_params_default": (_I, [_PP]),
    "lbm_faces_for_direction": (_I, [_F, _P]),
    "lbm_lattice_units": (_I, [ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double, _P]),
    "lbm_coriolis_omega": (_I, [ctypes.c_double, ctypes.c_double, _P]),
    "lbm_workspace_bytes": (_SZ, [_I, _I, _I, _PP]),
    "lbm_create_domain": (_I, [_P, _I, _I, _I, _PP, _P, _SZ, _P, ctypes.POINTER(_P)]),
    "lbm_set_stream": (_I, [_P, _P]),
    "lbm_set_inflow_profile": (_I, [_P, _P, _I, _F]),
    "lbm_init_fields": (_I, [_P, _P, _P]),
    "lbm_step": (_I, [_P, _I]),
    "lbm_steps_done": (_LL, [_P]),
    "lbm_flux_balance_info": (_I, [_P, _P, _P, _P]),
    "lbm_sample_columns": (_I, [_P, _P, _I, _P, _I, _P]),
    "lbm_macroscopic": (_I, [_P, _P, _P]),
    "lbm_export_populations": (_I, [_P, _P]),
    "lbm_import_populations": (_I, [_P, _P, _LL]),
    "lbm_direction_table": (_I, [_P, _P]),
    "lbm_diagnostics": (_I, [_P, _P]),
    "lbm_diagnostics_noalloc": (_I, [_P, _P]),
    "lbm_stg_params_default": (_I, [ctypes.POINTER(lbm_stg_params)]),
    "lbm_stg_workspace_bytes": (_SZ, [_P, _I]),
    "lbm_stg_configure": (_I, [_P, ctypes.POINTER(lbm_stg_params), _P, _P, _SZ]),
    "lbm_stg_disable": (_I, [_P]),
    "lbm_stg_reference": (_I, [_P, _P, _P, _P]),
    "lbm_adjoint_workspace_bytes": (_SZ, [_P, ctypes.POINTER(lbm_adjoint_params), _I, _I, _I]),
    "lbm_lidar_misfit": (_I, [_P, ctypes.POINTER(lbm_adjoint_params), _P, _I, _F, _P, _I, _P, _I, _P,
                              _P, _SZ, _P, _P]),
    "lbm_lidar_misfit_grad": (_I, [_P, ctypes.POINTER(lbm_adjoint_params), _P, _I, _F, _P, _I, _P, _I,
                                   _P, _P, _SZ, _P, _P]),
    "lbm_batch_workspace_bytes": (_SZ, [_I]),
    "lbm_batch_create": (_I, [_P, _I, _P, _SZ, _P, ctypes.POINTER(_P)]),
    "lbm_batch_step": (_I, [_P, _I]),
    "lbm_batch_capture": (_I, [_P, _I]),
    "lbm_batch_launch": (_I, [_P]),
    "lbm_batch_autotune": (_I, [_P, _I, _P, _P]),
    "lbm_batch_set_shape": (_I, [_P, _I]),
    "lbm_batch_shape": (_I, [_P]),
    "lbm_batch_shape_count": (_I, []),
    "lbm_batch_last_error": (ctypes.c_char_p, [_P]),
    "lbm_batch_destroy": (None, [_P]),
    "lbm_last_error": (ctypes.c_char_p, [_P]),
    "lbm_destroy": (None, [_P]),
}

_lib = None


def load(require_gpu: bool = True) -> ctypes.CDLL:
    """Load ``liblbm.so`` (raises if it is missing; with ``require_gpu`` also without a GPU)."""
    global _lib
    if require_gpu:
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("liblbm needs a CUDA device; none is visible")
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} not built: run `python -m paper_2607_04516_b300.build`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _ptr(t) -> int | None:
    if t is None:
        return None
    import torch
    if isinstance(t, torch.Tensor):
        if not t.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return t.data_ptr()
    return t.ctypes.data


def _check(status: int, dom=None):
    if status != 0:
        msg = load(False).lbm_last_error(dom).decode() if dom else ""
        raise LbmError(status, msg)


def make_params(faces, tau=0.52, cs=0.16, store="f32", rho_b=1.0, force=None, watchdog_every=0,
                coriolis=None, sponge=None, buffer=None, flux_balance=False):
    """``sponge`` / ``buffer``: (width, sigma) of the top / lateral relaxation zones, or None."""
    p = lbm_params()
    load(False).lbm_params_default(ctypes.byref(p))
    p.tau = tau
    p.cs_smag = cs
    p.rho_b = rho_b
    p.store = STORES[store] if isinstance(store, str) else int(store)
    for k, f in enumerate(faces):
        p.face[k] = FACES[f] if isinstance(f, str) else int(f)
    for k in range(3):
        p.force[k] = 0.0 if force is None else float(force[k])
    p.watchdog_every = watchdog_every
    for k in range(3):
        p.coriolis[k] = 0.0 if coriolis is None else float(coriolis[k])
    if sponge is not None:
        p.sponge_top, p.sponge_sigma = int(sponge[0]), float(sponge[1])
    if buffer is not None:
        p.buffer_width, p.buffer_sigma = int(buffer[0]), float(buffer[1])
    p.flux_balance = int(bool(flux_balance))
    return p


# ------------------------------------------------------------------ C-named entry points
def lbm_faces_for_direction(theta: float) -> tuple:
    face = (ctypes.c_int * 6)()
    _check(load(False).lbm_faces_for_direction(theta, face))
    return tuple(FACE_NAMES[v] for v in face)


def lbm_lattice_units(dx_si: float, u_ref_si: float, ma_lbm: float, nu_si: float) -> dict:
    out = (ctypes.c_double * 4)()
    _check(load(False).lbm_lattice_units(float(dx_si), float(u_ref_si), float(ma_lbm), float(nu_si), out))
    return {"dt_si": out[0], "u_lbm": out[1], "nu_lbm": out[2], "tau": out[3]}


def lbm_coriolis_omega(lat_deg: float, dt_si: float):
    out = (ctypes.c_float * 3)()
    _check(load(False).lbm_coriolis_omega(float(lat_deg), float(dt_si), out))
    return tuple(out)


def lbm_workspace_bytes(nx: int, ny: int, nz: int, params: lbm_params) -> int:
    return load(False).lbm_workspace_bytes(nx, ny, nz, ctypes.byref(params))


def lbm_import_populations(dom, g, step: int):
    _check(load().lbm_import_populations(dom, _ptr(g), int(step)), dom)


def lbm_direction_table():
    c = np.zeros(57, np.int32)
    w = np.zeros(19, np.float32)
    load(False).lbm_direction_table(c.ctypes.data, w.ctypes.data)
    return c.reshape(19, 3).astype(np.int64), w


def lbm_create_domain(solid: np.ndarray, params: lbm_params, workspace, stream: int | None):
    solid = np.ascontiguousarray(solid, np.uint8)
    nz, ny, nx = solid.shape
    out = _P()
    st = load().lbm_create_domain(solid.ctypes.data, nx, ny, nz, ctypes.byref(params),
                                  workspace.data_ptr(), workspace.numel() * workspace.element_size(),
                                  stream, ctypes.byref(out))
    _check(st)
    return out


def lbm_set_inflow_profile(dom, speed, theta: float):
    sp = np.ascontiguousarray(speed, np.float32) if not hasattr(speed, "data_ptr") else speed
    _check(load().lbm_set_inflow_profile(dom, _ptr(sp), len(sp), float(theta)), dom)


def lbm_init_fields(dom, rho=None, u=None):
    _check(load().lbm_init_fields(dom, _ptr(rho), _ptr(u)), dom)


def lbm_step(dom, n: int):
    _check(load().lbm_step(dom, int(n)), dom)


def lbm_steps_done(dom) -> int:
    return load().lbm_steps_done(dom)


def lbm_sample_columns(dom, ij, k, out):
    _check(load().lbm_sample_columns(dom, _ptr(ij), ij.shape[0], _ptr(k), k.shape[0], _ptr(out)), dom)


def lbm_macroscopic(dom, rho=None, u=None):
    _check(load().lbm_macroscopic(dom, _ptr(rho), _ptr(u)), dom)


def lbm_export_populations(dom, g):
    _check(load().lbm_export_populations(dom, _ptr(g)), dom)


def lbm_diagnostics(dom) -> dict:
    out = np.zeros(4, np.float64)
    _check(load().lbm_diagnostics(dom, out.ctypes.data), dom)
    return {"mass": out[0], "net_flux": out[1], "umax": out[2], "nonfinite": int(out[3])}


def lbm_diagnostics_noalloc(dom, out):
    """``out``: CUDA float64 tensor of 4 elements, filled asynchronously on the domain's stream."""
    import torch
    if out.dtype.itemsize != 8 or out.numel() < 4 or not out.is_cuda:
        raise ValueError("out must be a CUDA float64 tensor with 4 elements")
    if out.device.index != torch.cuda.current_device():
        raise ValueError("out must live on the current CUDA device (the domain's device)")
    _check(load().lbm_diagnostics_noalloc(dom, _ptr(out)), dom)


def make_stg_params(n_modes=64, length=20.0, intensity=0.1, sigma0=0.0, gain=(1.0, 1.0, 1.0),
                    char_normal=False, inflow_only=False, stride=1, interpolate=True) -> lbm_stg_params:
    p = lbm_stg_params()
    load(False).lbm_stg_params_default(ctypes.byref(p))
    p.n_modes, p.length, p.intensity, p.sigma0 = int(n_modes), float(length), float(intensity), float(sigma0)
    for a in range(3):
        p.gain[a] = float(gain[a])
    p.char_normal, p.inflow_only = int(bool(char_normal)), int(bool(inflow_only))
    p.stride, p.interpolate = int(stride), int(bool(interpolate))
    return p


def lbm_stg_workspace_bytes(dom, n_modes: int) -> int:
    return load(False).lbm_stg_workspace_bytes(dom, int(n_modes))


def lbm_stg_configure(dom, params: lbm_stg_params, uniforms: np.ndarray, workspace):
    """``uniforms``: float64 (6, n_modes, 6) host array; ``workspace``: CUDA uint8 tensor."""
    u = np.ascontiguousarray(uniforms, np.float64)
    if u.shape != (6, params.n_modes, 6):
        raise ValueError("uniforms must be (6, n_modes, 6)")
    _check(load().lbm_stg_configure(dom, ctypes.byref(params), u.ctypes.data, _ptr(workspace),
                                    workspace.numel() * workspace.element_size()), dom)


def lbm_stg_disable(dom):
    _check(load(False).lbm_stg_disable(dom), dom)


def lbm_stg_reference(dom):
    """(u_ref, e_c (3,), bit mask of turbulent faces)."""
    u = ctypes.c_double()
    e = np.zeros(3, np.float64)
    f = ctypes.c_int()
    _check(load(False).lbm_stg_reference(dom, ctypes.byref(u), e.ctypes.data, ctypes.byref(f)), dom)
    return u.value, e, f.value


def make_adjoint_params(n_steps: int, n_avg: int, checkpoint_every: int = 100) -> lbm_adjoint_params:
    p = lbm_adjoint_params()
    p.n_steps, p.n_avg, p.checkpoint_every = int(n_steps), int(n_avg), int(checkpoint_every)
    return p


def lbm_adjoint_workspace_bytes(dom, params: lbm_adjoint_params, ncol: int, nh: int, gradient: bool) -> int:
    return load(False).lbm_adjoint_workspace_bytes(dom, ctypes.byref(params), int(ncol), int(nh),
                                                   int(bool(gradient)))


def _lidar_args(speed, ij, k):
    sp = np.ascontiguousarray(speed, np.float32)
    ij = np.ascontiguousarray(ij, np.int32).reshape(-1, 2)
    k = np.ascontiguousarray(k, np.int32).reshape(-1)
    return sp, ij, k


def lbm_lidar_misfit(dom, params, speed, theta, ij, k, target, workspace, out=None, mean=None):
    """Host ``speed``, ``ij`` (ncol, 2), ``k`` (nh,); CUDA ``target`` float32 (ncol, nh, 2) or
    None, ``workspace`` uint8, ``out`` float64 (1,) and ``mean`` float64 (ncol, nh, 4) or None."""
    sp, ij, k = _lidar_args(speed, ij, k)
    _check(load().lbm_lidar_misfit(dom, ctypes.byref(params), sp.ctypes.data, len(sp), float(theta),
                                   ij.ctypes.data, ij.shape[0], k.ctypes.data, k.shape[0], _ptr(target),
                                   _ptr(workspace), workspace.numel(), _ptr(out), _ptr(mean)), dom)


def lbm_lidar_misfit_grad(dom, params, speed, theta, ij, k, target, workspace, out, mean=None):
    """As ``lbm_lidar_misfit``; ``out`` CUDA float64 (L + 2,) = J, dJ/dspeed[L], dJ/dtheta."""
    sp, ij, k = _lidar_args(speed, ij, k)
    _check(load().lbm_lidar_misfit_grad(dom, ctypes.byref(params), sp.ctypes.data, len(sp), float(theta),
                                        ij.ctypes.data, ij.shape[0], k.ctypes.data, k.shape[0],
                                        _ptr(target), _ptr(workspace), workspace.numel(), _ptr(out),
                                        _ptr(mean)), dom)


def lbm_destroy(dom):
    load(False).lbm_destroy(dom)


# ------------------------------------------------------------------ convenience wrapper
class Domain:
    """One lattice in a torch-owned workspace on the current CUDA device and stream."""

    def __init__(self, solid: np.ndarray, faces, tau: float = 0.52, cs: float = 0.16,
                 store: str = "f32", rho_b: float = 1.0, force=None, watchdog_every: int = 0,
                 device: str = "cuda", stream=None, coriolis=None, sponge=None, buffer=None,
                 flux_balance: bool = False):
        import torch
        load()
        self.shape = tuple(solid.shape)
        nz, ny, nx = self.shape
        self.N = nx * ny * nz
        self.faces = tuple(faces)
        self.store = store
        self.params = make_params(faces, tau, cs, store, rho_b, force, watchdog_every, coriolis,
                                  sponge, buffer, flux_balance)
        nbytes = lbm_workspace_bytes(nx, ny, nz, self.params)
        if nbytes == 0:
            raise LbmError(-1, "invalid domain arguments")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.workspace.device)
        self.dom = lbm_create_domain(solid, self.params, self.workspace, self.stream.cuda_stream)

    # the handle is released with the object; the workspace tensor is freed by torch
    def __del__(self):
        dom = getattr(self, "dom", None)
        if dom:
            lbm_destroy(dom)
            self.dom = None

    @property
    def device(self):
        return self.workspace.device

    def set_inflow_profile(self, speed, theta: float = 0.0):
        lbm_set_inflow_profile(self.dom, speed, theta)

    def init_fields(self, rho=None, u=None):
        import torch
        r = None if rho is None else torch.as_tensor(rho, dtype=torch.float32, device=self.device).contiguous()
        v = None if u is None else torch.as_tensor(u, dtype=torch.float32, device=self.device).contiguous()
        lbm_init_fields(self.dom, r, v)
        self._keep = (r, v)   # keep alive until the stream has consumed them

    def step(self, n: int = 1):
        lbm_step(self.dom, n)

    @property
    def steps_done(self) -> int:
        return lbm_steps_done(self.dom)

    def flux_balance_info(self):
        """(net inflow before, after, normal shift) of the equilibrium cells' profile velocities."""
        v = [ctypes.c_double() for _ in range(3)]
        _check(load(False).lbm_flux_balance_info(self.dom, *[ctypes.byref(x) for x in v]), self.dom)
        return tuple(x.value for x in v)

    def macroscopic(self):
        import torch
        nz, ny, nx = self.shape
        rho = torch.empty((nz, ny, nx), dtype=torch.float32, device=self.device)
        u = torch.empty((nz, ny, nx, 3), dtype=torch.float32, device=self.device)
        lbm_macroscopic(self.dom, rho, u)
        return rho, u

    def export_populations(self):
        import torch
        g = torch.empty((19,) + self.shape, dtype=torch.float32, device=self.device)
        lbm_export_populations(self.dom, g)
        return g

    def import_populations(self, g, step: int):
        """Resume from ``g`` (CUDA float32 (19, nz, ny, nx), as ``export_populations`` returns)."""
        import torch
        g = torch.as_tensor(g, dtype=torch.float32, device=self.device).contiguous()
        lbm_import_populations(self.dom, g, step)
        self._keep_import = g

    def sample_columns(self, ij, k, out=None):
        import torch
        ij = torch.as_tensor(ij, dtype=torch.int32, device=self.device).contiguous()
        k = torch.as_tensor(k, dtype=torch.int32, device=self.device).contiguous()
        if out is None:
            out = torch.empty((ij.shape[0], k.shape[0], 4), dtype=torch.float32, device=self.device)
        lbm_sample_columns(self.dom, ij, k, out)
        return out

    def diagnostics(self) -> dict:
        return lbm_diagnostics(self.dom)

    def configure_stg(self, uniforms, **kw):
        """Synthetic inflow turbulence (App. F) from the next step on; ``kw`` as make_stg_params,
        ``uniforms`` (6, n_modes, 6) random draws (e.g. ``synth.stg_uniforms``)."""
        import torch
        p = make_stg_params(**kw)
        nbytes = lbm_stg_workspace_bytes(self.dom, p.n_modes)
        if nbytes == 0:
            raise LbmError(-1, "no inflow face for synthetic turbulence, or n_modes out of range")
        ws = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        lbm_stg_configure(self.dom, p, uniforms, ws)
        self.stg_workspace = ws   # used by every later step; freed with the domain

    def disable_stg(self):
        lbm_stg_disable(self.dom)

    def stg_reference(self):
        return lbm_stg_reference(self.dom)


class LidarProblem:
    """Virtual-lidar misfit of a domain's inflow (see ``lbm_lidar_misfit_grad`` in ``lbm.h``):
    columns ``cols`` (ncol, 2) = (x, y), heights ``heights`` (nh,), target mean (u, v)
    (ncol, nh, 2); workspaces are torch tensors on the domain's device, allocated on first use."""

    def __init__(self, domain: Domain, cols, heights, target, n_steps: int, n_avg: int,
                 checkpoint_every: int = 100):
        import torch
        self.domain = domain
        self.cols = np.ascontiguousarray(cols, np.int32).reshape(-1, 2)
        self.heights = np.ascontiguousarray(heights, np.int32).reshape(-1)
        self.params = make_adjoint_params(n_steps, n_avg, checkpoint_every)
        self.target = torch.as_tensor(np.asarray(target, np.float32), device=domain.device).contiguous()
        self._ws = {}
        self.reverse_sweeps = 0       # calls that ran the reverse sweep (misfit_grad)

    def _workspace(self, grad: bool):
        import torch
        if grad not in self._ws:
            nb = lbm_adjoint_workspace_bytes(self.domain.dom, self.params, len(self.cols), len(self.heights), grad)
            if nb == 0:
                raise LbmError(-1, "invalid adjoint arguments")
            self._ws[grad] = torch.empty(nb, dtype=torch.uint8, device=self.domain.device)
        return self._ws[grad]

    def misfit(self, speed, theta, target=True):
        """(J, mean (ncol, nh, 4)) as CUDA float64 tensors (J is NaN without a target)."""
        import torch
        out = torch.full((1,), float("nan"), dtype=torch.float64, device=self.domain.device)
        mean = torch.empty((len(self.cols), len(self.heights), 4), dtype=torch.float64, device=self.domain.device)
        lbm_lidar_misfit(self.domain.dom, self.params, speed, theta, self.cols, self.heights,
                         self.target if target else None, self._workspace(False), out, mean)
        return out[0], mean

    def misfit_grad(self, speed, theta):
        """(J, dJ/d(speed..., theta) (L + 1,), mean) as CUDA float64 tensors."""
        import torch
        self.reverse_sweeps += 1
        L = len(speed)
        out = torch.empty((L + 2,), dtype=torch.float64, device=self.domain.device)
        mean = torch.empty((len(self.cols), len(self.heights), 4), dtype=torch.float64, device=self.domain.device)
        lbm_lidar_misfit_grad(self.domain.dom, self.params, speed, theta, self.cols, self.heights,
                              self.target, self._workspace(True), out, mean)
        return out[0], out[1:], mean


def _autograd_function():
    import torch

    class LidarMisfit(torch.autograd.Function):
        """J(p) for p = (speed_0 .. speed_{L-1}, theta) (float64 tensor): when p needs a gradient
        the forward call runs the forward model and the discrete adjoint together
        (``lbm_lidar_misfit_grad``) and backward returns the stored gradient times the incoming
        one; otherwise only the forward model runs (``lbm_lidar_misfit``)."""

        @staticmethod
        def forward(ctx, p, problem):
            pc = p.detach().to("cpu", torch.float64).numpy()
            if not ctx.needs_input_grad[0]:
                J, _ = problem.misfit(pc[:-1], float(pc[-1]))
                return J.to(p.device, p.dtype)
            J, grad, _ = problem.misfit_grad(pc[:-1], float(pc[-1]))
            ctx.save_for_backward(grad.to(p.device, p.dtype))
            return J.to(p.device, p.dtype)

        @staticmethod
        def backward(ctx, gJ):
            (grad,) = ctx.saved_tensors
            return gJ * grad, None

    return LidarMisfit


def lidar_misfit(p, problem: LidarProblem):
    """Differentiable J(p) (torch.autograd): ``p`` = (speed_0 .. speed_{L-1}, theta).  Under
    ``torch.no_grad()``, or for a ``p`` that does not require a gradient, only the forward model
    runs (no reverse sweep)."""
    import torch
    if not (torch.is_grad_enabled() and p.requires_grad):
        pc = p.detach().to("cpu", torch.float64).numpy()
        J, _ = problem.misfit(pc[:-1], float(pc[-1]))
        return J.to(p.device, p.dtype)
    global _LidarMisfit
    try:
        fn = _LidarMisfit
    except NameError:
        fn = _LidarMisfit = _autograd_function()
    return fn.apply(p, problem)


BATCH_SHAPES = ("256 threads, 4 blocks/SM, given order", "256 threads, 3 blocks/SM, given order",
                "256 threads, 4 blocks/SM, largest first", "256 threads, 3 blocks/SM, largest first",
                "one launch per member", "128 threads, 8 blocks/SM", "512 threads, 2 blocks/SM",
                "FP32 one cell per thread", "FP32 two cells per thread", "persistent grid")


def _bcheck(status: int, batch=None):
    if status != 0:
        msg = load(False).lbm_batch_last_error(batch).decode() if batch else ""
        raise LbmError(status, msg)


class Batch:
    """Several ``Domain`` objects advanced together (``lbm_batch_*`` in ``lbm.h``): one launch per
    step over all members, CUDA-graph replay, launch shape by ``autotune``."""

    def __init__(self, domains, stream=None):
        import torch
        self.domains = list(domains)
        n = len(self.domains)
        nbytes = load().lbm_batch_workspace_bytes(n)
        if nbytes == 0:
            raise LbmError(-1, "invalid batch size")
        dev = self.domains[0].device
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        self.stream = stream if stream is not None else self.domains[0].stream
        arr = (_P * n)(*[d.dom for d in self.domains])
        out = _P()
        _bcheck(load().lbm_batch_create(arr, n, self.workspace.data_ptr(), nbytes, self.stream.cuda_stream,
                                        ctypes.byref(out)))
        self.b = out

    def __del__(self):
        b = getattr(self, "b", None)
        if b:
            load(False).lbm_batch_destroy(b)
            self.b = None

    def step(self, n: int = 1):
        _bcheck(load().lbm_batch_step(self.b, int(n)), self.b)

    def capture(self, n: int):
        _bcheck(load().lbm_batch_capture(self.b, int(n)), self.b)

    def launch(self):
        _bcheck(load().lbm_batch_launch(self.b), self.b)

    def autotune(self, trial_steps: int = 20):
        """(chosen shape, ms per step of every shape; -1 where a shape is not available)."""
        choice = ctypes.c_int()
        ms = (ctypes.c_float * len(BATCH_SHAPES))()
        _bcheck(load().lbm_batch_autotune(self.b, int(trial_steps), ctypes.byref(choice), ms), self.b)
        return choice.value, list(ms)

    @property
    def shape(self) -> int:
        return load().lbm_batch_shape(self.b)

    @shape.setter
    def shape(self, s: int):
        _bcheck(load().lbm_batch_set_shape(self.b, int(s)), self.b)


def glups(cells: int, steps: int, seconds: float) -> float:
    return cells * steps / seconds / 1e9 if seconds > 0 else math.nan

"""GB300-native Press-Ryden-Spergel domain-wall evolution (arXiv:1710.10420).

Thin Python binding of the C ABI in ``include/prs.h`` (library ``_lib/libprs.so``).
The functions below carry the C names and only marshal arguments; every step of
the method runs in the library's CUDA kernels.  PyTorch is used for device
memory and streams (``Sim`` binds torch tensors as the field buffers).

There is no CPU fallback: if the library is missing or fails to load, every call
raises ``PRSError``.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

from . import _build

PRS_OK = 0
PRS_EINVAL = -1
PRS_ENOMEM = -2
PRS_ECUDA = -3
PRS_ETIMEOUT = -4
PRS_ENONFINITE = -5
PRS_ESTATE = -6
PRS_FP32 = 0
PRS_FP64 = 1
PRS_REPRO = 1
PRS_FP32_CR = 2
PRS_DEBUG = 4
PRS_OBS_GRAD_ENERGY = 0
PRS_OBS_SMOOTH_AREA = 1

HEADERS = [os.path.join(_build.INCLUDE, h) for h in sorted(os.listdir(_build.INCLUDE)) if h.endswith(".h")]


class PRSError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        msg = f"{where}: {strerror(status) if _lib is not None else status}"
        if detail:
            msg += f" ({detail})"
        super().__init__(msg)


class prs_params(ctypes.Structure):
    """Mirror of ``prs_params`` (include/prs.h)."""
    _fields_ = [
        ("dims", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("N", ctypes.c_int64),
        ("Ny", ctypes.c_int64),
        ("Nz", ctypes.c_int64),
        ("dx", ctypes.c_double),
        ("deta", ctypes.c_double),
        ("eta0", ctypes.c_double),
        ("alpha", ctypes.c_double),
        ("beta", ctypes.c_double),
        ("era_m", ctypes.c_double),
        ("W0", ctypes.c_double),
        ("phi0", ctypes.c_double),
        ("seed", ctypes.c_uint64),
        ("flags", ctypes.c_uint32),
        ("tblock", ctypes.c_int32),
    ]


class prs_diag(ctypes.Structure):
    """Mirror of ``prs_diag`` (include/prs.h)."""
    _fields_ = [
        ("area_per_volume", ctypes.c_double),
        ("gamma_v", ctypes.c_double),
        ("sum_w", ctypes.c_double),
        ("sum_ratio", ctypes.c_double),
        ("n_links", ctypes.c_int64),
        ("n_wall", ctypes.c_int64),
        ("n_vzero", ctypes.c_int64),
        ("n_nonfinite", ctypes.c_int64),
        ("step", ctypes.c_int64),
        ("eta", ctypes.c_double),
    ]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


def make_params(shape, precision=PRS_FP32, dx=1.0, deta=0.1, eta0=1.0, alpha=3.0, beta=0.0, era_m=1.0, W0=10.0,
                phi0=1.0, seed=0, flags=0, tblock=0) -> prs_params:
    """prs_params for a box of ``shape`` = (nx, ny) or (nx, ny, nz); x runs fastest."""
    shape = tuple(int(s) for s in shape)
    dims = len(shape)
    return prs_params(dims, precision, shape[0], shape[1], shape[2] if dims == 3 else 0, dx, deta, eta0, alpha, beta,
                      era_m, W0, phi0, seed, flags, tblock)


_lib = None
_P = ctypes.POINTER(prs_params)
_VP = ctypes.c_void_p
_I64P = ctypes.POINTER(ctypes.c_int64)
_DP = ctypes.POINTER(ctypes.c_double)

# name -> (restype, argtypes)
_SIGS = {
    "prs_create": (ctypes.c_int, [_P, _VP, ctypes.POINTER(_VP)]),
    "prs_bind": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "prs_init": (ctypes.c_int, [_VP, _VP, _VP]),
    "prs_step": (ctypes.c_int, [_VP, ctypes.c_int64]),
    "prs_measure": (ctypes.c_int, [_VP, _DP, _DP, _I64P, _I64P]),
    "prs_measure_ex": (ctypes.c_int, [_VP, ctypes.POINTER(prs_diag)]),
    "prs_step_measure": (ctypes.c_int, [_VP, ctypes.c_int64, ctypes.POINTER(prs_diag)]),
    "prs_get_state": (ctypes.c_int, [_VP, _VP, _VP, _I64P]),
    "prs_set_state": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int64]),
    "prs_set_state_async": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int64]),
    "prs_set_state_device": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int64]),
    "prs_device_state": (ctypes.c_int, [_VP, ctypes.POINTER(_VP), ctypes.POINTER(_VP), _I64P]),
    "prs_destroy": (ctypes.c_int, [_VP]),
    "prs_coefficients": (ctypes.c_int, [_P, ctypes.c_int64, _DP]),
    "prs_default_tblock": (ctypes.c_int, [_P]),
    "prs_max_tblock": (ctypes.c_int, [_P]),
    "prs_selftest_wait_timeout": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_uint)]),
    "prs_batch_create": (ctypes.c_int, [_P, ctypes.c_int, _VP, ctypes.POINTER(_VP)]),
    "prs_batch_run": (ctypes.c_int, [_VP, _I64P, ctypes.c_int64, _DP, ctypes.c_int64]),
    "prs_batch_get_state": (ctypes.c_int, [_VP, ctypes.c_int, _VP, _VP, _I64P]),
    "prs_batch_set_state": (ctypes.c_int, [_VP, ctypes.c_int, _VP, _VP, ctypes.c_int64]),
    "prs_batch_tuning": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_int), _DP]),
    "prs_batch_destroy": (ctypes.c_int, [_VP]),
    "prs_observable": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_double, _DP]),
    "prs_adjoint": (ctypes.c_int, [_VP, ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_int64, _DP, _DP, _VP,
                                   _VP]),
    "prs_measure_noalloc": (ctypes.c_int, [_P, _VP, _VP, _VP, ctypes.POINTER(prs_diag)]),
    "prs_adjoint_timing": (ctypes.c_int, [_VP, _DP]),
    "prs_set_deta": (ctypes.c_int, [_VP, ctypes.c_double]),
    "prs_stable_deta": (ctypes.c_int, [_P, ctypes.c_double, _DP]),
    "prs_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "prs_last_error": (ctypes.c_char_p, []),
}


def library_path() -> str:
    return _build.LIB


def load(build: bool = False) -> ctypes.CDLL:
    """Load libprs.so (building it first when ``build``); raises PRSError if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if build:
        _build.build()
    path = _build.LIB
    if not os.path.exists(path):
        raise PRSError(PRS_ESTATE, "load", f"{path} is missing: run __graft_entry__.build() (nvcc, sm_103a)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def declared_functions() -> list:
    """Names of every function declared in include/*.h."""
    names = []
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(prs_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def _check(rc: int, where: str, ok=(PRS_OK,)) -> int:
    if rc not in ok:
        detail = ""
        if rc in (PRS_ECUDA, PRS_ETIMEOUT):  # the library records the text of these
            detail = _lib.prs_last_error().decode()
        raise PRSError(rc, where, detail)
    return rc


def strerror(status: int) -> str:
    return load().prs_strerror(status).decode()


def _ptr(a) -> int:
    """Address of a numpy array or torch tensor (contiguous), or None."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return a.ctypes.data
    return a.data_ptr()


# ---------------------------------------------------------------- C names

def prs_create(params: prs_params, stream=None) -> ctypes.c_void_p:
    h = _VP()
    _check(load().prs_create(ctypes.byref(params), stream, ctypes.byref(h)), "prs_create")
    return h


def prs_bind(sim, d_phi_a, d_phi_b, d_dphi) -> None:
    _check(load().prs_bind(sim, _ptr(d_phi_a), _ptr(d_phi_b), _ptr(d_dphi)), "prs_bind")


def prs_init(sim, h_phi=None, h_dphi=None) -> None:
    _check(load().prs_init(sim, _ptr(h_phi), _ptr(h_dphi)), "prs_init")


def prs_step(sim, nsteps: int) -> None:
    _check(load().prs_step(sim, nsteps), "prs_step")


def prs_measure(sim):
    a, g = ctypes.c_double(), ctypes.c_double()
    nl, nw = ctypes.c_int64(), ctypes.c_int64()
    rc = load().prs_measure(sim, ctypes.byref(a), ctypes.byref(g), ctypes.byref(nl), ctypes.byref(nw))
    _check(rc, "prs_measure", ok=(PRS_OK, PRS_ENONFINITE))
    return a.value, g.value, nl.value, nw.value


def prs_measure_ex(sim) -> prs_diag:
    d = prs_diag()
    _check(load().prs_measure_ex(sim, ctypes.byref(d)), "prs_measure_ex", ok=(PRS_OK, PRS_ENONFINITE))
    return d


def prs_step_measure(sim, nsteps: int) -> prs_diag:
    """Diagnostics of the current state, computed inside the first of nsteps steps."""
    d = prs_diag()
    _check(load().prs_step_measure(sim, nsteps, ctypes.byref(d)), "prs_step_measure", ok=(PRS_OK, PRS_ENONFINITE))
    return d


def prs_get_state(sim, h_phi=None, h_dphi=None) -> int:
    n = ctypes.c_int64()
    _check(load().prs_get_state(sim, _ptr(h_phi), _ptr(h_dphi), ctypes.byref(n)), "prs_get_state")
    return n.value


def prs_set_state(sim, h_phi, h_dphi, n: int) -> None:
    _check(load().prs_set_state(sim, _ptr(h_phi), _ptr(h_dphi), n), "prs_set_state")


def prs_set_state_device(sim, d_phi, d_dphi, n: int) -> None:
    """Device-to-device state copy, queued on the run's stream (torch tensors or raw pointers)."""
    p = d_phi if isinstance(d_phi, int) else _ptr(d_phi)
    v = d_dphi if isinstance(d_dphi, int) else _ptr(d_dphi)
    _check(load().prs_set_state_device(sim, p, v, n), "prs_set_state_device")


def prs_set_state_async(sim, h_phi, h_dphi, n: int) -> None:
    """Queue the upload and return; the arrays must stay alive and unchanged until the run
    next synchronises (pinned memory, e.g. a torch tensor with pin_memory=True, overlaps)."""
    _check(load().prs_set_state_async(sim, _ptr(h_phi), _ptr(h_dphi), n), "prs_set_state_async")


def prs_device_state(sim):
    p, v, n = _VP(), _VP(), ctypes.c_int64()
    _check(load().prs_device_state(sim, ctypes.byref(p), ctypes.byref(v), ctypes.byref(n)), "prs_device_state")
    return p.value, v.value, n.value


def prs_destroy(sim) -> None:
    _check(load().prs_destroy(sim), "prs_destroy")


def prs_measure_noalloc(params: prs_params, d_phi, d_dphi, stream=None) -> prs_diag:
    """Diagnostics of caller-owned device fields; the call allocates no device memory."""
    d = prs_diag()
    p = d_phi if isinstance(d_phi, int) else _ptr(d_phi)
    v = d_dphi if isinstance(d_dphi, int) else _ptr(d_dphi)
    _check(load().prs_measure_noalloc(ctypes.byref(params), p, v, stream, ctypes.byref(d)), "prs_measure_noalloc",
           ok=(PRS_OK, PRS_ENONFINITE))
    return d


def prs_observable(sim, observable: int, eps_smooth: float = 0.1) -> float:
    J = ctypes.c_double()
    _check(load().prs_observable(sim, observable, eps_smooth, ctypes.byref(J)), "prs_observable")
    return J.value


def prs_adjoint(sim, nsteps: int, observable: int, eps_smooth: float = 0.1, ckpt_every: int = 64, d_dJ_dphi=None,
                d_dJ_dv=None):
    """Run nsteps and return (J, dJ/dalpha); gradients w.r.t. the start state go to the given device tensors."""
    J, da = ctypes.c_double(), ctypes.c_double()
    _check(load().prs_adjoint(sim, nsteps, observable, eps_smooth, ckpt_every, ctypes.byref(J), ctypes.byref(da),
                              _ptr(d_dJ_dphi), _ptr(d_dJ_dv)), "prs_adjoint")
    return J.value, da.value


def prs_batch_create(runs, stream=None) -> ctypes.c_void_p:
    """runs: a sequence of prs_params."""
    arr = (prs_params * len(runs))(*runs)
    h = _VP()
    _check(load().prs_batch_create(arr, len(runs), stream, ctypes.byref(h)), "prs_batch_create")
    return h


def prs_batch_run(batch, nsteps_per_run, measure_every: int = 0, out_capacity: int = 0):
    """Returns the diagnostic series as a numpy array [run][output][4] (step, A/V, gamma v, n_links)."""
    ns = np.ascontiguousarray(nsteps_per_run, dtype=np.int64)
    out = np.zeros((len(ns), max(out_capacity, 1), 4))
    _check(load().prs_batch_run(batch, ns.ctypes.data_as(_I64P), measure_every,
                                out.ctypes.data_as(_DP) if measure_every > 0 else None, out_capacity),
           "prs_batch_run")
    return out


def prs_batch_get_state(batch, run: int, h_phi=None, h_dphi=None) -> int:
    n = ctypes.c_int64()
    _check(load().prs_batch_get_state(batch, run, _ptr(h_phi), _ptr(h_dphi), ctypes.byref(n)), "prs_batch_get_state")
    return n.value


def prs_batch_set_state(batch, run: int, h_phi, h_dphi, n: int) -> None:
    phi = np.ascontiguousarray(h_phi, dtype=np.float32)  # kept alive across the call
    dphi = np.ascontiguousarray(h_dphi, dtype=np.float32)
    _check(load().prs_batch_set_state(batch, run, _ptr(phi), _ptr(dphi), n), "prs_batch_set_state")


def prs_batch_tuning(batch, run: int):
    t, g = ctypes.c_int(), ctypes.c_double()
    _check(load().prs_batch_tuning(batch, run, ctypes.byref(t), ctypes.byref(g)), "prs_batch_tuning")
    return t.value, g.value


def prs_batch_destroy(batch) -> None:
    _check(load().prs_batch_destroy(batch), "prs_batch_destroy")


def prs_selftest_wait_timeout(stream=None):
    """Returns (status, error bits): PRS_ETIMEOUT when every bounded wait gave up as it should."""
    codes = ctypes.c_uint()
    rc = load().prs_selftest_wait_timeout(stream, ctypes.byref(codes))
    return rc, codes.value


def prs_default_tblock(params: prs_params) -> int:
    rc = load().prs_default_tblock(ctypes.byref(params))
    if rc < 0:
        _check(rc, "prs_default_tblock")
    return rc


def prs_max_tblock(params: prs_params) -> int:
    rc = load().prs_max_tblock(ctypes.byref(params))
    if rc < 0:
        _check(rc, "prs_max_tblock")
    return rc


def prs_set_deta(sim, deta: float) -> None:
    _check(load().prs_set_deta(sim, deta), "prs_set_deta")


def prs_stable_deta(params: prs_params, eta: float) -> float:
    out = ctypes.c_double()
    _check(load().prs_stable_deta(ctypes.byref(params), eta, ctypes.byref(out)), "prs_stable_deta")
    return out.value


def prs_adjoint_timing(sim) -> dict:
    """Phase times of the last prs_adjoint call (ms): forward, recompute, reverse."""
    out = (ctypes.c_double * 3)()
    _check(load().prs_adjoint_timing(sim, out), "prs_adjoint_timing")
    return dict(forward_ms=out[0], recompute_ms=out[1], reverse_ms=out[2])


def prs_strerror(status: int) -> str:
    return strerror(status)


def prs_last_error() -> str:
    return load().prs_last_error().decode()


def prs_coefficients(params: prs_params, n: int) -> dict:
    out = (ctypes.c_double * 5)()
    _check(load().prs_coefficients(ctypes.byref(params), n, out), "prs_coefficients")
    return dict(c1=out[0], c2=out[1], cV=out[2], delta=out[3], ddelta_dalpha=out[4])


# ------------------------------------------------------------ convenience

class Sim:
    """One run whose field buffers are torch CUDA tensors bound through prs_bind.

    ``shape`` is (nx, ny[, nz]); tensors have shape (nz, ny, nx) / (ny, nx).
    """

    def __init__(self, shape, precision=PRS_FP32, stream=None, device=None, **kw):
        import torch

        self.params = make_params(shape, precision=precision, **kw)
        self.shape = tuple(int(s) for s in shape)
        self.array_shape = tuple(reversed(self.shape))
        self.dtype = torch.float32 if precision == PRS_FP32 else torch.float64
        self.np_dtype = np.float32 if precision == PRS_FP32 else np.float64
        dev = torch.device(device if device is not None else "cuda")
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        self._bufs = [torch.empty(self.array_shape, dtype=self.dtype, device=dev) for _ in range(3)]
        self.handle = prs_create(self.params, self.stream.cuda_stream)
        prs_bind(self.handle, *self._bufs)

    def init(self, phi=None, dphi=None):
        phi = None if phi is None else np.ascontiguousarray(phi, dtype=self.np_dtype)
        dphi = None if dphi is None else np.ascontiguousarray(dphi, dtype=self.np_dtype)
        prs_init(self.handle, phi, dphi)
        return self

    def step(self, nsteps: int):
        prs_step(self.handle, nsteps)
        return self

    def measure(self) -> dict:
        return prs_measure_ex(self.handle).as_dict()

    def get_state(self):
        phi = np.empty(self.array_shape, dtype=self.np_dtype)
        dphi = np.empty(self.array_shape, dtype=self.np_dtype)
        n = prs_get_state(self.handle, phi, dphi)
        return phi, dphi, n

    def set_state(self, phi, dphi, n: int):
        prs_set_state(self.handle, np.ascontiguousarray(phi, dtype=self.np_dtype),
                      np.ascontiguousarray(dphi, dtype=self.np_dtype), n)

    def tensors(self):
        """(phi, dphi, n): the torch tensors holding the current state (no copy)."""
        p, v, n = prs_device_state(self.handle)
        phi = next(b for b in self._bufs if b.data_ptr() == p)
        dphi = next(b for b in self._bufs if b.data_ptr() == v)
        return phi, dphi, n

    def close(self):
        if getattr(self, "handle", None) is not None:
            prs_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def observable_with_grad(shape, phi_init, v_init, nsteps, observable, eps_smooth=0.1, ckpt_every=64,
                         precision=PRS_FP32, **kw):
    """Differentiable J(phi after nsteps) as a torch.autograd.Function over (phi_init, v_init, alpha).

    phi_init, v_init: CUDA tensors of the field's shape; the returned scalar tensor
    backpropagates dJ/dphi_init, dJ/dv_init and dJ/dalpha (alpha is a 0-d tensor
    holding the damping coefficient of Eq. 2) through prs_adjoint.
    """
    import torch

    class _PRSObservable(torch.autograd.Function):
        @staticmethod
        def forward(ctx, phi0, v0, alpha):
            sim = Sim(shape, precision=precision, alpha=float(alpha.item()), device=phi0.device, **kw)
            # device to device, on the run's stream (the caller's current stream)
            phi_c = phi0.detach().to(sim.dtype).contiguous()
            v_c = v0.detach().to(device=phi0.device, dtype=sim.dtype).contiguous()
            sim.stream.wait_stream(torch.cuda.current_stream(phi0.device))
            prs_set_state_device(sim.handle, phi_c, v_c, 0)
            gphi = torch.empty_like(phi0)
            gv = torch.empty_like(v0)
            J, dA = prs_adjoint(sim.handle, nsteps, observable, eps_smooth, ckpt_every, gphi, gv)
            sim.close()
            ctx.save_for_backward(gphi, gv)
            ctx.dA = dA
            ctx.alpha_device = alpha.device
            return torch.tensor(J, dtype=torch.float64, device=phi0.device)

        @staticmethod
        def backward(ctx, gJ):
            gphi, gv = ctx.saved_tensors
            s = gJ.to(gphi.dtype)
            galpha = (gJ.detach() * ctx.dA).to(device=ctx.alpha_device, dtype=torch.float64)
            return gphi * s, gv * s, galpha

    alpha = kw.pop("alpha_tensor", None)
    if alpha is None:
        import torch as _t
        alpha = _t.tensor(kw.pop("alpha", 3.0), dtype=_t.float64, requires_grad=True)
    return _PRSObservable.apply(phi_init, v_init, alpha)

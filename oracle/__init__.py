"""FP64 CPU oracle for the Press-Ryden-Spergel domain-wall method (arXiv:1710.10420).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline / reference legs of ``bench.py`` may import this package.  It shares no
code with the CUDA library and the library never calls it.

The arithmetic lives in ``prs_oracle.c`` (plain C, FP64, compiled with
``-O2 -ffp-contract=off``); this module only compiles it with gcc and marshals
numpy arrays through ctypes.  Each function names the passage of the paper it
follows; the C file's header lists the readings taken where the paper is silent.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "prs_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")

CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c11"]


def build(force: bool = False) -> str:
    """Compile ``prs_oracle.c`` into ``oracle/_build/liboracle.so`` (gcc, no FMA)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=os.path.dirname(_LIB))
    os.close(fd)
    subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [
        ("dims", ctypes.c_int32),
        ("pad_", ctypes.c_int32),
        ("nx", ctypes.c_int64),
        ("ny", ctypes.c_int64),
        ("nz", ctypes.c_int64),
        ("dx", ctypes.c_double),
        ("deta", ctypes.c_double),
        ("eta0", ctypes.c_double),
        ("alpha", ctypes.c_double),
        ("beta", ctypes.c_double),
        ("era_m", ctypes.c_double),
        ("W0", ctypes.c_double),
        ("phi0", ctypes.c_double),
    ]


class _Diag(ctypes.Structure):
    _fields_ = [
        ("area_per_volume", ctypes.c_double),
        ("gamma_v", ctypes.c_double),
        ("sum_w", ctypes.c_double),
        ("sum_ratio", ctypes.c_double),
        ("n_links", ctypes.c_int64),
        ("n_wall", ctypes.c_int64),
        ("n_vzero", ctypes.c_int64),
        ("n_nonfinite", ctypes.c_int64),
    ]


_lib = None


def _L():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.POINTER(_Params)
        D = ctypes.POINTER(ctypes.c_double)
        lib.orc_splitmix64.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        lib.orc_splitmix64.restype = ctypes.c_uint64
        lib.orc_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        lib.orc_uniform.restype = ctypes.c_double
        lib.orc_init_random.argtypes = [P, ctypes.c_uint64, D, D]
        lib.orc_init_random.restype = None
        lib.orc_V0.argtypes = [P]
        lib.orc_V0.restype = ctypes.c_double
        lib.orc_coeffs.argtypes = [P, ctypes.c_int64, D]
        lib.orc_coeffs.restype = None
        lib.orc_step.argtypes = [P, ctypes.c_int64, ctypes.c_int64, D, D]
        lib.orc_step.restype = ctypes.c_int
        lib.orc_measure.argtypes = [P, D, D, ctypes.POINTER(_Diag)]
        lib.orc_measure.restype = None
        lib.orc_observable.argtypes = [P, ctypes.c_int, ctypes.c_double, D]
        lib.orc_observable.restype = ctypes.c_double
        lib.orc_observable_grad.argtypes = [P, ctypes.c_int, ctypes.c_double, D, D]
        lib.orc_observable_grad.restype = None
        lib.orc_adjoint.argtypes = [P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_double, D, D, D, D,
                                    D, D]
        lib.orc_adjoint.restype = ctypes.c_int
        _lib = lib
    return _lib


@dataclass
class Params:
    """Physical and lattice parameters (Eq. 2, Eq. 6; configs use dx=1, deta=0.1, eta0=1).

    ``shape`` is (nx, ny) in 2D or (nx, ny, nz) in 3D; x runs fastest in memory.
    PRS is alpha=3, beta=0 (Sec. II); ``era_m`` = dln a / dln eta (1 radiation, 2 matter).
    ``W0`` is the wall thickness, V0 = pi^2/(2 W0^2); ``math.inf`` gives a free field.
    """

    shape: tuple
    dx: float = 1.0
    deta: float = 0.1
    eta0: float = 1.0
    alpha: float = 3.0
    beta: float = 0.0
    era_m: float = 1.0
    W0: float = 10.0
    phi0: float = 1.0

    @property
    def dims(self) -> int:
        return len(self.shape)

    @property
    def sites(self) -> int:
        return int(np.prod(self.shape))

    def _c(self) -> _Params:
        nx, ny = int(self.shape[0]), int(self.shape[1])
        nz = int(self.shape[2]) if self.dims == 3 else 1
        if self.dims not in (2, 3):
            raise ValueError("dims must be 2 or 3")
        return _Params(self.dims, 0, nx, ny, nz, self.dx, self.deta, self.eta0, self.alpha, self.beta, self.era_m,
                       self.W0, self.phi0)

    def array_shape(self) -> tuple:
        """numpy shape of a field: (nz, ny, nx) or (ny, nx), x last (fastest)."""
        return tuple(reversed([int(n) for n in self.shape]))


def _dptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def splitmix64(seed: int, idx: int) -> int:
    """SplitMix64 output number ``idx`` of the generator seeded with ``seed``."""
    return int(_L().orc_splitmix64(seed, idx))


def uniform(seed: int, idx: int) -> float:
    """Initial-condition value (2k+1) 2^-24 - 1 from the top 24 bits of SplitMix64."""
    return float(_L().orc_uniform(seed, idx))


def init_random(p: Params, seed: int):
    """Random initial field phi in (-1, 1) and zero velocity (the paper's random ICs)."""
    phi = np.empty(p.array_shape())
    v = np.empty(p.array_shape())
    c = p._c()
    _L().orc_init_random(ctypes.byref(c), seed, _dptr(phi), _dptr(v))
    return phi, v


def V0(p: Params) -> float:
    c = p._c()
    return float(_L().orc_V0(ctypes.byref(c)))


def coeffs(p: Params, n: int) -> dict:
    """Step-n coefficients: c1, c2 (Eq. 4 with Eq. 6), cV (force prefactor), delta, d delta/d alpha."""
    out = (ctypes.c_double * 5)()
    c = p._c()
    _L().orc_coeffs(ctypes.byref(c), n, out)
    return dict(c1=out[0], c2=out[1], cV=out[2], delta=out[3], ddelta_dalpha=out[4])


def step(p: Params, phi, v, nsteps: int, n0: int = 0):
    """Apply ``nsteps`` leapfrog steps (Eqs. 3-5) starting at step index n0; returns new arrays."""
    phi = _f64(phi).copy()
    v = _f64(v).copy()
    c = p._c()
    if _L().orc_step(ctypes.byref(c), n0, nsteps, _dptr(phi), _dptr(v)) != 0:
        raise MemoryError("oracle step: out of memory")
    return phi, v


@dataclass
class Diag:
    area_per_volume: float
    gamma_v: float
    sum_w: float
    sum_ratio: float
    n_links: int
    n_wall: int
    n_vzero: int
    n_nonfinite: int


def measure(p: Params, phi, v) -> Diag:
    """Wall diagnostics of Eq. 7 (A/V) and Eq. 8 (gamma v) on (phi^n, dphi^{n-1/2})."""
    phi = _f64(phi)
    v = _f64(v)
    d = _Diag()
    c = p._c()
    _L().orc_measure(ctypes.byref(c), _dptr(phi), _dptr(v), ctypes.byref(d))
    return Diag(d.area_per_volume, d.gamma_v, d.sum_w, d.sum_ratio, d.n_links, d.n_wall, d.n_vzero, d.n_nonfinite)


def observable(p: Params, obs: int, phi, eps: float = 0.1) -> float:
    """obs 0: gradient energy; obs 1: tanh(phi/eps)-smoothed wall area per volume."""
    c = p._c()
    return float(_L().orc_observable(ctypes.byref(c), obs, eps, _dptr(_f64(phi))))


def observable_grad(p: Params, obs: int, phi, eps: float = 0.1) -> np.ndarray:
    phi = _f64(phi)
    g = np.empty_like(phi)
    c = p._c()
    _L().orc_observable_grad(ctypes.byref(c), obs, eps, _dptr(phi), _dptr(g))
    return g


def adjoint(p: Params, phi, v, nsteps: int, obs: int, eps: float = 0.1, n0: int = 0):
    """J(phi after nsteps) and its gradient w.r.t. (phi_init, v_init, alpha), by reverse-time adjoint."""
    phi = _f64(phi)
    v = _f64(v)
    gphi = np.empty_like(phi)
    gv = np.empty_like(phi)
    J = ctypes.c_double()
    dA = ctypes.c_double()
    c = p._c()
    rc = _L().orc_adjoint(ctypes.byref(c), n0, nsteps, obs, eps, _dptr(phi), _dptr(v), ctypes.byref(J),
                          ctypes.byref(dA), _dptr(gphi), _dptr(gv))
    if rc != 0:
        raise MemoryError("oracle adjoint: out of memory")
    return dict(J=J.value, dJ_dalpha=dA.value, dJ_dphi=gphi, dJ_dv=gv)


__all__ = ["Params", "Diag", "build", "splitmix64", "uniform", "init_random", "V0", "coeffs", "step", "measure",
           "observable", "observable_grad", "adjoint"]

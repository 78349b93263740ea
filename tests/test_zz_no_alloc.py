"""prs_measure_noalloc: the diagnostics for callers that cannot allocate device memory.

Such callers (an application that owns every device allocation, or a loop that
cannot afford cudaMalloc's device-wide synchronisation) get the same record as
prs_measure_ex, computed with scratch in a fixed array compiled into the library.
These tests call it through the C ABI on fields held by an ordinary run and
compare it with prs_measure_ex: counts exactly; A/V and gamma v to 1e-13 relative
in FP64 (only the order of the FP64 reduction differs) and to the FP32 diagnostic
tolerance of the parity tests, 1e-5, in FP32 (for x sides that are multiples of
128, prs_measure_ex uses the plane-staged kernel, whose per-site float rounding
may differ).  The file is collected last so that a failure here comes after
every other test has run.
"""
import ctypes

import numpy as np
import pytest

import paper_1710_10420_gb300 as prs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch

    assert torch.cuda.is_available()
    prs.load(build=True)


def _check_same(d, ref, precision):
    tol = 1e-13 if precision == prs.PRS_FP64 else 1e-5
    assert (d.n_links, d.n_wall, d.n_vzero, d.n_nonfinite) == (ref.n_links, ref.n_wall, ref.n_vzero, ref.n_nonfinite)
    assert d.area_per_volume == pytest.approx(ref.area_per_volume, rel=tol)
    assert d.gamma_v == pytest.approx(ref.gamma_v, rel=tol)


def _sim(shape, precision, seed, nsteps):
    sim = prs.Sim(shape, precision=precision, seed=seed, W0=6.0)
    sim.init()
    sim.step(nsteps)
    return sim


@pytest.mark.parametrize("precision,shape", [(prs.PRS_FP64, (64, 48)), (prs.PRS_FP32, (96, 80, 40)),
                                             (prs.PRS_FP32, (256, 256, 256))])
def test_noalloc_matches_measure_twice(precision, shape):
    sim = _sim(shape, precision, seed=5, nsteps=15)
    ref = prs.prs_measure_ex(sim.handle)
    d_phi, d_dphi, _ = prs.prs_device_state(sim.handle)
    stream = sim.stream.cuda_stream
    for _ in range(2):
        d = prs.prs_measure_noalloc(sim.params, d_phi, d_dphi, stream)
        _check_same(d, ref, precision)
    sim.close()


def test_noalloc_at_its_site_limit():
    """2^30 sites (1024^3 FP32, the headline box), the documented maximum: the blocks
    stride over the rows on a grid that stays within CUDA's gridDim.y limit."""
    import torch

    shape = (1024, 1024, 1024)
    sim = _sim(shape, prs.PRS_FP32, seed=9, nsteps=3)
    ref = prs.prs_measure_ex(sim.handle)
    d_phi, d_dphi, _ = prs.prs_device_state(sim.handle)
    for _ in range(2):
        d = prs.prs_measure_noalloc(sim.params, d_phi, d_dphi, sim.stream.cuda_stream)
        _check_same(d, ref, prs.PRS_FP32)
    sim.close()
    del sim
    torch.cuda.empty_cache()


def test_noalloc_alternating_runs():
    """The shared array keeps the previous call's contents; results must not depend on it."""
    a = _sim((128, 96), prs.PRS_FP32, seed=1, nsteps=10)
    b = _sim((40, 36, 30), prs.PRS_FP64, seed=2, nsteps=10)
    ra, rb = prs.prs_measure_ex(a.handle), prs.prs_measure_ex(b.handle)
    for sim, ref, prec in [(a, ra, prs.PRS_FP32), (b, rb, prs.PRS_FP64), (a, ra, prs.PRS_FP32)]:
        p, v, _ = prs.prs_device_state(sim.handle)
        _check_same(prs.prs_measure_noalloc(sim.params, p, v, sim.stream.cuda_stream), ref, prec)
    a.close()
    b.close()


def test_noalloc_rejects_lattices_beyond_the_scratch():
    sim = _sim((16, 16), prs.PRS_FP32, seed=3, nsteps=1)
    p, v, _ = prs.prs_device_state(sim.handle)
    big = prs.make_params((2048, 1024, 1024))
    out = prs.prs_diag()
    rc = prs.load().prs_measure_noalloc(ctypes.byref(big), p, v, None, ctypes.byref(out))
    assert rc == prs.PRS_EINVAL
    assert "exceed the static scratch" in prs.prs_last_error()
    sim.close()

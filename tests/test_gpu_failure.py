"""Failure detection on the GPU without a fault: bounded waits that give up, allocation
failure and calls out of order all come back as status codes, and the context stays usable."""
import ctypes

import numpy as np
import pytest

import oracle
import paper_1710_10420_gb300 as prs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch

    assert torch.cuda.is_available()
    prs.load(build=True)


def _still_works():
    shape = (32, 24)
    sim = prs.Sim(shape, precision=prs.PRS_FP64, flags=prs.PRS_REPRO, seed=3)
    sim.init()
    sim.step(5)
    phi, _, _ = sim.get_state()
    sim.close()
    p = oracle.Params(shape)
    ophi, _ = oracle.step(p, *oracle.init_random(p, 3), 5)
    assert np.array_equal(phi, ophi)


def test_bounded_waits_give_up_and_report():
    rc, codes = prs.prs_selftest_wait_timeout()
    assert rc == prs.PRS_ETIMEOUT
    assert codes == 7  # mbarrier wait (1, 2) and flag wait (4) both gave up
    _still_works()


def test_allocation_failure_is_reported():
    lib = prs.load()
    p = prs.make_params((1 << 16, 1 << 16, 1 << 12))  # 70 TB of fields
    h = ctypes.c_void_p()
    assert lib.prs_create(ctypes.byref(p), None, ctypes.byref(h)) == prs.PRS_OK
    assert lib.prs_init(h, None, None) == prs.PRS_ENOMEM
    assert lib.prs_destroy(h) == prs.PRS_OK
    _still_works()


def test_calls_out_of_order():
    lib = prs.load()
    p = prs.make_params((16, 16))
    h = ctypes.c_void_p()
    assert lib.prs_create(ctypes.byref(p), None, ctypes.byref(h)) == prs.PRS_OK
    assert lib.prs_step(h, 3) == prs.PRS_ESTATE
    assert lib.prs_measure(h, None, None, None, None) == prs.PRS_ESTATE
    d = ctypes.c_double()
    assert lib.prs_observable(h, 0, 0.1, ctypes.byref(d)) == prs.PRS_ESTATE
    assert lib.prs_destroy(h) == prs.PRS_OK


def test_stability_limit_checked_at_every_call():
    """With beta > 0 the force grows as a^beta = eta^(m beta); prs_step refuses steps past the CFL limit."""
    lib = prs.load()
    p = prs.make_params((16, 16), beta=2.0, era_m=1.0, W0=4.0)
    h = ctypes.c_void_p()
    assert lib.prs_create(ctypes.byref(p), None, ctypes.byref(h)) == prs.PRS_OK
    assert lib.prs_init(h, None, None) == prs.PRS_OK
    assert lib.prs_step(h, 10) == prs.PRS_OK
    assert lib.prs_step(h, 1000) == prs.PRS_EINVAL  # cV eta^2 grows past the leapfrog limit
    assert lib.prs_destroy(h) == prs.PRS_OK


# ------------------------------------------------------------------ PRS_DEBUG

def _raw_run(shape, flags, precision=prs.PRS_FP32, seed=5, tblock=0):
    """A run on library-owned buffers (prs_create + prs_init), as a C caller makes one."""
    import torch

    h = prs.prs_create(prs.make_params(shape, precision=precision, seed=seed, flags=flags, tblock=tblock),
                       torch.cuda.current_stream().cuda_stream)
    prs.prs_init(h)
    return h


class _DeviceBytes:
    """A byte view of device memory for torch (CUDA array interface)."""

    def __init__(self, ptr, nbytes):
        self.__cuda_array_interface__ = {"data": (ptr, False), "shape": (nbytes,), "typestr": "|u1", "version": 3}


@pytest.mark.parametrize("shape,precision", [((256, 64, 16), prs.PRS_FP32), ((512, 96), prs.PRS_FP32),
                                             ((37, 23), prs.PRS_FP64), ((12, 10, 9), prs.PRS_FP32)])
def test_debug_run_matches_a_plain_run(shape, precision):
    dt = np.float32 if precision == prs.PRS_FP32 else np.float64
    res = []
    for flags in (0, prs.PRS_DEBUG):
        h = _raw_run(shape, flags, precision)
        try:
            prs.prs_step(h, 9)
            d = prs.prs_step_measure(h, 4).as_dict()
            phi = np.empty(tuple(reversed(shape)), dt)
            v = np.empty_like(phi)
            assert prs.prs_get_state(h, phi, v) == 13
        finally:
            prs.prs_destroy(h)
        res.append((d, phi, v))
    assert res[0][0] == res[1][0]
    assert np.array_equal(res[0][1], res[1][1]) and np.array_equal(res[0][2], res[1][2])


@pytest.mark.parametrize("which", ["after dphi", "before phi[0]"])
def test_debug_reports_an_overwritten_guard_band(which):
    """Bytes written just past a field (here by the test, from the host side) are reported by
    the next call, which returns PRS_ECUDA naming the band; the context stays usable."""
    import torch

    shape = (256, 64, 16)
    h = _raw_run(shape, prs.PRS_DEBUG)
    try:
        prs.prs_step(h, 2)  # clean so far
        p, v, _ = prs.prs_device_state(h)
        nbytes = 4 * int(np.prod(shape))
        # phi^n is phi[0] after an even number of steps
        target = v + nbytes if which == "after dphi" else p - 16
        torch.as_tensor(_DeviceBytes(target, 16), device="cuda").fill_(0)
        torch.cuda.synchronize()
        assert prs.load().prs_step(h, 1) == prs.PRS_ECUDA
        assert f"guard band {which} overwritten" in prs.prs_last_error()
    finally:
        prs.prs_destroy(h)
    _still_works()


def test_debug_reports_a_nonfinite_state():
    shape = (128, 64)
    phi = (0.5 * np.ones(tuple(reversed(shape)))).astype(np.float32)
    phi[5, 7] = np.inf
    v = np.zeros_like(phi)
    lib = prs.load()
    for flags, expect in ((0, prs.PRS_OK), (prs.PRS_DEBUG, prs.PRS_ENONFINITE)):
        h = prs.prs_create(prs.make_params(shape, flags=flags))
        try:
            rc = lib.prs_set_state(h, phi.ctypes.data_as(ctypes.c_void_p), v.ctypes.data_as(ctypes.c_void_p), 0)
            assert rc == expect
            assert lib.prs_step(h, 3) == expect
        finally:
            prs.prs_destroy(h)
    _still_works()


@pytest.mark.parametrize("tblock", [2, 3])
@pytest.mark.parametrize("shape", [(4096, 40), (512, 96), (256, 64, 24), (128, 32, 8), (128, 32, 40)])
def test_debug_multi_step_passes_stay_in_bounds(shape, tblock):
    """Two- and three-step passes (2D and 3D) under PRS_DEBUG: the guard bands around the fields
    stay intact and the state matches one step per pass to FP32 rounding (7 steps: three pairs or
    two triples, then the single step that brings dphi back to the run's buffer)."""
    out = []
    for flags, tb in ((prs.PRS_DEBUG, tblock), (0, 1)):
        h = _raw_run(shape, flags, tblock=tb)
        try:
            assert prs.load().prs_step(h, 7) == prs.PRS_OK, prs.prs_last_error()
            phi = np.empty(tuple(reversed(shape)), np.float32)
            v = np.empty_like(phi)
            prs.prs_get_state(h, phi, v)
        finally:
            prs.prs_destroy(h)
        out.append((phi, v))
    (pa, va), (pb, vb) = out
    assert np.max(np.abs(pa - pb)) <= 1e-5 * np.max(np.abs(pb))
    assert np.max(np.abs(va - vb)) <= 1e-5 * np.max(np.abs(vb))

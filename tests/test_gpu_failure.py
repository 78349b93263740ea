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

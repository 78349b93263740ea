"""Run state handling through the C ABI: device-side state uploads, and where dphi lives
after two-step passes (Eqs. 3-5 read dphi across sites in a two-step pass, so it goes
out of place).  Fields are compared with the oracle (FP32: 1e-5 relative, as the parity
tests) or bit for bit between two routes to the same state."""
import numpy as np
import pytest

import oracle
import paper_1710_10420_gb300 as prs
import prs_inputs as inp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch

    assert torch.cuda.is_available()
    prs.load(build=True)


def _rel(a, b):
    return float(np.max(np.abs(np.asarray(a, np.float64) - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("precision", [prs.PRS_FP32, prs.PRS_FP64])
def test_set_state_device_matches_host_upload(precision):
    import torch

    shape = (128, 24, 10)
    dt = np.float32 if precision == prs.PRS_FP32 else np.float64
    phi = inp.random_field(shape, 3).astype(dt)
    v = (0.1 * inp.random_field(shape, 4)).astype(dt)
    a = prs.Sim(shape, precision=precision)
    a.set_state(phi, v, 5)
    a.step(7)
    b = prs.Sim(shape, precision=precision)
    prs.prs_set_state_device(b.handle, torch.from_numpy(phi).cuda(), torch.from_numpy(v).cuda(), 5)
    b.step(7)
    pa, va, na = a.get_state()
    pb, vb, nb = b.get_state()
    a.close()
    b.close()
    assert na == nb == 12 and np.array_equal(pa, pb) and np.array_equal(va, vb)


@pytest.mark.parametrize("shape,tblock", [((256, 32, 16), 2), ((4096, 64), 2), ((256, 32, 16), 3),
                                          ((384, 16, 24), 3)])
def test_owned_run_keeps_every_pass(shape, tblock):
    """A run with library-owned buffers stepping by tblock: every call is one multi-step pass and
    the two dphi buffers swap roles after it; the field follows the oracle and prs_device_state
    names the buffer that holds dphi."""
    p = prs.make_params(shape, seed=6, tblock=tblock)
    h = prs.prs_create(p)
    prs.prs_init(h)
    seen = set()
    for _ in range(5):
        prs.prs_step(h, tblock)
        seen.add(prs.prs_device_state(h)[1])
    fshape = tuple(reversed(shape))
    phi = np.empty(fshape, np.float32)
    v = np.empty(fshape, np.float32)
    n = prs.prs_get_state(h, phi, v)
    prs.prs_destroy(h)
    assert n == 5 * tblock and len(seen) == 2  # dphi alternated between the two buffers
    op = oracle.Params(shape)
    ophi, ov = oracle.step(op, *oracle.init_random(op, 6), 5 * tblock)
    assert _rel(phi, ophi) <= 1e-5 and _rel(v, ov) <= 1e-5


@pytest.mark.parametrize("tblock,calls", [(2, (2, 6, 3, 4)), (3, (3, 6, 2, 4, 1, 5, 9))])
def test_bound_run_keeps_dphi_home(tblock, calls):
    """With bound (caller-owned) buffers dphi is in the bound buffer after every call, whatever mix
    of multi-step passes and single steps the call's step count implies."""
    import torch

    shape = (256, 32, 16)
    sim = prs.Sim(shape, seed=6, tblock=tblock)
    sim.init()
    home = sim._bufs[2].data_ptr()
    for k in calls:
        sim.step(k)
        assert prs.prs_device_state(sim.handle)[1] == home
    phi, v, n = sim.get_state()
    sim.close()
    op = oracle.Params(shape)
    ophi, ov = oracle.step(op, *oracle.init_random(op, 6), sum(calls))
    assert n == sum(calls) and _rel(phi, ophi) <= 1e-5 and _rel(v, ov) <= 1e-5
    torch.cuda.synchronize()


def test_stability_checked_at_both_ends():
    """beta > 0: the force grows as a^beta, so a long call fails at its last step even though its
    first step is stable; the call is rejected before any work is queued."""
    shape = (32, 32)
    sim = prs.Sim(shape, precision=prs.PRS_FP64, beta=2.0, era_m=1.0, W0=10.0, deta=0.1)
    sim.init()
    sim.step(10)
    with pytest.raises(prs.PRSError) as e:
        sim.step(100000)
    assert e.value.status == prs.PRS_EINVAL
    assert sim.get_state()[2] == 10
    sim.close()


@pytest.mark.parametrize("owned", [True, False])
def test_default_passes_take_a_triple_for_odd_counts(owned):
    """With the library's choice of steps per pass (two here), an odd step count on a box of the
    three-step pass runs one three-step pass in place of a pair and a single step: library-owned
    buffers keep every multi-step pass (dphi alternates between the two buffers), bound buffers keep
    dphi at home after every call; the field follows one step per pass either way (one step per
    pass follows the oracle in the parity tests; the oracle itself takes close to a minute on a box
    this large)."""
    import torch

    shape = (128, 16, 8200)  # 2^24 sites and more: two steps per pass by default
    calls = (3, 5, 2, 7)
    p = prs.make_params(shape, seed=6)
    assert prs.prs_default_tblock(p) == 2 and prs.prs_max_tblock(p) == 3
    fshape = tuple(reversed(shape))
    if owned:
        h = prs.prs_create(p)
        prs.prs_init(h)
        for k in calls:
            prs.prs_step(h, k)
        phi = np.empty(fshape, np.float32)
        v = np.empty(fshape, np.float32)
        n = prs.prs_get_state(h, phi, v)
        prs.prs_destroy(h)
    else:
        sim = prs.Sim(shape, seed=6)
        sim.init()
        home = sim._bufs[2].data_ptr()
        for k in calls:
            sim.step(k)
            assert prs.prs_device_state(sim.handle)[1] == home
        phi, v, n = sim.get_state()
        sim.close()
    h = prs.prs_create(prs.make_params(shape, seed=6, tblock=1))
    prs.prs_init(h)
    prs.prs_step(h, sum(calls))
    ophi = np.empty(fshape, np.float32)
    ov = np.empty(fshape, np.float32)
    assert prs.prs_get_state(h, ophi, ov) == sum(calls)
    prs.prs_destroy(h)
    ophi, ov = ophi.astype(np.float64), ov.astype(np.float64)
    assert n == sum(calls) and _rel(phi, ophi) <= 1e-5 and _rel(v, ov) <= 1e-5
    torch.cuda.synchronize()

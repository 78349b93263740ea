"""FP32 with correctly rounded division and square root in the wall diagnostics (PRS_FP32_CR).

Sec. III compares single precision with and without correctly rounded divide and
square root.  Here the FP32 leapfrog step has neither operation, so the flag may not
change a field by one bit; it changes only how Eqs. 7 and 8 divide and take roots.

Tolerance: with every operation correctly rounded, each link weight and each Eq. 8
term carries at most about eight FP32 roundings (2^-24 each, about 5e-7 in all)
relative to the FP64 value of the same FP32 inputs, and sums of positive terms keep
that relative bound, so A/V and gamma v must match the oracle to 1e-6 relative.
"""
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


SHAPES = [(128, 128), (512, 32), (128, 64, 40), (256, 32, 16), (37, 23)]


@pytest.mark.parametrize("shape", SHAPES)
def test_flag_leaves_the_fields_unchanged(shape):
    """With one step per pass the two runs execute the same step kernels (the flag only moves
    prs_step_measure's diagnostics into a separate pass), so the fields agree bit for bit."""
    out = []
    for flags in (0, prs.PRS_FP32_CR):
        sim = prs.Sim(shape, precision=prs.PRS_FP32, seed=21, flags=flags, tblock=1)
        sim.init()
        prs.prs_step_measure(sim.handle, 6)
        sim.step(11)
        out.append(sim.get_state())
        sim.close()
    (pa, va, na), (pb, vb, nb) = out
    assert na == nb == 17
    assert np.array_equal(pa, pb) and np.array_equal(va, vb)


@pytest.mark.parametrize("shape", SHAPES)
def test_correctly_rounded_diagnostics_match_the_oracle(shape):
    W0 = 6.0
    fields = [("random", inp.random_field(shape, 41), 0.3 * inp.random_field(shape, 42)),
              ("boosted",) + inp.boosted_kink_pair(shape, W0, 0.4, axis=len(shape) - 1),
              ("bubble",) + inp.bubble(shape, min(shape) / 4, W0)]
    for name, phi, v in fields:
        phi, v = phi.astype(np.float32), v.astype(np.float32)
        sim = prs.Sim(shape, precision=prs.PRS_FP32, W0=W0, flags=prs.PRS_FP32_CR)
        sim.set_state(phi, v, 0)
        d = sim.measure()
        sim.close()
        od = oracle.measure(oracle.Params(shape, W0=W0), phi.astype(np.float64), v.astype(np.float64))
        assert (d["n_links"], d["n_wall"], d["n_vzero"]) == (od.n_links, od.n_wall, od.n_vzero), name
        assert d["area_per_volume"] == pytest.approx(od.area_per_volume, rel=1e-6), name
        assert d["gamma_v"] == pytest.approx(od.gamma_v, rel=1e-6), name


@pytest.mark.parametrize("shape,axis", [((256, 64), 0), ((128, 32, 24), 2), ((37, 23), 1)])
def test_planar_walls_weigh_exactly_one(shape, axis):
    """A wall normal to an axis: the link's own difference g, no transverse part; with
    correctly rounded operations sqrt(g*g)/|g| is exactly 1, so the FP64 sum of weights
    equals the number of crossing links."""
    phi, v = inp.kink_pair(shape, 10.0, axis=axis)
    sim = prs.Sim(shape, precision=prs.PRS_FP32, flags=prs.PRS_FP32_CR)
    sim.set_state(phi.astype(np.float32), v.astype(np.float32), 0)
    d = prs.prs_measure_ex(sim.handle)
    sim.close()
    n_plane = int(np.prod(shape)) // shape[axis]
    assert d.n_links == 2 * n_plane
    assert d.sum_w == float(d.n_links)


def test_step_measure_with_flag_is_measure_then_step():
    shape = (256, 64, 16)
    a = prs.Sim(shape, precision=prs.PRS_FP32, seed=5, flags=prs.PRS_FP32_CR)
    b = prs.Sim(shape, precision=prs.PRS_FP32, seed=5, flags=prs.PRS_FP32_CR)
    a.init().step(4)
    b.init().step(4)
    ref = a.measure()
    a.step(9)
    assert prs.prs_step_measure(b.handle, 9).as_dict() == ref
    pa, va, _ = a.get_state()
    pb, vb, _ = b.get_state()
    a.close()
    b.close()
    assert np.array_equal(pa, pb) and np.array_equal(va, vb)


def test_batch_rejects_the_flag():
    import ctypes

    p = [prs.make_params((256, 64), flags=prs.PRS_FP32_CR)]
    arr = (prs.prs_params * 1)(*p)
    h = ctypes.c_void_p()
    assert prs.load().prs_batch_create(arr, 1, None, ctypes.byref(h)) == prs.PRS_EINVAL

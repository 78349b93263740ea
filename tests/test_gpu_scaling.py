"""Long-run checks: a 3D FP64 run bit-exact with the oracle over hundreds of steps, and the
scaling exponent of the wall density (Eq. 9) against the paper's Table I as a sanity band.

Table I (2048^2, five seeds, points beyond ln(eta) = 2.58): mu = -0.9381 +- 0.0003.  The
paper's initial-condition recipe and seeds are not given, so this is a band (|dmu| < 0.08),
not parity; likewise for 128^3, fitted past the start-up transient of the white-noise field.
"""
import math

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


def test_3d_fp64_long_run_bit_exact():
    """3D 32^3 FP64 PRS, radiation era, 300 steps, diagnostics every 20: fields bit-exact, counts exact."""
    shape = (32, 32, 32)
    p = oracle.Params(shape)
    sim = prs.Sim(shape, precision=prs.PRS_FP64, flags=prs.PRS_REPRO, seed=2)
    sim.init()
    phi, v = oracle.init_random(p, 2)
    n = 0
    while n < 300:
        sim.step(20)
        phi, v = oracle.step(p, phi, v, 20, n0=n)
        n += 20
        d, od = sim.measure(), oracle.measure(p, phi, v)
        assert (d["n_links"], d["n_wall"]) == (od.n_links, od.n_wall)
        assert d["area_per_volume"] == pytest.approx(od.area_per_volume, rel=1e-13)
        assert d["gamma_v"] == pytest.approx(od.gamma_v, rel=1e-12)
    gphi, gv, _ = sim.get_state()
    sim.close()
    assert np.array_equal(gphi, phi) and np.array_equal(gv, v)


def test_2d_density_scaling_exponent_band():
    """Five 2048^2 FP32 radiation-era runs to eta = 1024 on the ensemble engine; rho ~ eta^mu."""
    n, seeds, every = 2048, 5, 10
    nsteps = int(round((n / 2 - 1) / 0.1))
    b = prs.prs_batch_create([prs.make_params((n, n), seed=s) for s in range(1, seeds + 1)])
    out = prs.prs_batch_run(b, [nsteps] * seeds, measure_every=every, out_capacity=nsteps // every + 1)
    prs.prs_batch_destroy(b)
    mus = []
    for r in range(seeds):
        eta = 1.0 + 0.1 * out[r, :, 0]
        m = np.log(eta) > 2.58
        mus.append(np.polyfit(np.log(eta[m]), np.log(out[r, m, 1]), 1)[0])
    mu = float(np.mean(mus))
    assert abs(mu - (-0.9381)) < 0.08, mus
    # the walls are still there and move (gamma v is unbounded: collapsing domains are fast)
    assert np.all(out[:, -1, 3] > 0) and np.all((out[:, -1, 2] > 0.1) & np.isfinite(out[:, -1, 2]))


def test_3d_density_scaling_exponent_band_after_the_transient():
    """Five 128^3 FP32 radiation-era runs to eta = 64 (W0 = 10, white-noise start) on the ensemble
    engine.  The paper does not state its 3D set-up; from this start gamma v first collapses and
    recovers by eta ~ 27, so rho ~ eta^mu is fitted beyond ln(eta) = 3.3 and kept within 0.08 of
    the middle of Table I's 128^3 values (-0.956 FP32, -0.905 FP64): a band, not parity."""
    n, seeds, every = 128, 5, 10
    nsteps = int(round((n / 2 - 1) / 0.1))
    b = prs.prs_batch_create([prs.make_params((n, n, n), seed=s) for s in range(1, seeds + 1)])
    out = prs.prs_batch_run(b, [nsteps] * seeds, measure_every=every, out_capacity=nsteps // every + 1)
    prs.prs_batch_destroy(b)
    mus = []
    for r in range(seeds):
        eta = 1.0 + 0.1 * out[r, :, 0]
        m = np.log(eta) > 3.3
        mus.append(np.polyfit(np.log(eta[m]), np.log(out[r, m, 1]), 1)[0])
    assert abs(float(np.mean(mus)) - (-0.93)) < 0.08, mus


def _series_fp64(shape, seed, nsteps, every):
    sim = prs.Sim(shape, precision=prs.PRS_FP64, seed=seed)
    sim.init()
    rows = []
    for _ in range(nsteps // every + 1):
        d = prs.prs_measure_ex(sim.handle)
        rows.append((d.eta, d.area_per_volume, d.gamma_v))
        if d.step < nsteps:
            sim.step(every)
    sim.close()
    return np.array(rows)


def _slopes(eta, area, gv):
    m = np.log(eta) > 2.58
    return (np.polyfit(np.log(eta[m]), np.log(area[m]), 1)[0], np.polyfit(np.log(eta[m]), np.log(gv[m]), 1)[0])


def test_fp32_and_fp64_runs_give_the_same_exponents():
    """Sec. III, Table I: single and double precision runs from one (FP32-exact) initial field
    give the same scaling exponents.  2D 1024^2, three seeds, eta 1 -> 512, every unit of eta;
    the FP32 runs go through the ensemble engine, the FP64 runs through prs_step/prs_measure."""
    n, seeds, every = 1024, (1, 2, 3), 10
    nsteps = int(round((n / 2 - 1) / 0.1))
    b = prs.prs_batch_create([prs.make_params((n, n), seed=s) for s in seeds])
    out = prs.prs_batch_run(b, [nsteps] * len(seeds), measure_every=every, out_capacity=nsteps // every + 1)
    prs.prs_batch_destroy(b)
    for r, s in enumerate(seeds):
        f64 = _series_fp64((n, n), s, nsteps, every)
        eta32 = 1.0 + 0.1 * out[r, :, 0]
        assert np.allclose(eta32, f64[:, 0], rtol=0, atol=1e-9)
        mu32, nu32 = _slopes(eta32, out[r, :, 1], out[r, :, 2])
        mu64, nu64 = _slopes(*f64.T)
        assert abs(mu32 - mu64) < 1e-3 and abs(nu32 - nu64) < 1e-2, (s, mu32, mu64, nu32, nu64)

"""Parity across parameter space: seeded random boxes and parameters through the C ABI.

* FP64 with PRS_REPRO on random boxes (odd, tiny, non-cubic sides) and random physical and
  lattice parameters (dx, deta, eta0, alpha, beta, the era, W0 including a free field, phi0):
  fields bit-identical to the oracle after the steps, link and wall counts exact, A/V and
  gamma v within 1e-13 (only the order of the FP64 reduction differs).
* FP32 on boxes of the staged kernels, with every steps-per-pass setting: fields within 1e-5
  of the oracle (||d||_inf / ||phi||_inf) and counts of the final state exact.

Draws that would break the leapfrog stability limit at some step, or make delta >= 1, are
drawn again; the library would reject them (test_abi covers that).
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


def _stable(kw, shape, nsteps):
    p = prs.make_params(shape, **kw)
    D = len(shape)
    for n in range(nsteps):
        c = prs.prs_coefficients(p, n)
        lam = 4.0 * D / (kw["dx"] ** 2) + 2.0 * c["cV"] * kw["phi0"] ** 2
        if not (kw["deta"] ** 2 * lam < 3.5 and c["delta"] < 0.9):
            return False
    return True


def _draw_params(rng, shape, nsteps):
    while True:
        kw = dict(dx=float(rng.choice([1.0, 0.7, 1.6])), deta=float(rng.choice([0.05, 0.1, 0.2])),
                  eta0=float(rng.choice([1.0, 1.5, 3.0])), alpha=float(rng.choice([3.0, 2.0, 0.5])),
                  beta=float(rng.choice([0.0, 0.0, 2.0])), era_m=float(rng.choice([1.0, 2.0])),
                  W0=float(rng.choice([5.0, 10.0, math.inf])), phi0=float(rng.choice([1.0, 0.7, 1.3])))
        if _stable(kw, shape, nsteps):
            return kw


def _fp64_cases(n=24, seed=2024):
    rng = np.random.Generator(np.random.PCG64(seed))
    cases = []
    for k in range(n):
        if k % 2:
            shape = tuple(int(v) for v in rng.integers(3, 15, size=3))
        else:
            shape = tuple(int(v) for v in rng.integers(3, 49, size=2))
        nsteps = int(rng.integers(1, 13))
        cases.append((shape, nsteps, _draw_params(rng, shape, nsteps), int(rng.integers(0, 2 ** 32))))
    return cases


def _fp32_cases(n=24, seed=7):
    rng = np.random.Generator(np.random.PCG64(seed))
    cases = []
    for k in range(n):
        if k % 2:
            nx = int(rng.choice([128, 256, 512]))
            ty = 4096 // nx
            shape = (nx, ty * int(rng.integers(1, 4)), int(rng.integers(3, 12)))
        else:
            nx = int(rng.choice([128, 256, 512, 1024]))
            rb = 4096 // nx
            shape = (nx, rb * int(rng.integers(1, 5)))
        nsteps = int(rng.integers(1, 13))
        tblock = int(rng.choice([0, 1, 2]))
        cases.append((shape, nsteps, tblock, _draw_params(rng, shape, nsteps), int(rng.integers(0, 2 ** 32))))
    return cases


FP64_CASES = _fp64_cases()
FP32_CASES = _fp32_cases()


@pytest.mark.parametrize("case", range(len(FP64_CASES)))
def test_fp64_repro_random_parameters(case):
    shape, nsteps, kw, seed = FP64_CASES[case]
    p = oracle.Params(shape, **kw)
    sim = prs.Sim(shape, precision=prs.PRS_FP64, flags=prs.PRS_REPRO, seed=seed, **kw)
    sim.init()
    sim.step(nsteps)
    phi, v, n = sim.get_state()
    d = sim.measure()
    sim.close()
    ophi, ov = oracle.step(p, *oracle.init_random(p, seed), nsteps)
    assert n == nsteps
    assert np.array_equal(phi, ophi) and np.array_equal(v, ov), (shape, kw)
    od = oracle.measure(p, ophi, ov)
    assert (d["n_links"], d["n_wall"], d["n_vzero"]) == (od.n_links, od.n_wall, od.n_vzero), (shape, kw)
    assert d["area_per_volume"] == pytest.approx(od.area_per_volume, rel=1e-13, abs=1e-300)
    assert d["gamma_v"] == pytest.approx(od.gamma_v, rel=1e-13, abs=1e-300)


@pytest.mark.parametrize("case", range(len(FP32_CASES)))
def test_fp32_staged_random_parameters(case):
    shape, nsteps, tblock, kw, seed = FP32_CASES[case]
    p = oracle.Params(shape, **kw)
    sim = prs.Sim(shape, precision=prs.PRS_FP32, seed=seed, tblock=tblock, **kw)
    sim.init()
    sim.step(nsteps)
    phi, v, n = sim.get_state()
    d = sim.measure()
    sim.close()
    ophi, ov = oracle.step(p, *oracle.init_random(p, seed), nsteps)
    assert n == nsteps
    scale = np.max(np.abs(ophi))
    assert np.max(np.abs(phi - ophi)) <= 1e-5 * scale, (shape, tblock, kw)
    assert np.max(np.abs(v - ov)) <= 1e-5 * max(np.max(np.abs(ov)), 1e-30) + 1e-6 * scale, (shape, tblock, kw)
    # the diagnostics of the GPU's own FP32 field, against the oracle on that field
    od = oracle.measure(p, phi.astype(np.float64), v.astype(np.float64))
    assert (d["n_links"], d["n_wall"]) == (od.n_links, od.n_wall), (shape, tblock, kw)
    assert d["area_per_volume"] == pytest.approx(od.area_per_volume, rel=1e-5)

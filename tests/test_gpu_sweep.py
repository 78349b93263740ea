"""Parity across parameter space: seeded random boxes and parameters through the C ABI.

* FP64 with PRS_REPRO on random boxes (odd, tiny, non-cubic sides) and random physical and
  lattice parameters (dx, deta, eta0, alpha, beta, the era, W0 including a free field, phi0):
  fields bit-identical to the oracle after the steps, link and wall counts exact, A/V and
  gamma v within 1e-13 (only the order of the FP64 reduction differs).
* FP32 on boxes of the staged kernels, with every steps-per-pass setting: fields within 1e-5
  of the oracle (||d||_inf / ||phi||_inf) and counts of the final state exact.
* FP64 adjoint gradients and FP32 ensembles on the persistent engine, the same way.

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
        tblock = int(rng.choice([0, 1, 2, 3]))
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


# ------------------------------------------------------------ adjoint and ensembles

def _adjoint_cases(n=10, seed=99):
    rng = np.random.Generator(np.random.PCG64(seed))
    cases = []
    for k in range(n):
        shape = tuple(int(v) for v in rng.integers(3, 12, size=3)) if k % 2 else \
            tuple(int(v) for v in rng.integers(4, 33, size=2))
        nsteps = int(rng.integers(2, 16))
        kw = _draw_params(rng, shape, nsteps)
        while kw["W0"] == math.inf:  # the observables need walls to matter
            kw = _draw_params(rng, shape, nsteps)
        obs = int(rng.integers(0, 2))
        K = int(rng.choice([0, 1, 3, 5, 64]))
        cases.append((shape, nsteps, kw, obs, K, float(rng.choice([0.2, 0.5]))))
    return cases


ADJ_CASES = _adjoint_cases()


@pytest.mark.parametrize("case", range(len(ADJ_CASES)))
def test_fp64_adjoint_random_parameters(case):
    """prs_adjoint in FP64 against the oracle's adjoint: J to 1e-12, dJ/dphi, dJ/d(dphi) and
    dJ/dalpha to 1e-10, for random parameters, observables and checkpoint intervals."""
    import torch

    shape, nsteps, kw, obs, K, eps = ADJ_CASES[case]
    p = oracle.Params(shape, **kw)
    rng = np.random.Generator(np.random.PCG64(case))
    phi0 = rng.uniform(-1.0, 1.0, tuple(reversed(shape))) * kw["phi0"]
    v0 = 0.05 * rng.uniform(-1.0, 1.0, phi0.shape)
    ref = oracle.adjoint(p, phi0, v0, nsteps, obs, eps)
    sim = prs.Sim(shape, precision=prs.PRS_FP64, **kw)
    sim.set_state(phi0, v0, 0)
    gphi = torch.empty(phi0.shape, dtype=torch.float64, device="cuda")
    gv = torch.empty_like(gphi)
    J, dA = prs.prs_adjoint(sim.handle, nsteps, obs, eps, K, gphi, gv)
    sim.close()

    def rel(a, b):
        return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))

    assert J == pytest.approx(ref["J"], rel=1e-12), (shape, kw, obs, K)
    assert rel(gphi.cpu().numpy(), ref["dJ_dphi"]) <= 1e-10, (shape, kw, obs, K)
    assert rel(gv.cpu().numpy(), ref["dJ_dv"]) <= 1e-10, (shape, kw, obs, K)
    assert dA == pytest.approx(ref["dJ_dalpha"], rel=1e-10, abs=1e-14 * abs(J)), (shape, kw, obs, K)


def _batch_cases(n=4, seed=5):
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(n):
        runs = []
        for r in range(int(rng.integers(2, 6))):
            if rng.integers(0, 2):
                nx = int(rng.choice([128, 256]))
                shape = (nx, (4096 // nx) * int(rng.integers(1, 3)), int(rng.integers(3, 9)))
            else:
                nx = int(rng.choice([128, 256, 512, 1024]))
                shape = (nx, (4096 // nx) * int(rng.integers(1, 4)))
            nsteps = int(rng.integers(0, 14))
            kw = _draw_params(rng, shape, max(nsteps, 1))
            runs.append((shape, nsteps, kw, int(rng.integers(0, 2 ** 32))))
        out.append(runs)
    return out


BATCH_CASES = _batch_cases()


@pytest.mark.parametrize("case", range(len(BATCH_CASES)))
def test_fp32_ensembles_random_parameters(case):
    """Random mixed ensembles (2D/3D, own parameters, seeds and step counts) on the persistent
    engine: every run's field within 1e-5 of the oracle; the output at step 0 has the oracle's
    link count exactly."""
    runs = BATCH_CASES[case]
    b = prs.prs_batch_create([prs.make_params(s, seed=sd, **kw) for s, _, kw, sd in runs])
    try:
        out = prs.prs_batch_run(b, [n for _, n, _, _ in runs], measure_every=4, out_capacity=5)
        for r, (shape, nsteps, kw, sd) in enumerate(runs):
            phi = np.empty(tuple(reversed(shape)), np.float32)
            assert prs.prs_batch_get_state(b, r, phi, None) == nsteps
            p = oracle.Params(shape, **kw)
            phi0, v0 = oracle.init_random(p, sd)
            assert out[r, 0, 3] == oracle.measure(p, phi0, v0).n_links
            ophi, _ = oracle.step(p, phi0, v0, nsteps)
            assert np.max(np.abs(phi - ophi)) <= 1e-5 * np.max(np.abs(ophi)), (shape, nsteps, kw)
    finally:
        prs.prs_batch_destroy(b)

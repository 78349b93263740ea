"""GPU reverse-time adjoint (prs_adjoint) against the oracle's adjoint and finite differences.

Tolerances: FP64 gradients within 1e-10 of the oracle (relative to the largest
component), FP32 within 1e-5; J to 1e-12 (FP64); dJ/dalpha as the gradients.
"""
import math

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
    a = np.asarray(a, np.float64)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _gpu_adjoint(shape, precision, phi0, v0, nsteps, obs, K, eps=0.1, **kw):
    import torch

    sim = prs.Sim(shape, precision=precision, **kw)
    sim.set_state(phi0, v0, 0)
    dt = torch.float32 if precision == prs.PRS_FP32 else torch.float64
    gphi = torch.empty(tuple(reversed(shape)), dtype=dt, device="cuda")
    gv = torch.empty_like(gphi)
    J, dA = prs.prs_adjoint(sim.handle, nsteps, obs, eps, K, gphi, gv)
    end_phi, end_v, n = sim.get_state()
    sim.close()
    return J, dA, gphi.cpu().numpy(), gv.cpu().numpy(), end_phi, n


CASES = [((16, 12), 0, 30, 7), ((16, 12), 1, 25, 4), ((8, 6, 5), 0, 20, 6), ((8, 6, 5), 1, 20, 20),
         ((128, 32), 0, 24, 5), ((128, 16, 8), 1, 16, 3)]


@pytest.mark.parametrize("shape,obs,nsteps,K", CASES)
def test_fp64_adjoint_matches_oracle(shape, obs, nsteps, K):
    p = oracle.Params(shape, W0=4.0, eta0=2.0)
    phi0 = 0.8 * inp.random_field(shape, seed=11)
    v0 = 0.05 * inp.random_field(shape, seed=12)
    ref = oracle.adjoint(p, phi0, v0, nsteps, obs)
    J, dA, gphi, gv, end_phi, n = _gpu_adjoint(shape, prs.PRS_FP64, phi0, v0, nsteps, obs, K, W0=4.0, eta0=2.0)
    assert n == nsteps
    assert J == pytest.approx(ref["J"], rel=1e-12)
    assert _rel(gphi, ref["dJ_dphi"]) <= 1e-10
    assert _rel(gv, ref["dJ_dv"]) <= 1e-10
    assert dA == pytest.approx(ref["dJ_dalpha"], rel=1e-10)
    # the run ends where a plain forward run ends
    ophi, _ = oracle.step(p, phi0, v0, nsteps)
    assert _rel(end_phi, ophi) <= 1e-12


@pytest.mark.parametrize("K", [8, 0])
@pytest.mark.parametrize("shape,obs", [((128, 64), 0), ((64, 32, 16), 0), ((128, 32, 8), 1), ((37, 29), 1),
                                       ((256, 16, 12), 0), ((512, 40), 1)])
def test_fp32_adjoint_matches_oracle(shape, obs, K):
    nsteps = 20
    p = oracle.Params(shape, W0=6.0, eta0=2.0)
    phi0 = (0.8 * inp.random_field(shape, seed=1)).astype(np.float32)
    v0 = (0.05 * inp.random_field(shape, seed=2)).astype(np.float32)
    ref = oracle.adjoint(p, phi0.astype(np.float64), v0.astype(np.float64), nsteps, obs, eps=0.3)
    J, dA, gphi, gv, _, _ = _gpu_adjoint(shape, prs.PRS_FP32, phi0, v0, nsteps, obs, K, eps=0.3, W0=6.0, eta0=2.0)
    assert J == pytest.approx(ref["J"], rel=1e-5)
    assert _rel(gphi, ref["dJ_dphi"]) <= 1e-5
    assert _rel(gv, ref["dJ_dv"]) <= 1e-5
    assert dA == pytest.approx(ref["dJ_dalpha"], rel=1e-5)


@pytest.mark.parametrize("K", [8, 5, 0])
def test_fp32_adjoint_on_a_tensor_copy_box(K):
    """512-wide 3D rows: the forward and the stored or recomputed states go through the two-step
    pass with tensor copies, its variant that also stores the state between the two steps."""
    shape, nsteps = (512, 16, 8), 22
    p = oracle.Params(shape, W0=6.0, eta0=2.0)
    phi0 = (0.8 * inp.random_field(shape, seed=31)).astype(np.float32)
    v0 = (0.05 * inp.random_field(shape, seed=32)).astype(np.float32)
    ref = oracle.adjoint(p, phi0.astype(np.float64), v0.astype(np.float64), nsteps, 1, eps=0.1)
    J, dA, gphi, gv, end_phi, n = _gpu_adjoint(shape, prs.PRS_FP32, phi0, v0, nsteps, 1, K, eps=0.1, W0=6.0,
                                                eta0=2.0)
    assert n == nsteps
    assert J == pytest.approx(ref["J"], rel=1e-5)
    assert _rel(gphi, ref["dJ_dphi"]) <= 1e-5 and _rel(gv, ref["dJ_dv"]) <= 1e-5
    assert dA == pytest.approx(ref["dJ_dalpha"], rel=1e-5)
    ophi, _ = oracle.step(p, phi0.astype(np.float64), v0.astype(np.float64), nsteps)
    assert _rel(end_phi, ophi) <= 1e-5


@pytest.mark.parametrize("K", [8, 0])
@pytest.mark.parametrize("shape", [(128, 32, 8), (256, 16, 12), (256, 64)])
def test_fp32_adjoint_configured_smoothing(shape, K):
    """The configured observable, the tanh(phi/0.1)-smoothed wall area, in FP32 on boxes of the
    staged (TMA) kernels, against the FP64 oracle's gradient: 1e-5 as for the other FP32 cases."""
    nsteps = 24
    p = oracle.Params(shape, W0=6.0, eta0=2.0)
    phi0 = (0.8 * inp.random_field(shape, seed=21)).astype(np.float32)
    v0 = (0.05 * inp.random_field(shape, seed=22)).astype(np.float32)
    ref = oracle.adjoint(p, phi0.astype(np.float64), v0.astype(np.float64), nsteps, 1, eps=0.1)
    J, dA, gphi, gv, _, _ = _gpu_adjoint(shape, prs.PRS_FP32, phi0, v0, nsteps, 1, K, eps=0.1, W0=6.0, eta0=2.0)
    assert J == pytest.approx(ref["J"], rel=1e-5)
    assert _rel(gphi, ref["dJ_dphi"]) <= 1e-5
    assert _rel(gv, ref["dJ_dv"]) <= 1e-5
    assert dA == pytest.approx(ref["dJ_dalpha"], rel=1e-5)


def test_checkpoint_interval_does_not_change_the_gradient():
    """Recomputed segments replay the same kernels: every checkpoint interval gives identical bits."""
    shape = (24, 20, 12)
    phi0 = inp.random_field(shape, seed=5)
    v0 = np.zeros_like(phi0)
    # K = 0: every state kept, no recomputation
    outs = [_gpu_adjoint(shape, prs.PRS_FP64, phi0, v0, 23, 0, K, flags=prs.PRS_REPRO) for K in (1, 5, 23, 64, 0)]
    for o in outs[1:]:
        assert o[0] == outs[0][0] and o[1] == outs[0][1]
        assert np.array_equal(o[2], outs[0][2]) and np.array_equal(o[3], outs[0][3])


def test_central_differences_32cubed_fp64():
    """dJ/dphi_init along random directions and dJ/dalpha vs central differences (eps = 1e-3, FP64, 32^3)."""
    import torch

    shape = (32, 32, 32)
    nsteps = 60
    kw = dict(W0=10.0)
    phi0 = inp.random_field(shape, seed=8)
    v0 = np.zeros_like(phi0)

    def J_of(ph, alpha=3.0):
        sim = prs.Sim(shape, precision=prs.PRS_FP64, alpha=alpha, **kw)
        sim.set_state(ph, v0, 0)
        sim.step(nsteps)
        J = prs.prs_observable(sim.handle, prs.PRS_OBS_GRAD_ENERGY)
        sim.close()
        return J

    J, dA, gphi, gv, _, _ = _gpu_adjoint(shape, prs.PRS_FP64, phi0, v0, nsteps, 0, 16, **kw)
    assert J == pytest.approx(J_of(phi0), rel=1e-14)
    rng = np.random.Generator(np.random.PCG64(3))
    h = 1e-3
    for _ in range(4):
        d = rng.standard_normal(phi0.shape)
        fd = (J_of(phi0 + h * d) - J_of(phi0 - h * d)) / (2 * h)
        assert float(np.sum(gphi * d)) == pytest.approx(fd, rel=1e-6)
    fda = (J_of(phi0, 3.0 + h) - J_of(phi0, 3.0 - h)) / (2 * h)
    assert dA == pytest.approx(fda, rel=1e-6)


def test_autograd_function():
    import torch

    shape = (16, 12)
    phi0 = torch.tensor(0.7 * inp.random_field(shape, seed=2), dtype=torch.float64, device="cuda",
                        requires_grad=True)
    v0 = torch.zeros_like(phi0, requires_grad=True)
    alpha = torch.tensor(3.0, dtype=torch.float64, requires_grad=True)
    J = prs.observable_with_grad(shape, phi0, v0, 15, prs.PRS_OBS_SMOOTH_AREA, 0.2, 4, precision=prs.PRS_FP64,
                                 alpha_tensor=alpha, W0=5.0)
    (2.0 * J).backward()
    ref = oracle.adjoint(oracle.Params(shape, W0=5.0), phi0.detach().cpu().numpy(), np.zeros(phi0.shape), 15, 1,
                         eps=0.2)
    assert float(J.detach()) == pytest.approx(ref["J"], rel=1e-12)
    assert _rel(phi0.grad.cpu().numpy(), 2.0 * ref["dJ_dphi"]) <= 1e-10
    assert _rel(v0.grad.cpu().numpy(), 2.0 * ref["dJ_dv"]) <= 1e-10
    assert float(alpha.grad) == pytest.approx(2.0 * ref["dJ_dalpha"], rel=1e-10)


def test_adjoint_timing_reports_the_phases():
    """prs_adjoint_timing: the forward, recomputation and reverse-sweep times of the last call, from
    events on the run's stream; no recomputation when every state is kept."""
    import time

    shape = (128, 32, 16)
    sim = prs.Sim(shape, precision=prs.PRS_FP32, seed=3)
    sim.init()
    with pytest.raises(prs.PRSError) as e:
        prs.prs_adjoint_timing(sim.handle)
    assert e.value.status == prs.PRS_ESTATE
    t0 = time.perf_counter()
    prs.prs_adjoint(sim.handle, 40, prs.PRS_OBS_GRAD_ENERGY, 0.1, 8, None, None)
    wall = (time.perf_counter() - t0) * 1e3
    t = prs.prs_adjoint_timing(sim.handle)
    assert t["forward_ms"] > 0 and t["recompute_ms"] > 0 and t["reverse_ms"] > 0
    assert t["forward_ms"] + t["recompute_ms"] + t["reverse_ms"] <= wall
    sim.init()
    prs.prs_adjoint(sim.handle, 40, prs.PRS_OBS_GRAD_ENERGY, 0.1, 0, None, None)
    t = prs.prs_adjoint_timing(sim.handle)
    assert t["recompute_ms"] < 0.05 * t["reverse_ms"]  # events only: nothing is recomputed
    sim.close()

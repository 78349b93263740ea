"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (written in each test):
  * FP64 with PRS_REPRO: fields bit-identical to the oracle; link and wall counts exact;
    A/V and gamma v within 1e-13 relative (only the order of the FP64 reduction differs).
  * FP64 without PRS_REPRO (fused multiply-add allowed): fields within 1e-12 relative
    after 20 steps.
  * FP32: fields within 1e-5 relative (||d||_inf / ||phi||_inf) after 20 steps.  On one
    given FP32 field the counts are exact and A/V, gamma v agree to 1e-5 (each site
    weight is a few float roundings; the sums are FP64).
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
    yield
    torch.cuda.synchronize()


def _rel(a, b):
    return float(np.max(np.abs(np.asarray(a, np.float64) - b)) / max(np.max(np.abs(b)), 1e-300))


def _run(shape, precision, nsteps, phi0=None, v0=None, **kw):
    sim = prs.Sim(shape, precision=precision, **kw)
    sim.init(phi0, v0)
    sim.step(nsteps)
    phi, v, n = sim.get_state()
    sim.close()
    assert n == nsteps
    return phi, v


# ------------------------------------------------------------------ init

@pytest.mark.parametrize("precision", [prs.PRS_FP32, prs.PRS_FP64])
@pytest.mark.parametrize("shape", [(17, 19), (8, 6, 5), (128, 128)])
def test_random_initial_field_bit_exact(precision, shape):
    sim = prs.Sim(shape, precision=precision, seed=12345)
    sim.init()
    phi, v, n = sim.get_state()
    sim.close()
    ophi, ov = oracle.init_random(oracle.Params(shape), 12345)
    assert n == 0
    assert np.array_equal(phi.astype(np.float64), ophi) and np.all(v == 0)


# ----------------------------------------------------------------- steps

REPRO_CASES = [((128, 128), 20), ((17, 19), 25), ((3, 3), 7), ((32, 32, 32), 20), ((9, 7, 5), 15), ((36, 4, 3), 9),
               ((130, 66), 11)]


@pytest.mark.parametrize("shape,nsteps", REPRO_CASES)
def test_fp64_repro_bit_exact(shape, nsteps):
    p = oracle.Params(shape, W0=6.0)
    ophi, ov = oracle.init_random(p, 3)
    ov = 0.2 * inp.random_field(shape, seed=4)
    phi, v = _run(shape, prs.PRS_FP64, nsteps, ophi, ov, W0=6.0, flags=prs.PRS_REPRO)
    ophi, ov = oracle.step(p, ophi, ov, nsteps)
    assert np.array_equal(phi, ophi)
    assert np.array_equal(v, ov)


def test_config_128sq_fp64_full_run():
    """2D 128^2, FP64, PRS radiation era, eta 1 -> 64 (630 steps), diagnostics every 10 steps."""
    shape = (128, 128)
    p = oracle.Params(shape)
    sim = prs.Sim(shape, precision=prs.PRS_FP64, flags=prs.PRS_REPRO, seed=0)
    sim.init()
    phi, v = oracle.init_random(p, 0)
    n = 0
    while n < 630:
        d = sim.measure()
        od = oracle.measure(p, phi, v)
        assert d["step"] == n
        assert (d["n_links"], d["n_wall"], d["n_vzero"]) == (od.n_links, od.n_wall, od.n_vzero)
        assert d["area_per_volume"] == pytest.approx(od.area_per_volume, rel=1e-13)
        assert d["gamma_v"] == pytest.approx(od.gamma_v, rel=1e-13, abs=1e-300)
        k = 10
        sim.step(k)
        phi, v = oracle.step(p, phi, v, k, n0=n)
        n += k
    gphi, gv, gn = sim.get_state()
    sim.close()
    assert gn == 630 and np.array_equal(gphi, phi) and np.array_equal(gv, v)


@pytest.mark.parametrize("shape", [(64, 64), (33, 31), (16, 16, 16), (12, 10, 14)])
def test_fp64_fma_close(shape):
    p = oracle.Params(shape, era_m=2.0)
    ophi, ov = oracle.init_random(p, 9)
    phi, v = _run(shape, prs.PRS_FP64, 20, ophi, ov, era_m=2.0)
    ophi, ov = oracle.step(p, ophi, ov, 20)
    assert _rel(phi, ophi) <= 1e-12
    assert _rel(v, ov) <= 1e-12


# generic kernel: x side not a multiple of 128 (or too few rows for a tile)
# fast kernel: x side a multiple of 128; 3D tiles of 4096/nx rows, 2D bands of 4096/nx rows
FP32_CASES = [(130, 66), (17, 19), (64, 64, 64), (32, 16, 24), (20, 12, 9), (128, 8, 8),
              (128, 128), (256, 64), (4096, 6), (2048, 40), (1024, 12),
              (128, 64, 40), (256, 32, 20), (512, 16, 24), (1024, 8, 10), (128, 32, 3), (256, 16, 17)]


@pytest.mark.parametrize("shape", FP32_CASES)
@pytest.mark.parametrize("era_m", [1.0, 2.0])
def test_fp32_close(shape, era_m):
    p = oracle.Params(shape, era_m=era_m)
    ophi, ov = oracle.init_random(p, 21)
    phi, v = _run(shape, prs.PRS_FP32, 20, None, None, era_m=era_m, seed=21)
    ophi, ov = oracle.step(p, ophi, ov, 20)
    assert _rel(phi, ophi) <= 1e-5
    assert _rel(v, ov) <= 1e-5


@pytest.mark.parametrize("nsteps", [23, 8, 6, 3, 2, 1])
@pytest.mark.parametrize("tblock", [0, 1, 2, 3])
@pytest.mark.parametrize("shape", [(256, 256), (64, 48, 40), (128, 64, 40), (256, 32, 24), (512, 16, 12),
                                   (1024, 8, 10), (128, 32, 3), (256, 48, 7), (384, 12, 7), (256, 7, 4),
                                   (640, 8, 6), (768, 10, 5), (2048, 6, 3),
                                   (512, 96), (4096, 12), (1024, 5), (2048, 40), (128, 3)])
def test_fp32_temporal_blocks(shape, tblock, nsteps):
    """Every fused-steps-per-pass setting (0: the library's choice, which mixes passes of two and
    three steps; the mix of multi-step and single steps each count implies) gives the oracle's
    field to FP32 rounding; dphi always ends in the run's own buffer."""
    p = oracle.Params(shape)
    ophi, ov = oracle.init_random(p, 5)
    phi, v = _run(shape, prs.PRS_FP32, nsteps, None, None, seed=5, tblock=tblock)
    ophi, ov = oracle.step(p, ophi, ov, nsteps)
    assert _rel(phi, ophi) <= 1e-5 and _rel(v, ov) <= 1e-5


@pytest.mark.parametrize("nsteps", [2, 7, 12])
@pytest.mark.parametrize("shape", [(512, 16, 12), (768, 24, 9), (1280, 16, 5), (512, 32, 3), (1024, 40, 17)])
def test_tensor_copy_two_step_pass(shape, nsteps):
    """The two-step pass with TMA tensor copies (x sides multiples of 256, at least 512; y sides
    multiples of 8, at least 16): x tiles at both periodic ends and inside, both y-wrapping tiles
    (ny = 16: every tile wraps), the minimal z side, uneven z chunks; fields to 1e-5 of the oracle."""
    p = oracle.Params(shape)
    ophi, ov = oracle.init_random(p, 21)
    ov = 0.1 * inp.random_field(shape, 22)
    phi, v = _run(shape, prs.PRS_FP32, nsteps, ophi.astype(np.float32), ov.astype(np.float32), seed=21, tblock=2)
    ophi, ov = oracle.step(p, ophi, ov, nsteps)
    assert _rel(phi, ophi) <= 1e-5 and _rel(v, ov) <= 1e-5


@pytest.mark.parametrize("nsteps", [4, 7, 11])
@pytest.mark.parametrize("shape", [(128, 16, 12), (384, 24, 9), (128, 16, 48), (512, 32, 3), (768, 16, 40),
                                   (1024, 24, 7), (256, 48, 30)])
def test_tensor_copy_three_step_pass(shape, nsteps):
    """The three-step pass (x sides multiples of 128: 128-column tiles where 256 does not divide the
    side, 256-column tiles where it does; y sides multiples of 8, at least 16): both y-wrapping
    tiles (ny = 16: every tile wraps), x tiles at both periodic ends and inside, a whole 128- or
    256-wide row as one tile, the minimal z side, several and uneven z chunks; passes of three
    steps followed by a single step (4, 7) or a pair (11); fields to 1e-5 of the oracle."""
    p = oracle.Params(shape)
    ophi, ov = oracle.init_random(p, 31)
    ov = 0.1 * inp.random_field(shape, 32)
    phi, v = _run(shape, prs.PRS_FP32, nsteps, ophi.astype(np.float32), ov.astype(np.float32), seed=31, tblock=3)
    ophi, ov = oracle.step(p, ophi, ov, nsteps)
    assert _rel(phi, ophi) <= 1e-5 and _rel(v, ov) <= 1e-5


@pytest.mark.parametrize("tblock", [2, 3])
@pytest.mark.parametrize("shape", [(256, 64, 48), (1024, 32, 24), (384, 40, 36)])
def test_multi_step_passes_match_single_steps(shape, tblock):
    """Two- and three-step passes agree with one-step passes to FP32 rounding over many passes (3D:
    whole rows, rows in 256- and 128-column tiles)."""
    a = _run(shape, prs.PRS_FP32, 40, None, None, seed=3, tblock=1)
    b = _run(shape, prs.PRS_FP32, 40, None, None, seed=3, tblock=tblock)
    assert _rel(b[0], a[0].astype(np.float64)) <= 1e-5 and _rel(b[1], a[1].astype(np.float64)) <= 1e-5


def test_zero_steps_and_resume_bit_exact():
    shape = (48, 40, 8)
    sim = prs.Sim(shape, precision=prs.PRS_FP32, seed=2)
    sim.init()
    sim.step(0)
    a_phi, a_v, n = sim.get_state()
    assert n == 0
    sim.step(7)
    mid_phi, mid_v, n = sim.get_state()
    sim.step(6)
    end_phi, end_v, n = sim.get_state()
    assert n == 13
    # restart from the checkpoint at step 7 in a fresh run
    sim2 = prs.Sim(shape, precision=prs.PRS_FP32, seed=99)
    sim2.set_state(mid_phi, mid_v, 7)
    sim2.step(6)
    r_phi, r_v, n2 = sim2.get_state()
    assert n2 == 13 and np.array_equal(r_phi, end_phi) and np.array_equal(r_v, end_v)
    sim.close()
    sim2.close()


def test_library_owned_buffers():
    """Without prs_bind the library allocates the fields itself."""
    shape = (32, 24)
    p = prs.make_params(shape, precision=prs.PRS_FP64, flags=prs.PRS_REPRO, seed=1)
    h = prs.prs_create(p)
    prs.prs_init(h)
    prs.prs_step(h, 5)
    phi = np.empty((24, 32))
    v = np.empty((24, 32))
    assert prs.prs_get_state(h, phi, v) == 5
    a, g, nl, nw = prs.prs_measure(h)
    prs.prs_destroy(h)
    op = oracle.Params(shape)
    ophi, ov = oracle.step(op, *oracle.init_random(op, 1), 5)
    assert np.array_equal(phi, ophi)
    od = oracle.measure(op, ophi, ov)
    assert (nl, nw) == (od.n_links, od.n_wall)


# ------------------------------------------------------------ diagnostics

def _fields(shape):
    yield "random", inp.random_field(shape, 31), 0.3 * inp.random_field(shape, 32)
    W0 = 6.0
    phi, v = inp.boosted_kink_pair(shape, W0, 0.4, axis=len(shape) - 1)
    yield "boosted", phi, v
    if shape[0] == shape[1]:
        phi, v = inp.tilted_wall_pair(shape, W0)
        yield "tilted", phi, v + 0.01
    phi, v = inp.bubble(shape, min(shape) / 4, W0)
    yield "bubble", phi, v - 0.02


MEASURE_SHAPES = [(64, 64), (37, 23), (24, 24, 24), (13, 11, 40),  # generic kernel
                  (128, 128), (512, 32), (4096, 8), (128, 64, 40), (256, 32, 16), (1024, 8, 6)]  # fast (FP32)


@pytest.mark.parametrize("precision", [prs.PRS_FP32, prs.PRS_FP64])
@pytest.mark.parametrize("shape", MEASURE_SHAPES)
def test_measure_parity(precision, shape):
    for name, phi, v in _fields(shape):
        np_dtype = np.float32 if precision == prs.PRS_FP32 else np.float64
        phi = phi.astype(np_dtype)
        v = v.astype(np_dtype)
        sim = prs.Sim(shape, precision=precision, W0=6.0)
        sim.set_state(phi, v, 0)
        d = sim.measure()
        sim.close()
        od = oracle.measure(oracle.Params(shape, W0=6.0), phi.astype(np.float64), v.astype(np.float64))
        assert (d["n_links"], d["n_wall"], d["n_vzero"], d["n_nonfinite"]) == \
            (od.n_links, od.n_wall, od.n_vzero, od.n_nonfinite), name
        tol = 1e-13 if precision == prs.PRS_FP64 else 1e-5
        assert d["area_per_volume"] == pytest.approx(od.area_per_volume, rel=tol), name
        assert d["gamma_v"] == pytest.approx(od.gamma_v, rel=tol), name


@pytest.mark.parametrize("shape", [(128, 64), (37, 23), (128, 32, 8), (13, 11, 9)])
def test_measure_tiny_magnitudes(shape):
    """Fields of size 1e-25 (normal FP32 numbers whose squares underflow) keep their weights."""
    phi = (1e-25 * inp.random_signs(shape, seed=4)).astype(np.float32)
    v = np.zeros_like(phi)
    sim = prs.Sim(shape, precision=prs.PRS_FP32)
    sim.set_state(phi, v, 0)
    d = sim.measure()
    sim.close()
    od = oracle.measure(oracle.Params(shape), phi.astype(np.float64), v.astype(np.float64))
    assert d["n_links"] == od.n_links and d["n_wall"] == od.n_wall
    assert d["area_per_volume"] == pytest.approx(od.area_per_volume, rel=1e-5)


@pytest.mark.parametrize("precision,shape", [(prs.PRS_FP32, (256, 64, 40)), (prs.PRS_FP32, (512, 96)),
                                             (prs.PRS_FP32, (1024, 16, 12)), (prs.PRS_FP32, (37, 23)),
                                             (prs.PRS_FP64, (32, 24, 16))])
def test_step_measure_fused(precision, shape):
    """prs_step_measure = prs_measure_ex of the start state, then prs_step: same numbers, same field
    (1024-wide 3D rows: the fused pass's instantiation for that width)."""
    a = prs.Sim(shape, precision=precision, seed=9)
    b = prs.Sim(shape, precision=precision, seed=9)
    a.init().step(7)
    b.init().step(7)
    ref = a.measure()
    a.step(13)
    d = prs.prs_step_measure(b.handle, 13).as_dict()
    assert d == ref
    pa, va, na = a.get_state()
    pb, vb, nb = b.get_state()
    a.close()
    b.close()
    assert na == nb == 20
    # the fused kernel evaluates the same expressions, but the compiler may contract
    # a*b+c into a fused multiply-add differently there: FP32-rounding agreement
    assert _rel(pb, pa.astype(np.float64)) <= 1e-6 and _rel(vb, va.astype(np.float64)) <= 1e-6


@pytest.mark.parametrize("shape", [(1024, 16, 12), (1024, 24, 16)])
@pytest.mark.parametrize("field", ["random", "boosted"])
def test_step_measure_1024_wide_vs_oracle(shape, field):
    """The bench's fused step + diagnostics pass for 1024-wide 3D rows (Eqs. 3-5, 7, 8 from one
    read of the state) against the oracle directly: exact counts, A/V and gamma v to 1e-5 on the
    start state, then the fields after the following steps to 1e-5."""
    if field == "random":
        phi = inp.random_field(shape, 41).astype(np.float32)
        v = (0.3 * inp.random_field(shape, 42)).astype(np.float32)
    else:
        phi, v = inp.boosted_kink_pair(shape, 6.0, 0.4, axis=0)
        phi, v = phi.astype(np.float32), v.astype(np.float32)
    sim = prs.Sim(shape, precision=prs.PRS_FP32, W0=6.0)
    sim.set_state(phi, v, 0)
    d = prs.prs_step_measure(sim.handle, 9)
    pg, vg, n = sim.get_state()
    sim.close()
    p = oracle.Params(shape, W0=6.0)
    od = oracle.measure(p, phi.astype(np.float64), v.astype(np.float64))
    assert (d.n_links, d.n_wall, d.n_vzero, d.n_nonfinite) == (od.n_links, od.n_wall, od.n_vzero, od.n_nonfinite)
    assert d.area_per_volume == pytest.approx(od.area_per_volume, rel=1e-5)
    assert d.gamma_v == pytest.approx(od.gamma_v, rel=1e-5)
    ophi, ov = oracle.step(p, phi.astype(np.float64), v.astype(np.float64), 9)
    assert n == 9 and _rel(pg, ophi) <= 1e-5 and _rel(vg, ov) <= 1e-5


def test_measure_nonfinite_and_empty():
    shape = (16, 16)
    sim = prs.Sim(shape, precision=prs.PRS_FP64)
    phi = np.full((16, 16), 0.5)
    v = np.zeros((16, 16))
    sim.set_state(phi, v, 0)
    d = sim.measure()
    assert d["n_links"] == 0 and d["n_wall"] == 0 and d["gamma_v"] == 0.0 and d["area_per_volume"] == 0.0
    phi[3, 4] = np.nan
    sim.set_state(phi, v, 0)
    out = prs.prs_diag()
    rc = prs.load().prs_measure_ex(sim.handle, prs.ctypes.byref(out))
    assert rc == prs.PRS_ENONFINITE and out.n_nonfinite == 1
    sim.close()


def test_measure_repeatable_bitwise():
    """The FP64 reduction has a fixed order: repeated measurements agree bit for bit."""
    shape = (96, 80, 40)
    sim = prs.Sim(shape, precision=prs.PRS_FP32, seed=4)
    sim.init()
    sim.step(30)
    a = sim.measure()
    b = sim.measure()
    sim.close()
    assert a == b


# ------------------------------------------------- full-size sampled checks

def _subcube(field, centre, r):
    """Periodic (2r+1)^D neighbourhood of ``centre`` (numpy index order) of a torch tensor, as FP64 numpy."""
    import torch

    idx = np.ix_(*[np.arange(c - r, c + r + 1) % n for c, n in zip(centre, field.shape)])
    tidx = tuple(torch.as_tensor(i, device=field.device) for i in idx)
    return field[tidx].cpu().numpy().astype(np.float64)


def _sampled_step_check(shape, nsteps, tblock, nsamples=48, seed=0):
    """Run nsteps on the full box, then check sampled sites against the oracle on periodic
    (2 nsteps + 3)^D neighbourhoods (a site after k steps depends only on sites within k)."""
    sim = prs.Sim(shape, precision=prs.PRS_FP32, seed=seed, tblock=tblock)
    sim.init()
    phi0_t, _, _ = sim.tensors()
    fshape = tuple(phi0_t.shape)
    rng = np.random.Generator(np.random.PCG64(77))
    r = nsteps + 1
    picks = [tuple(int(rng.integers(0, s)) for s in fshape) for _ in range(nsamples)]
    picks += [tuple(0 for _ in fshape), tuple(s - 1 for s in fshape)]  # the periodic seams
    subs = [_subcube(phi0_t, c, r) for c in picks]
    sim.step(nsteps)
    phi_t, v_t, n = sim.tensors()
    assert n == nsteps
    worst = 0.0
    mid = tuple([r] * len(fshape))
    for c, sub in zip(picks, subs):
        p = oracle.Params(tuple(reversed(sub.shape)))
        ophi, ov = oracle.step(p, sub, np.zeros_like(sub), nsteps)
        worst = max(worst, abs(float(phi_t[c].item()) - ophi[mid]), abs(float(v_t[c].item()) - ov[mid]))
    sim.close()
    return worst


@pytest.mark.parametrize("tblock,nsteps", [(0, 4), (2, 4), (3, 7)])
def test_full_size_3d_1024_sampled(tblock, nsteps):
    """3D 1024^3 FP32 (0: the benchmark's launch configuration; 2: two-step passes; 3: two three-step
    passes and a single step): sampled sites after nsteps steps."""
    worst = _sampled_step_check((1024, 1024, 1024), nsteps, tblock)
    assert worst <= 1e-5  # |phi| < 1.1: absolute ~ relative


@pytest.mark.parametrize("tblock,nsteps", [(0, 6), (2, 6), (3, 7)])
def test_full_size_2d_4096_sampled(tblock, nsteps):
    """2D 4096^2 FP32 (0: the library default; 2: two-step passes; 3: two three-step passes and a
    single step): sampled sites after nsteps steps."""
    worst = _sampled_step_check((4096, 4096), nsteps, tblock)
    assert worst <= 1e-5


@pytest.mark.parametrize("tblock", [2, 3])
@pytest.mark.parametrize("shape", [(4096, 64), (2048, 152), (512, 40)])
def test_multi_step_passes_match_single_steps_2d(shape, tblock):
    """2D two- and three-step passes against one-step passes over many passes (whole rows of up to
    4096 columns; chunks of one row to several per SM)."""
    a = _run(shape, prs.PRS_FP32, 40, None, None, seed=3, tblock=1)
    b = _run(shape, prs.PRS_FP32, 40, None, None, seed=3, tblock=tblock)
    assert _rel(b[0], a[0].astype(np.float64)) <= 1e-5 and _rel(b[1], a[1].astype(np.float64)) <= 1e-5


def _fill(sim, phi_profile, v_profile, axis_len_last=True):
    """Write a field that depends on the slowest axis only into the run's current buffers."""
    import torch

    phi_t, v_t, _ = sim.tensors()
    shape = (phi_t.shape[0],) + (1,) * (phi_t.dim() - 1)
    phi_t.copy_(torch.as_tensor(phi_profile, dtype=phi_t.dtype, device=phi_t.device).reshape(shape).expand_as(phi_t))
    v_t.copy_(torch.as_tensor(v_profile, dtype=v_t.dtype, device=v_t.device).reshape(shape).expand_as(v_t))
    torch.cuda.synchronize()


def test_full_size_3d_1024_measure_exact_cases():
    """1024^3 FP32 diagnostics on fields with known answers (planar and boosted walls along z)."""
    import torch

    n = 1024
    sim = prs.Sim((n, n, n), precision=prs.PRS_FP32, seed=1)
    sim.init()
    prof, vprof = inp.kink_pair((4, 4, n), 10.0, axis=2)
    _fill(sim, prof[:, 0, 0], vprof[:, 0, 0])
    d = sim.measure()
    assert d["n_links"] == 2 * n * n and d["n_wall"] == 4 * n * n
    assert d["area_per_volume"] == pytest.approx(2.0 / n, rel=1e-12)  # every weight is exactly 1
    u = 0.3
    prof, vprof = inp.boosted_kink_pair((4, 4, n), 10.0, u, axis=2)
    _fill(sim, prof[:, 0, 0], vprof[:, 0, 0])
    d = sim.measure()
    assert d["gamma_v"] == pytest.approx(u / math.sqrt(1 - u * u), rel=1e-5)
    # Z2: the negated random field measures identically, bit for bit
    sim.init()
    sim.step(3)
    a = sim.measure()
    phi_t, _, _ = sim.tensors()
    phi_t.neg_()
    torch.cuda.synchronize()
    b = sim.measure()
    sim.close()
    assert {k: a[k] for k in a if k not in ("step", "eta")} == {k: b[k] for k in b if k not in ("step", "eta")}


def test_two_host_threads_on_two_runs():
    """Calls on different handles may overlap from two host threads (each run has its own
    stream): every run ends bit-identical to the same run driven alone."""
    import threading

    import torch

    shapes = [(256, 64, 32), (512, 128)]
    alone = []
    for i, shape in enumerate(shapes):
        sim = prs.Sim(shape, precision=prs.PRS_FP32, seed=40 + i)
        sim.init()
        diags = [prs.prs_step_measure(sim.handle, 7).as_dict() for _ in range(6)]
        alone.append((diags, sim.get_state()))
        sim.close()
    sims = [prs.Sim(shape, precision=prs.PRS_FP32, seed=40 + i, stream=torch.cuda.Stream())
            for i, shape in enumerate(shapes)]
    out = [None, None]
    errors = []

    def run(i):
        try:
            sims[i].init()
            out[i] = [prs.prs_step_measure(sims[i].handle, 7).as_dict() for _ in range(6)]
        except Exception as e:
            errors.append(e)

    threads = [threading.Thread(target=run, args=(i,)) for i in range(2)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    for i, sim in enumerate(sims):
        phi, v, n = sim.get_state()
        sim.close()
        assert out[i] == alone[i][0]
        assert n == alone[i][1][2] and np.array_equal(phi, alone[i][1][0]) and np.array_equal(v, alone[i][1][1])


def test_set_state_async():
    """prs_set_state_async queues the upload and returns; a run set this way (from pinned
    memory, two runs interleaved from one thread) steps exactly as one set with prs_set_state."""
    import torch

    shape = (256, 64, 24)
    fshape = tuple(reversed(shape))
    phi = torch.from_numpy(inp.random_field(shape, 17).astype(np.float32)).pin_memory()
    v = torch.from_numpy((0.1 * inp.random_field(shape, 18)).astype(np.float32)).pin_memory()
    ref = prs.Sim(shape, precision=prs.PRS_FP32)
    ref.set_state(phi.numpy(), v.numpy(), 5)
    dref = prs.prs_step_measure(ref.handle, 9).as_dict()
    pref, vref, nref = ref.get_state()
    ref.close()
    runs = [prs.Sim(shape, precision=prs.PRS_FP32, stream=torch.cuda.Stream()) for _ in range(2)]
    prs.prs_set_state_async(runs[0].handle, phi.numpy(), v.numpy(), 5)
    prs.prs_set_state_async(runs[1].handle, phi.numpy(), v.numpy(), 5)
    for r in runs:
        assert prs.prs_step_measure(r.handle, 9).as_dict() == dref
        p2, v2, n2 = r.get_state()
        r.close()
        assert n2 == nref and np.array_equal(p2, pref) and np.array_equal(v2, vref)

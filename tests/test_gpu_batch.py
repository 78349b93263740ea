"""The persistent ensemble engine (prs_batch_*) against the oracle and the single-run path.

Every run of a mixed 2D/3D ensemble, each with its own seed, era and number of
steps, must match the FP64 oracle to the FP32 field tolerance (1e-5 relative);
the fused diagnostics at output steps must match the oracle's on fields where
FP32 cannot move a sign (static walls), exactly in the counts.
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
    return float(np.max(np.abs(np.asarray(a, np.float64) - b)) / max(np.max(np.abs(b)), 1e-300))


RUNS = [  # shape, era_m, seed, nsteps
    ((256, 128), 1.0, 11, 23),
    ((128, 128), 2.0, 12, 17),
    ((512, 64), 1.0, 13, 0),
    ((128, 32, 16), 2.0, 14, 19),
    ((256, 32, 12), 1.0, 15, 11),
    ((4096, 8), 2.0, 16, 7),
    ((1024, 8, 6), 1.0, 17, 14),
]


def _params(shape, era, seed):
    return prs.make_params(shape, precision=prs.PRS_FP32, era_m=era, seed=seed)


def test_mixed_ensemble_matches_oracle():
    b = prs.prs_batch_create([_params(s, e, sd) for s, e, sd, _ in RUNS])
    try:
        ns = [n for *_, n in RUNS]
        prs.prs_batch_run(b, ns)
        for r, (shape, era, seed, n) in enumerate(RUNS):
            fshape = tuple(reversed(shape))
            phi = np.empty(fshape, np.float32)
            v = np.empty(fshape, np.float32)
            assert prs.prs_batch_get_state(b, r, phi, v) == n
            p = oracle.Params(shape, era_m=era)
            ophi, ov = oracle.step(p, *oracle.init_random(p, seed), n)
            assert _rel(phi, ophi) <= 1e-5, (shape, n)
            assert _rel(v, ov) <= 1e-5 if n else np.all(v == 0)
        # a second call continues every run from where it stopped
        prs.prs_batch_run(b, [5] * len(RUNS))
        for r, (shape, era, seed, n) in enumerate(RUNS[:3]):
            phi = np.empty(tuple(reversed(shape)), np.float32)
            assert prs.prs_batch_get_state(b, r, phi, None) == n + 5
            p = oracle.Params(shape, era_m=era)
            ophi, _ = oracle.step(p, *oracle.init_random(p, seed), n + 5)
            assert _rel(phi, ophi) <= 1e-5
    finally:
        prs.prs_batch_destroy(b)


def test_fused_diagnostics_on_static_walls():
    """Kink pairs stay put: every output must give the oracle's exact counts and A/V = 2/(N dx)."""
    runs = [((256, 64), 0), ((128, 64, 16), 2), ((128, 128), 1)]
    b = prs.prs_batch_create([_params(s, 1.0, 1) for s, _ in runs])
    try:
        fields = []
        for r, (shape, axis) in enumerate(runs):
            phi, v = inp.kink_pair(shape, 10.0, axis=axis)
            prs.prs_batch_set_state(b, r, phi, v, 0)
            fields.append((phi, v))
        out = prs.prs_batch_run(b, [20, 20, 20], measure_every=5, out_capacity=5)
        for r, (shape, axis) in enumerate(runs):
            p = oracle.Params(shape)
            phi, v = fields[r]
            d0 = oracle.measure(p, phi, v)
            N = shape[axis]
            for k in range(5):
                step, area, gv, nl = out[r, k]
                assert step == 5 * k
                assert nl == d0.n_links
                assert area == pytest.approx(2.0 / N, rel=1e-6)  # hardware rsqrt/reciprocal: a few ulp per weight
            assert out[r, 0, 2] == pytest.approx(d0.gamma_v, abs=1e-12)  # zero velocity at step 0
    finally:
        prs.prs_batch_destroy(b)


def test_diagnostics_at_step_zero_random_fields():
    runs = RUNS[:5]
    b = prs.prs_batch_create([_params(s, e, sd) for s, e, sd, _ in runs])
    try:
        out = prs.prs_batch_run(b, [0] * len(runs), measure_every=1, out_capacity=1)
        for r, (shape, era, seed, _) in enumerate(runs):
            p = oracle.Params(shape, era_m=era)
            d = oracle.measure(p, *oracle.init_random(p, seed))
            assert out[r, 0, 3] == d.n_links
            assert out[r, 0, 1] == pytest.approx(d.area_per_volume, rel=1e-5)
    finally:
        prs.prs_batch_destroy(b)


def test_batch_is_deterministic_and_matches_single_runs():
    """Two fresh ensembles give identical fields and counts (the diagnostic sums group per-tile
    partials in FP64, so tile lengths picked by the timing-based autotuner may regroup them:
    1e-12); each run agrees with prs_step + prs_measure."""
    runs = RUNS[:5]
    ns = [12, 9, 10, 8, 13]
    outs, states = [], []
    for _ in range(2):
        b = prs.prs_batch_create([_params(s, e, sd) for s, e, sd, _ in runs])
        outs.append(prs.prs_batch_run(b, ns, measure_every=4, out_capacity=4))
        st = []
        for r, (shape, *_rest) in enumerate(runs):
            phi = np.empty(tuple(reversed(shape)), np.float32)
            prs.prs_batch_get_state(b, r, phi, None)
            st.append(phi)
        states.append(st)
        prs.prs_batch_destroy(b)
    assert np.array_equal(outs[0][..., [0, 3]], outs[1][..., [0, 3]])  # steps and link counts
    assert np.allclose(outs[0], outs[1], rtol=1e-12, atol=0)
    for a, c in zip(states[0], states[1]):
        assert np.array_equal(a, c)
    for r, (shape, era, seed, _) in enumerate(runs):
        sim = prs.Sim(shape, precision=prs.PRS_FP32, era_m=era, seed=seed)
        sim.init()
        sim.step(ns[r])
        phi, _, _ = sim.get_state()
        sim.close()
        assert _rel(phi, states[0][r].astype(np.float64)) <= 1e-6


def test_autotuner_reports_a_choice():
    """One tile length per geometry class, from the candidates 4 .. 32."""
    runs = RUNS[:3] + RUNS[:3]
    b = prs.prs_batch_create([_params(s, e, sd + 100 * (i >= 3)) for i, (s, e, sd, _) in enumerate(runs)])
    try:
        t = [prs.prs_batch_tuning(b, r)[0] for r in range(len(runs))]
        assert all(x in (4, 8, 16, 32) for x in t) and prs.prs_batch_tuning(b, 0)[1] > 0
        for r in range(3):  # runs of one box share their class's choice
            assert t[r] == t[r + 3] or runs[r][0] != runs[r + 3][0]
    finally:
        prs.prs_batch_destroy(b)


def test_batch_rejects_unsupported_runs():
    import ctypes

    p = [prs.make_params((130, 64))]  # x side not a multiple of 128
    arr = (prs.prs_params * 1)(*p)
    h = ctypes.c_void_p()
    assert prs.load().prs_batch_create(arr, 1, None, ctypes.byref(h)) == prs.PRS_EINVAL


def test_production_box_sizes_match_single_runs():
    """Matter-era runs at the production box sizes (3D 1024^3, 2D 4096^2) in one ensemble agree
    with the same runs stepped alone: the diagnostics of the initial field exactly in the counts,
    later outputs and the final fields to FP32 rounding (the ensemble and the single-run kernels
    run the same tile routine; the compiler may contract a*b+c differently in each)."""
    runs = [((1024, 1024, 1024), 2.0, 7), ((4096, 4096), 2.0, 8)]
    ns, every = 12, 4
    b = prs.prs_batch_create([_params(s, e, sd) for s, e, sd in runs])
    try:
        out = prs.prs_batch_run(b, [ns] * len(runs), measure_every=every, out_capacity=ns // every + 1)
        states = []
        for r, (shape, *_rest) in enumerate(runs):
            phi = np.empty(tuple(reversed(shape)), np.float32)
            assert prs.prs_batch_get_state(b, r, phi, None) == ns
            states.append(phi)
    finally:
        prs.prs_batch_destroy(b)
    for r, (shape, era, seed) in enumerate(runs):
        sim = prs.Sim(shape, precision=prs.PRS_FP32, era_m=era, seed=seed)
        sim.init()
        for k in range(ns // every + 1):
            d = prs.prs_step_measure(sim.handle, every if k < ns // every else 0)
            assert out[r, k, 0] == every * k == d.step
            if k == 0:
                assert out[r, k, 3] == d.n_links
                assert out[r, k, 1] == pytest.approx(d.area_per_volume, rel=1e-12)
            else:
                assert out[r, k, 3] == pytest.approx(d.n_links, rel=1e-5)
                assert out[r, k, 1] == pytest.approx(d.area_per_volume, rel=1e-5)
                assert out[r, k, 2] == pytest.approx(d.gamma_v, rel=1e-4)
        phi, _, n = sim.get_state()
        sim.close()
        assert n == ns
        assert _rel(states[r], phi.astype(np.float64)) <= 1e-6
        del phi
        states[r] = None


@pytest.mark.parametrize("big,ns", [((2048, 2048), [13, 9, 12]), ((2048, 2048), [12, 7, 5]),
                                    ((2048, 2048), [13, 9, 13]), ((2048, 2048), [12, 7, 12]),
                                    ((4096, 4096), [13, 9, 13])])
def test_large_runs_are_stepped_alone(big, ns):
    """Runs of 2^22 sites or more that the library steps with multi-step passes (2D 2048^2 and
    4096^2, three steps per pass) leave the persistent kernel and are stepped alone per output
    interval, runs of one box at the same step count together (one launch of each pass for both,
    different eras); their fields are those of the same run stepped by prs_step_measure, bit for bit
    (the same tile routines and passes), their counts exactly and their sums to FP64 rounding (the
    grouped launch groups the FP64 block sums differently), whether the last output falls on a step
    of the call or not; the small run beside them stays in the persistent kernel
    and follows a single run."""
    runs = [(big, 1.0, 21), ((256, 128), 2.0, 22), (big, 2.0, 23)]
    every = 4
    cap = max(ns) // every + 1
    b = prs.prs_batch_create([_params(s, e, sd) for s, e, sd in runs])
    try:
        assert [prs.prs_batch_tuning(b, r)[0] for r in range(3)][::2] == [0, 0]
        assert prs.prs_batch_tuning(b, 1)[0] in (4, 8, 16, 32)
        out = prs.prs_batch_run(b, ns, measure_every=every, out_capacity=cap)
        states = []
        for r, (shape, *_rest) in enumerate(runs):
            phi = np.empty(tuple(reversed(shape)), np.float32)
            v = np.empty(tuple(reversed(shape)), np.float32)
            assert prs.prs_batch_get_state(b, r, phi, v) == ns[r]
            states.append((phi, v))
        # a second call continues from the state the first left (buffers handed back)
        out2 = prs.prs_batch_run(b, [3, 2, 3], measure_every=every, out_capacity=cap)
        phi2 = np.empty(tuple(reversed(big)), np.float32)
        assert prs.prs_batch_get_state(b, 2, phi2, None) == ns[2] + 3
    finally:
        prs.prs_batch_destroy(b)
    for r, (shape, era, seed) in enumerate(runs):
        sim = prs.Sim(shape, precision=prs.PRS_FP32, era_m=era, seed=seed)
        sim.init()
        for k in range(ns[r] // every + 1):
            left = ns[r] - k * every
            d = prs.prs_step_measure(sim.handle, min(left, every))
            assert out[r, k, 0] == every * k == d.step
            if r != 1:
                assert out[r, k, 3] == d.n_links and out[r, k, 1] == pytest.approx(d.area_per_volume, rel=1e-12)
                assert out[r, k, 2] == pytest.approx(d.gamma_v, rel=1e-12)
        phi, v, n = sim.get_state()
        assert n == ns[r]
        if r != 1:
            assert np.array_equal(states[r][0], phi) and np.array_equal(states[r][1], v)
        else:
            assert _rel(states[r][0], phi.astype(np.float64)) <= 1e-6
        if r == 2:
            d = prs.prs_step_measure(sim.handle, 3)
            assert out2[2, 0, 0] == ns[2] and out2[2, 0, 3] == d.n_links
            assert out2[2, 0, 1] == pytest.approx(d.area_per_volume, rel=1e-12)
            p2, _, _ = sim.get_state()
            assert np.array_equal(phi2, p2)
        sim.close()


@pytest.mark.parametrize("every", [6, 8, 10])
def test_grouped_passes_follow_the_single_run_plan(every):
    """Three 2048^2 runs stepped together (one launch per round of three-step passes) through
    output intervals whose remaining steps plan as a triple and a pair (every 6), two triples and
    a single step (every 8) and three triples that bound buffers turn into two triples, a pair
    and a single step (every 10): fields and outputs bit for bit those of each run stepped by
    prs_step_measure."""
    runs = [((2048, 2048), 1.0, 31), ((2048, 2048), 2.0, 32), ((2048, 2048), 1.0, 33)]
    ns = 23
    cap = ns // every + 1
    b = prs.prs_batch_create([_params(s, e, sd) for s, e, sd in runs])
    try:
        out = prs.prs_batch_run(b, [ns] * 3, measure_every=every, out_capacity=cap)
        states = []
        for r in range(3):
            phi = np.empty((2048, 2048), np.float32)
            v = np.empty((2048, 2048), np.float32)
            assert prs.prs_batch_get_state(b, r, phi, v) == ns
            states.append((phi, v))
    finally:
        prs.prs_batch_destroy(b)
    for r, (shape, era, seed) in enumerate(runs):
        sim = prs.Sim(shape, precision=prs.PRS_FP32, era_m=era, seed=seed)
        sim.init()
        for k in range(ns // every + 1):
            d = prs.prs_step_measure(sim.handle, min(ns - k * every, every))
            assert out[r, k, 0] == d.step and out[r, k, 3] == d.n_links
            assert out[r, k, 1] == pytest.approx(d.area_per_volume, rel=1e-12)
            assert out[r, k, 2] == pytest.approx(d.gamma_v, rel=1e-12)
        phi, v, n = sim.get_state()
        sim.close()
        assert n == ns and np.array_equal(states[r][0], phi) and np.array_equal(states[r][1], v)


@pytest.mark.parametrize("n1024", [8, 7])
def test_classes_of_1024_rows_go_alone_in_numbers(n1024):
    """2D runs of 1024^2 (2^20 sites, rows of 1024 columns) are stepped alone, their three-step
    passes launched together, when the ensemble holds at least 8 of them; with 7 they stay in the
    persistent kernel.  Either way each run's fields follow the run stepped alone (bit for bit when
    stepped alone, with counts exact and sums to FP64 rounding; to FP32 rounding in the persistent
    kernel)."""
    runs = [((1024, 1024), 1.0 + (i & 1), 40 + i) for i in range(n1024)] + [((256, 128), 2.0, 60)]
    ns, every = 11, 5
    b = prs.prs_batch_create([_params(s, e, sd) for s, e, sd in runs])
    try:
        tl = [prs.prs_batch_tuning(b, r)[0] for r in range(len(runs))]
        alone = n1024 >= 8
        assert all((t == 0) == alone for t in tl[:-1]) and tl[-1] in (4, 8, 16, 32)
        out = prs.prs_batch_run(b, [ns] * len(runs), measure_every=every, out_capacity=ns // every + 1)
        states = []
        for r, (shape, *_rest) in enumerate(runs):
            phi = np.empty(tuple(reversed(shape)), np.float32)
            assert prs.prs_batch_get_state(b, r, phi, None) == ns
            states.append(phi)
    finally:
        prs.prs_batch_destroy(b)
    for r in (0, 1, n1024 - 1):
        shape, era, seed = runs[r]
        sim = prs.Sim(shape, precision=prs.PRS_FP32, era_m=era, seed=seed)
        sim.init()
        for k in range(ns // every + 1):
            d = prs.prs_step_measure(sim.handle, min(ns - k * every, every))
            assert out[r, k, 0] == d.step
            if alone:
                assert out[r, k, 3] == d.n_links and out[r, k, 1] == pytest.approx(d.area_per_volume, rel=1e-12)
        phi, _, _ = sim.get_state()
        sim.close()
        if alone:
            assert np.array_equal(states[r], phi)
        else:
            assert _rel(states[r], phi.astype(np.float64)) <= 1e-6

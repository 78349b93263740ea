"""Host-side logic of bench.py, without a GPU: the Eq. 9 exponent fit, the replica
aggregate, the clock-sample parsing, the kernel-source hash, and the reference arm's JSON
line (which times the oracle on the host)."""
import importlib.util
import json
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_scaling_exponents_recover_power_laws(bench):
    """rho = A eta^mu, gamma v = B eta^nu: the fit beyond ln(eta) = 2.58 returns mu and nu; the
    error is the standard error of the per-run slopes."""
    eta = 1.0 + np.arange(0, 1024, 1.0)
    runs = []
    mus = [-0.95, -0.93, -0.97]
    nus = [0.01, -0.03, 0.02]
    for mu, nu in zip(mus, nus):
        area = 3.0 * eta ** mu
        gv = 0.4 * eta ** nu
        area[np.log(eta) <= 2.58] = 7.0  # the early part must not enter the fit
        runs.append((eta, area, gv))
    r = bench.scaling_exponents(runs)
    assert r["mu"] == pytest.approx(np.mean(mus), abs=1e-12)
    assert r["nu"] == pytest.approx(np.mean(nus), abs=1e-12)
    assert r["mu_err"] == pytest.approx(np.std(mus, ddof=1) / np.sqrt(3), rel=1e-9)
    assert r["mu_runs"] == pytest.approx(mus, abs=1e-12)
    late = bench.scaling_exponents(runs, ln_eta_min=5.0)
    assert late["mu"] == pytest.approx(np.mean(mus), abs=1e-12)


def test_aggregate_is_all_units_over_the_slowest_rank(bench):
    assert bench.aggregate(1000, 4, 2.0) == 2000.0


def test_clock_summary(bench):
    c = bench.ClockSampler(0)
    c.lines = ["2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
               "2055, 2070, 1300.0, 0x4, Not Active, Not Active, Not Active, Active",
               "2070, 2070, 1350.2, 0x4, Not Active, Not Active, Not Active, Active",
               "garbage line"]
    s = c.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
    c.lines = []
    assert c.summary()["reasons"] == ["unsampled"]


def test_interval_calls_split_an_interval(bench):
    """After the fused step + diagnostics, an interval's other steps are one call of whole passes of
    the step kernel (the bracket the roofline times) and a remainder shorter than a pass."""
    for tb in (1, 2):
        for tmax in (tb, 3):
            for interval in range(1, 64):
                pure, tail, launches = bench.interval_calls(interval, tb, tmax)
                assert pure + tail == interval - 1 and pure % tb == 0
                if tb == 2 and tmax == 3 and tail == 3:  # a pair and the odd step as one three-step pass
                    assert launches == 1 and (interval - 1) % 2 == 1
                else:
                    assert 0 <= tail < tb and launches == tail
    assert bench.interval_calls(20, 2) == (18, 1, 1) and bench.interval_calls(20, 1) == (19, 0, 0)
    assert bench.interval_calls(20, 2, 3) == (16, 3, 1)


def test_kernel_source_hash_and_traffic_record(bench):
    h = bench.kernel_sources_sha()
    assert len(h) == 16 and h == bench.kernel_sources_sha()
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        rec = json.load(f)["3d1024"]
    for name in rec["sources"]:
        assert os.path.exists(os.path.join(ROOT, "paper_1710_10420_gb300", "csrc", name))
    # a record is used only for its steps per pass and while its kernel's sources are unchanged
    tb = rec.get("tblock", 1)
    same = rec["sources_sha"] == bench.kernel_sources_sha(tuple(rec["sources"]))
    assert (bench.traffic_record("3d1024", tb) is not None) == same
    assert bench.traffic_record("3d1024", 3 - tb) is None


def test_reference_arm_prints_one_json_line(bench):
    import oracle

    oracle.build()
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                        "--warmup", "1", "--interval", "2"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 1 and d["value"] > 0
    assert d["metric"] == bench.METRIC  # the GPU arm's metric: the driver can form the ratio
    for key in ("metric", "unit", "n_gpus", "ms_per_step", "higher_is_better", "dtype", "config", "cpu_baseline",
                "e2e"):
        assert key in d
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]

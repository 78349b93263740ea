"""The C ABI: library loads, exports every declared symbol, validates arguments (CPU only).

No compute call is made here: only host-side entry points that fail before
touching the device, and the host coefficient schedule.
"""
import ctypes
import math

import pytest

import paper_1710_10420_gb300 as prs


@pytest.fixture(scope="module")
def lib():
    return prs.load(build=True)


def test_every_declared_symbol_is_exported(lib):
    names = prs.declared_functions()
    assert "prs_create" in names and "prs_step" in names and "prs_measure" in names
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_the_header():
    for n in prs.declared_functions():
        assert hasattr(prs, n), f"binding lacks {n}"


def test_header_constants_match_the_binding():
    """Every #define PRS_<NAME> value in include/prs.h equals the binding's constant."""
    import pathlib
    import re

    text = (pathlib.Path(__file__).resolve().parents[1] / "include" / "prs.h").read_text()
    found = re.findall(r"^#define\s+(PRS_\w+)\s+\(?(-?\d+)u?\)?", text, flags=re.M)
    assert len(found) >= 12
    for name, value in found:
        assert getattr(prs, name) == int(value), name


def test_strerror(lib):
    assert prs.strerror(prs.PRS_OK) == "ok"
    assert prs.strerror(prs.PRS_EINVAL) == "invalid argument"
    assert prs.strerror(12345) == "unknown status"


@pytest.mark.parametrize("bad", [
    dict(shape=(2, 8)),                       # side < 3
    dict(shape=(8, 8), deta=1.0),             # leapfrog unstable: deta^2 * 8 >= 4
    dict(shape=(8, 8, 8), deta=0.82),         # 3D limit deta < 0.816
    dict(shape=(8, 8), precision=7),
    dict(shape=(8, 8), dx=0.0),
    dict(shape=(8, 8), eta0=0.0),
    dict(shape=(8, 8), eta0=0.1, deta=0.2),   # delta >= 1 at the first step
    dict(shape=(8, 8), tblock=99),
    dict(shape=(8, 8), flags=8),
])
def test_create_rejects_bad_parameters(lib, bad):
    shape = bad.pop("shape")
    p = prs.make_params(shape, **bad)
    h = ctypes.c_void_p()
    assert lib.prs_create(ctypes.byref(p), None, ctypes.byref(h)) == prs.PRS_EINVAL
    assert h.value is None


def test_null_handles_are_rejected(lib):
    assert lib.prs_step(None, 1) == prs.PRS_EINVAL
    assert lib.prs_measure(None, None, None, None, None) == prs.PRS_EINVAL
    assert lib.prs_destroy(None) == prs.PRS_EINVAL
    assert lib.prs_create(None, None, None) == prs.PRS_EINVAL


def test_host_coefficients_follow_eq6():
    """delta_n = alpha deta m/(2 eta_n): the paper's radiation-era PRS first step has delta = 0.15."""
    p = prs.make_params((8, 8))
    c = prs.prs_coefficients(p, 0)
    assert c["delta"] == pytest.approx(0.15, rel=1e-15)
    assert c["c1"] == pytest.approx(0.85 / 1.15, rel=1e-15)
    assert c["c2"] == pytest.approx(0.1 / 1.15, rel=1e-15)
    assert c["cV"] == pytest.approx(4 * math.pi ** 2 / 200, rel=1e-15)
    c = prs.prs_coefficients(prs.make_params((8, 8), era_m=2.0), 10)  # eta = 2
    assert c["delta"] == pytest.approx(0.5 * 3 * 0.1 * 2 / 2.0, rel=1e-15)
    assert prs.prs_coefficients(prs.make_params((8, 8), W0=math.inf), 0)["cV"] == 0.0


def test_default_steps_per_pass(lib):
    """The library's default steps per pass (host logic): FP32 3D, one below 2^24 sites, else two
    where the two-step tiles get at least 4 rows of y; FP32 2D, three on rows of 2048 or more and on
    boxes of at most 1024 rows, else two from 2^24 sites and one below; one
    otherwise (FP64, boxes the staged kernels do not take, a prime y side)."""
    cases = [((512, 512, 512), prs.PRS_FP32, 2), ((128, 128, 128), prs.PRS_FP32, 1),
             ((256, 128, 128), prs.PRS_FP32, 1), ((256, 256, 256), prs.PRS_FP32, 2),
             ((256, 256, 1024), prs.PRS_FP32, 2), ((1024, 1024, 1024), prs.PRS_FP32, 2),
             ((1024, 1024, 256), prs.PRS_FP32, 2), ((4096, 4096), prs.PRS_FP32, 3),
             ((2048, 2048), prs.PRS_FP32, 3), ((512, 512, 512), prs.PRS_FP64, 1),
             ((500, 500, 500), prs.PRS_FP32, 1), ((4096, 4096), prs.PRS_FP64, 1),
             ((256, 251, 64), prs.PRS_FP32, 1), ((384, 96, 32), prs.PRS_FP32, 1),
             ((2048, 8192), prs.PRS_FP32, 3), ((4096, 8192), prs.PRS_FP32, 3), ((1024, 16384), prs.PRS_FP32, 2),
             ((256, 256), prs.PRS_FP32, 3), ((1024, 1024), prs.PRS_FP32, 3), ((512, 2048), prs.PRS_FP32, 1),
             ((1024, 4096), prs.PRS_FP32, 1), ((2048, 512), prs.PRS_FP32, 3), ((384, 128, 512), prs.PRS_FP32, 2)]
    for shape, precision, want in cases:
        assert prs.prs_default_tblock(prs.make_params(shape, precision=precision)) == want, shape


def test_max_steps_per_pass(lib):
    """The most steps one pass fuses: three for FP32 3D boxes of the three-step pass (x sides that are
    multiples of 128, y sides multiples of 8 of at least 16) and FP32 2D boxes of the 2D three-step
    pass (x sides that are multiples of 128 up to 4096), one for FP64 and boxes the staged kernels do
    not take; never below the default."""
    cases = [((512, 512, 512), prs.PRS_FP32, 3), ((128, 128, 128), prs.PRS_FP32, 3),
             ((1024, 1024, 1024), prs.PRS_FP32, 3), ((384, 96, 32), prs.PRS_FP32, 3),
             ((4096, 4096), prs.PRS_FP32, 3), ((2048, 2048), prs.PRS_FP32, 3), ((128, 3), prs.PRS_FP32, 3),
             ((512, 512, 512), prs.PRS_FP64, 1), ((500, 500, 500), prs.PRS_FP32, 1),
             ((4096, 4096), prs.PRS_FP64, 1)]
    for shape, precision, want in cases:
        p = prs.make_params(shape, precision=precision)
        assert prs.prs_max_tblock(p) == want, shape
        assert prs.prs_max_tblock(p) >= prs.prs_default_tblock(p), shape

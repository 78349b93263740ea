"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each test checks the oracle against something other than itself: a published test
vector, a closed form of the discrete scheme, an exact invariant, or a brute-force
loop written separately below.  A plausible slip in the oracle (a dropped 1/dx^2,
a wrong force coefficient, a sign or index error, a transposed neighbour) fails
at least one of them.
"""
import math
import os

import numpy as np
import pytest

import oracle
import prs_inputs as inp

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------- random numbers

def test_splitmix64_published_vectors():
    """SplitMix64 (Steele, Lea & Flood 2014) outputs for state 0: the source of the ICs (Sec. III)."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "splitmix64_seed0.txt")) if l.strip() and l[0] != "#"]
    assert len(rows) >= 4
    for idx, hexval in rows:
        assert oracle.splitmix64(0, int(idx)) == int(hexval, 16)


def test_uniform_ic_distribution():
    """Random ICs (Sec. III): i.i.d. uniform in (-1,1), on the FP32-exact 24-bit grid, never 0."""
    p = oracle.Params((1000, 1000))
    phi, v = oracle.init_random(p, seed=0)
    assert np.all(v == 0.0)
    assert np.all(np.abs(phi) < 1.0) and np.all(phi != 0.0)
    assert np.array_equal(phi.astype(np.float32).astype(np.float64), phi)
    k = (phi + 1.0) * 2.0 ** 23 - 0.5  # (2k+1)/2^24 - 1  ->  k
    assert np.array_equal(k, np.round(k)) and k.min() >= 0 and k.max() < 2 ** 24
    n = phi.size
    sig = math.sqrt(1.0 / 3.0 / n)
    assert abs(phi.mean()) < 5 * sig
    assert abs(phi.var() - 1.0 / 3.0) < 5 * math.sqrt(4.0 / 45.0 / n)
    # different seeds give different, uncorrelated fields
    phi1, _ = oracle.init_random(p, seed=1)
    assert abs(np.corrcoef(phi.ravel(), phi1.ravel())[0, 1]) < 5 / math.sqrt(n)
    # the linear index is the counter: a row of the 2D field equals the 1D stream
    assert phi.ravel()[12345] == oracle.uniform(0, 12345)


# ---------------------------------------------------- linear part: dispersion

def _theta(deta, omega2):
    """Discrete-time leapfrog phase per step: 4 sin^2(theta/2) = deta^2 Omega^2."""
    return 2.0 * math.asin(math.sqrt(deta * deta * omega2) / 2.0)


def _omega2(k, dx, m2=0.0):
    """Lattice dispersion: Omega^2 = sum_i 4 sin^2(k_i dx/2)/dx^2 + m^2."""
    return sum(4.0 * math.sin(ki * dx / 2.0) ** 2 / dx ** 2 for ki in k) + m2


@pytest.mark.parametrize("shape,modes,dx,deta,nsteps", [
    ((16, 12), (3, 2), 1.0, 0.1, 300),
    ((16, 12), (8, 6), 1.0, 0.3, 200),     # Nyquist mode: the stencil's largest eigenvalue
    ((10, 8, 6), (1, 3, 2), 0.7, 0.2, 150),  # dx != 1 checks the 1/dx^2 of the Laplacian
    ((9, 7, 5), (2, 1, 1), 1.0, 0.1, 120),   # odd sides
])
def test_free_field_dispersion(shape, modes, dx, deta, nsteps):
    """V0 = 0, alpha = 0: phi^n = A cos(k.x) cos((n+1/2) theta)/cos(theta/2) exactly (Eqs. 3-5)."""
    p = oracle.Params(shape, dx=dx, deta=deta, alpha=0.0, W0=math.inf)
    phi0, v0, k = inp.plane_wave(shape, modes, amp=1.0, dx=dx)
    th = _theta(deta, _omega2(k, dx))
    phi, v = oracle.step(p, phi0, v0, nsteps)
    expect = phi0 * math.cos((nsteps + 0.5) * th) / math.cos(th / 2)
    assert np.max(np.abs(phi - expect)) < 1e-11
    # velocity at n+1/2 is (phi^{n+1}-phi^n)/deta: closed form of the same solution
    vexp = phi0 * (math.cos((nsteps + 0.5) * th) - math.cos((nsteps - 0.5) * th)) / (deta * math.cos(th / 2))
    assert np.max(np.abs(v - vexp)) < 1e-10


@pytest.mark.parametrize("shape,modes,W0", [((32, 16), (2, 1), 10.0), ((12, 10, 8), (1, 2, 1), 6.0)])
def test_vacuum_perturbation_dispersion(shape, modes, W0):
    """phi = phi0 + eps cos(k.x) about the vacuum oscillates with m^2 = V''(phi0) = 8 V0/phi0^2."""
    eps = 1e-7
    p = oracle.Params(shape, alpha=0.0, W0=W0)
    phi0, v0, k = inp.plane_wave(shape, modes, amp=eps, offset=1.0)
    m2 = 8.0 * (math.pi ** 2 / (2.0 * W0 ** 2))
    th = _theta(p.deta, _omega2(k, p.dx, m2))
    n = 200
    phi, _ = oracle.step(p, phi0, v0, n)
    expect = (phi0 - 1.0) * math.cos((n + 0.5) * th) / math.cos(th / 2)
    err = np.max(np.abs((phi - 1.0) - expect)) / eps
    assert err < 5e-5  # nonlinear corrections are O(eps) relative
    # a wrong mass (e.g. V''(phi0) = 4 V0) would miss by O(1)
    th_bad = _theta(p.deta, _omega2(k, p.dx, m2 / 2))
    bad = (phi0 - 1.0) * math.cos((n + 0.5) * th_bad) / math.cos(th_bad / 2)
    assert np.max(np.abs((phi - 1.0) - bad)) / eps > 1e-2


# ------------------------------------------------------------------ damping

@pytest.mark.parametrize("era_m,alpha", [(1.0, 3.0), (2.0, 3.0), (1.0, 2.0)])
def test_damping_gamma_closed_form(era_m, alpha):
    """Uniform field, V0 = 0: v^{n+1/2} = prod_k (1-delta_k)/(1+delta_k) v^{-1/2} (Eqs. 4, 6).

    With delta_k = a/eta_k, a = alpha deta m/2, eta_k = eta0 + k deta, the product is
    Gamma(n+p) Gamma(q) / (Gamma(p) Gamma(n+q)), p = (eta0-a)/deta, q = (eta0+a)/deta.
    """
    shape = (4, 3)
    p = oracle.Params(shape, alpha=alpha, era_m=era_m, W0=math.inf, eta0=1.0, deta=0.1)
    phi0 = np.full((3, 4), 0.3)
    v0 = np.full((3, 4), 0.5)
    a = 0.5 * alpha * p.deta * era_m
    pp, qq = (p.eta0 - a) / p.deta, (p.eta0 + a) / p.deta
    for n in (1, 7, 100, 630):
        phi, v = oracle.step(p, phi0, v0, n)
        ratio = math.exp(math.lgamma(n + pp) + math.lgamma(qq) - math.lgamma(pp) - math.lgamma(n + qq))
        assert np.all(v == v[0, 0]) and np.all(phi == phi[0, 0])
        assert abs(v[0, 0] / (0.5 * ratio) - 1.0) < 1e-12
    # delta of the first step at eta0 = 1 in the radiation era with PRS alpha = 3 is 0.15
    c = oracle.coeffs(oracle.Params(shape), 0)
    assert abs(c["delta"] - 0.15) < 1e-15


# ------------------------------------------------------------- static kink

@pytest.mark.parametrize("shape,axis", [((64, 6), 0), ((5, 64), 1), ((4, 6, 64), 2)])
def test_static_kink_pair(shape, axis):
    """A tanh kink of width W0 is (nearly) static under PRS beta=0 and measures A/V = 2/(N dx)."""
    W0 = 10.0
    p = oracle.Params(shape, W0=W0)
    phi0, v0 = inp.kink_pair(shape, W0, axis=axis)
    npax = p.dims - 1 - axis  # numpy axis of the lattice axis
    mirror = lambda f: np.flip(f, axis=npax)
    assert np.array_equal(mirror(phi0), phi0)
    sign0 = phi0 < 0
    N = shape[axis]
    d0 = oracle.measure(p, phi0, v0)
    assert d0.n_links == 2 * p.sites // N
    assert d0.area_per_volume == pytest.approx(2.0 / (N * p.dx), rel=1e-14)
    phi, v = phi0, v0
    for _ in range(6):
        phi, v = oracle.step(p, phi, v, 50)
        # the walls do not move: the zero crossings stay between the same sites
        assert np.array_equal(phi < 0, sign0)
        # the lattice mirror symmetry about N/2 - 1/2 is kept bit for bit
        assert np.array_equal(mirror(phi), phi)
        d = oracle.measure(p, phi, v)
        assert d.area_per_volume == pytest.approx(2.0 / (N * p.dx), rel=1e-14)
    # the profile only relaxes to the lattice kink: O((pi dx/W0)^2/12) ~ 1e-2
    assert np.max(np.abs(phi - phi0)) < 0.03


def test_kink_width_fixes_the_force():
    """With the potential of a wall twice as thick the same profile is far from static."""
    shape = (64, 4)
    phi0, v0 = inp.kink_pair(shape, 10.0)
    phi, _ = oracle.step(oracle.Params(shape, W0=20.0), phi0, v0, 300)
    assert np.max(np.abs(phi - phi0)) > 0.1


# -------------------------------------------------------------- symmetries

@pytest.mark.parametrize("shape", [(16, 12), (6, 5, 7)])
def test_z2_translation_reflection(shape):
    """V is even: phi -> -phi commutes with the step bit for bit; so do periodic shifts and mirrors."""
    p = oracle.Params(shape, W0=4.0)
    phi0 = inp.random_field(shape, seed=5)
    v0 = 0.1 * inp.random_field(shape, seed=6)
    phi, v = oracle.step(p, phi0, v0, 40)
    phin, vn = oracle.step(p, -phi0, -v0, 40)
    assert np.array_equal(phin, -phi) and np.array_equal(vn, -v)
    sh = tuple(range(1, p.dims + 1))
    phis, vs = oracle.step(p, np.roll(phi0, sh, axis=tuple(range(p.dims))), np.roll(v0, sh, axis=tuple(range(p.dims))),
                           40)
    assert np.array_equal(phis, np.roll(phi, sh, axis=tuple(range(p.dims))))
    for ax in range(p.dims):
        # x -> -x on the periodic lattice maps site i to (N - i) mod N
        refl = lambda f: np.roll(np.flip(f, axis=ax), 1, axis=ax)
        phr, vr = oracle.step(p, refl(phi0), refl(v0), 40)
        assert np.array_equal(phr, refl(phi)) and np.array_equal(vr, refl(v))
    d, dn = oracle.measure(p, phi, v), oracle.measure(p, phin, vn)
    assert (d.n_links, d.n_wall) == (dn.n_links, dn.n_wall)
    assert d.sum_w == dn.sum_w and d.sum_ratio == dn.sum_ratio


# ------------------------------------------------------------ area estimator

@pytest.mark.parametrize("shape,axis,dx", [((32, 32), 0, 1.0), ((32, 32), 1, 0.5), ((16, 16, 16), 2, 1.0),
                                           ((12, 20, 8), 1, 2.0)])
def test_planar_wall_area_exact(shape, axis, dx):
    """Eq. 7 on a planar wall pair gives exactly 2/(N dx): every weight is 1."""
    p = oracle.Params(shape, dx=dx)
    phi, v = inp.kink_pair(shape, 10.0, axis=axis)
    d = oracle.measure(p, phi, v)
    assert d.n_links == 2 * p.sites // shape[axis]
    assert d.sum_w == d.n_links
    assert d.area_per_volume == pytest.approx(2.0 / (shape[axis] * dx), rel=1e-15)


@pytest.mark.parametrize("shape", [(128, 128), (64, 64, 4)])
def test_tilted_wall_area(shape):
    """A 45 degree wall pair: A/V = 2 sqrt(2)/N; |grad phi| over the L1 norm recovers it to ~1%.

    Without the Eq. 7 weight the raw link count would overshoot by sqrt(2).
    """
    p = oracle.Params(shape)
    phi, v = inp.tilted_wall_pair(shape, 10.0)
    d = oracle.measure(p, phi, v)
    true = 2.0 * math.sqrt(2.0) / shape[0]
    assert abs(d.area_per_volume / true - 1.0) < 0.02
    assert d.n_links / p.sites / true == pytest.approx(math.sqrt(2.0), rel=0.02)


def test_bubble_area():
    """A tanh disc / ball of radius R = N/4: A/V -> 2 pi R/N^2 (2D), 4 pi R^2/N^3 (3D)."""
    n = 128
    p = oracle.Params((n, n))
    phi, v = inp.bubble((n, n), n / 4, 6.0)
    d = oracle.measure(p, phi, v)
    assert abs(d.area_per_volume / (2 * math.pi * (n / 4) / n ** 2) - 1.0) < 0.03
    n = 48
    p = oracle.Params((n, n, n))
    phi, v = inp.bubble((n, n, n), n / 4, 6.0)
    d = oracle.measure(p, phi, v)
    assert abs(d.area_per_volume / (4 * math.pi * (n / 4) ** 2 / n ** 3) - 1.0) < 0.05


# ----------------------------------------------------------- brute force counts

def _brute_counts(sign_neg):
    """Link and wall-site counts by direct enumeration of the periodic lattice (independent loop)."""
    arr = np.asarray(sign_neg, dtype=bool)
    dims = arr.ndim
    n_links = 0
    n_wall = 0
    for idx in np.ndindex(*arr.shape):
        wall = False
        for ax in range(dims):
            for step in (+1, -1):
                j = list(idx)
                j[ax] = (j[ax] + step) % arr.shape[ax]
                differs = arr[idx] != arr[tuple(j)]
                if differs and step == +1:
                    n_links += 1
                wall = wall or differs
        n_wall += wall
    return n_links, n_wall


def _all_patterns(fshape):
    n = int(np.prod(fshape))
    for bits in range(1 << n):
        yield np.array([(bits >> i) & 1 for i in range(n)], dtype=bool).reshape(fshape)


@pytest.mark.parametrize("shape", [(3, 3), (2, 2, 2), (4, 2), (3, 2)])
def test_link_counts_all_sign_patterns(shape):
    """Every sign pattern of tiny periodic grids: N_links and N_wall match enumeration exactly."""
    p = oracle.Params(shape)
    fshape = p.array_shape()
    for i, neg in enumerate(_all_patterns(fshape)):
        phi = inp.random_signs(shape, seed=i, signs=np.where(neg, -1.0, 1.0))
        d = oracle.measure(p, phi, np.zeros_like(phi))
        assert (d.n_links, d.n_wall) == _brute_counts(neg), neg


@pytest.mark.parametrize("shape,seed", [((5, 4), 1), ((3, 5), 2), ((4, 3, 2), 3), ((3, 3, 5), 4), ((7, 6), 5)])
def test_link_counts_random(shape, seed):
    p = oracle.Params(shape)
    phi = inp.random_signs(shape, seed=seed)
    d = oracle.measure(p, phi, np.zeros_like(phi))
    assert (d.n_links, d.n_wall) == _brute_counts(phi < 0)


def test_negative_zero_is_nonnegative():
    """The (phi < 0) rule: +0 and -0 both count as non-negative; no link between them."""
    p = oracle.Params((4, 4))
    phi = np.full((4, 4), 0.5)
    phi[1, 1] = -0.0
    phi[2, 2] = 0.0
    assert oracle.measure(p, phi, np.zeros_like(phi)).n_links == 0
    phi[1, 2] = -1e-300
    assert oracle.measure(p, phi, np.zeros_like(phi)).n_links == 4


# --------------------------------------------------------- velocity estimator

@pytest.mark.parametrize("u", [0.3, 0.6])
def test_boosted_kink_gamma_v(u):
    """A wall moving at speed u has dphi^2/(2V) = (gamma u)^2 at every site (Eq. 8)."""
    shape = (256, 4)
    p = oracle.Params(shape)
    phi, v = inp.boosted_kink_pair(shape, 10.0, u)
    d = oracle.measure(p, phi, v)
    g = 1.0 / math.sqrt(1 - u * u)
    assert d.n_wall == 4 * shape[1] and d.n_vzero == 0
    assert d.gamma_v == pytest.approx(g * u, rel=1e-12)
    # a 3D box with the walls along z
    shape = (4, 3, 256)
    p = oracle.Params(shape)
    phi, v = inp.boosted_kink_pair(shape, 10.0, u, axis=2)
    assert oracle.measure(p, phi, v).gamma_v == pytest.approx(g * u, rel=1e-12)


def test_vzero_sites_are_skipped():
    """A wall site sitting exactly in a vacuum (V = 0) is counted apart and left out of Eq. 8."""
    p = oracle.Params((4, 4))
    phi = np.full((4, 4), 1.0)
    phi[0, 0] = -0.5
    v = np.full((4, 4), 0.2)
    d = oracle.measure(p, phi, v)
    assert d.n_wall == 5 and d.n_vzero == 4
    V = math.pi ** 2 / 200.0 * (0.25 - 1.0) ** 2
    assert d.gamma_v == pytest.approx(math.sqrt(0.04 / V / 2.0), rel=1e-14)


def test_nonfinite_count():
    p = oracle.Params((4, 4))
    phi = np.full((4, 4), 0.5)
    phi[1, 2] = np.nan
    v = np.zeros((4, 4))
    v[3, 3] = np.inf
    assert oracle.measure(p, phi, v).n_nonfinite == 2


# ----------------------------------------------------------------- adjoint

def _fd(p, phi0, v0, nsteps, obs, dphi, dv, h):
    Jp = oracle.observable(p, obs, oracle.step(p, phi0 + h * dphi, v0 + h * dv, nsteps)[0])
    Jm = oracle.observable(p, obs, oracle.step(p, phi0 - h * dphi, v0 - h * dv, nsteps)[0])
    return (Jp - Jm) / (2 * h)


@pytest.mark.parametrize("shape,obs,nsteps", [((12, 10), 0, 40), ((12, 10), 1, 30), ((6, 5, 4), 0, 25),
                                              ((6, 5, 4), 1, 20)])
def test_adjoint_against_central_differences(shape, obs, nsteps):
    """Reverse-time adjoint of Eqs. 3-5 vs central finite differences (FP64)."""
    p = oracle.Params(shape, W0=4.0, eta0=2.0)
    phi0 = 0.8 * inp.random_field(shape, seed=11)
    v0 = 0.05 * inp.random_field(shape, seed=12)
    r = oracle.adjoint(p, phi0, v0, nsteps, obs)
    assert r["J"] == oracle.observable(p, obs, oracle.step(p, phi0, v0, nsteps)[0])
    rng = np.random.Generator(np.random.PCG64(13))
    h = 1e-4 if obs == 0 else 1e-5
    for _ in range(3):
        d = rng.standard_normal(phi0.shape)
        fd = _fd(p, phi0, v0, nsteps, obs, d, 0 * d, h)
        ad = float(np.sum(r["dJ_dphi"] * d))
        assert abs(ad - fd) <= 1e-6 * max(abs(fd), 1e-3 * abs(r["J"]))
        fdv = _fd(p, phi0, v0, nsteps, obs, 0 * d, d, h)
        adv = float(np.sum(r["dJ_dv"] * d))
        assert abs(adv - fdv) <= 1e-6 * max(abs(fdv), 1e-3 * abs(r["J"]))
    # d/d alpha by central differences of the parameter
    ha = 1e-5
    pp = oracle.Params(shape, W0=4.0, eta0=2.0, alpha=p.alpha + ha)
    pm = oracle.Params(shape, W0=4.0, eta0=2.0, alpha=p.alpha - ha)
    fda = (oracle.observable(pp, obs, oracle.step(pp, phi0, v0, nsteps)[0])
           - oracle.observable(pm, obs, oracle.step(pm, phi0, v0, nsteps)[0])) / (2 * ha)
    assert abs(r["dJ_dalpha"] - fda) <= 1e-6 * max(abs(fda), 1e-3 * abs(r["J"]))


def test_observables_closed_form():
    """Gradient energy of a plane wave and the smoothed area of a kink pair."""
    shape = (16, 8)
    p = oracle.Params(shape)
    phi, _, k = inp.plane_wave(shape, (2, 0), amp=0.5)
    # sum_s (phi_{s+1}-phi_s)^2/2 = S * amp^2 * (1 - cos(k dx)) / 2
    assert oracle.observable(p, 0, phi) == pytest.approx(p.sites * 0.25 * (1 - math.cos(k[0])) / 2, rel=1e-12)
    kp, _ = inp.kink_pair((64, 4), 2.0)
    J = oracle.observable(oracle.Params((64, 4)), 1, kp, eps=1e-3)
    assert J == pytest.approx(2.0 / 64, rel=1e-6)


@pytest.mark.parametrize("shape", [(12, 12), (7, 7, 7)])
def test_diagnostics_lattice_symmetries(shape):
    """A/V, gamma v and the counts are invariant under the lattice's reflections and axis swaps.

    The Eq. 7 weight is taken at the link midpoint, so reversing a link's direction
    leaves it unchanged; a weight taken at one end only would break this.
    """
    p = oracle.Params(shape)
    phi = inp.random_field(shape, seed=21)
    v = 0.3 * inp.random_field(shape, seed=22)
    d = oracle.measure(p, phi, v)
    variants = []
    for ax in range(p.dims):
        refl = lambda f, ax=ax: np.roll(np.flip(f, axis=ax), 1, axis=ax)
        variants.append((refl(phi), refl(v)))
    variants.append((np.swapaxes(phi, 0, 1), np.swapaxes(v, 0, 1)))
    for ph, vv in variants:
        e = oracle.measure(p, np.ascontiguousarray(ph), np.ascontiguousarray(vv))
        assert (e.n_links, e.n_wall) == (d.n_links, d.n_wall)
        assert e.area_per_volume == pytest.approx(d.area_per_volume, rel=1e-13)
        assert e.gamma_v == pytest.approx(d.gamma_v, rel=1e-13)

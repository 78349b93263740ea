"""Seeded synthetic inputs shared by the oracle tests, the GPU parity tests and the benchmark.

This module holds none of the PRS method's arithmetic (no Laplacian, no kick, no
drift, no diagnostic).  It only builds initial fields with a known structure:

* ``random_field``   i.i.d. uniform values in (-1, 1) on the 24-bit grid
  (2k+1) 2^-24 - 1, drawn with numpy's PCG64 (so every value is exact in FP32);
  this matches the distribution of the paper's random initial conditions.
* ``kink_pair``      two static tanh walls (a kink at N/4 - 1/2 and an antikink at
  3N/4 - 1/2 along one axis, constant across it), zero crossings between sites.
* ``boosted_kink_pair`` the same pair moving with speed u (Lorentz-contracted).
* ``tilted_wall_pair`` the pair along the diagonal x + y of a square box.
* ``bubble``         a tanh disc (2D) or ball (3D) of radius R.
* ``plane_wave``     offset + amp * cos(k . x) with k on the lattice's Fourier grid.
* ``random_signs``   magnitudes in [0.1, 1) with a given or random sign pattern.

Arrays are numpy, shape (ny, nx) in 2D or (nz, ny, nx) in 3D: x runs fastest, the
layout of both the oracle and the library.  ``shape`` arguments are (nx, ny[, nz]).
"""
from __future__ import annotations

import math

import numpy as np


def _grid(shape):
    """Coordinate arrays x, y[, z] broadcast to the field's numpy shape."""
    axes = [np.arange(n, dtype=np.float64) for n in shape]
    mesh = np.meshgrid(*reversed(axes), indexing="ij")  # (z), y, x order
    return list(reversed(mesh))  # x, y[, z]


def random_field(shape, seed: int, dtype=np.float64) -> np.ndarray:
    """Uniform (-1, 1) values on the 24-bit grid (2k+1)/2^24 - 1, from numpy's PCG64."""
    rng = np.random.Generator(np.random.PCG64(seed))
    k = rng.integers(0, 1 << 24, size=tuple(reversed(shape)), dtype=np.int64)
    return ((2 * k + 1).astype(np.float64) / float(1 << 24) - 1.0).astype(dtype)


def random_signs(shape, seed: int, signs=None) -> np.ndarray:
    """Magnitudes in [0.1, 1) times a sign pattern (+1/-1 array of the field's shape, or random)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    fshape = tuple(reversed(shape))
    mag = 0.1 + 0.9 * rng.random(fshape)
    if signs is None:
        signs = np.where(rng.random(fshape) < 0.5, -1.0, 1.0)
    return mag * np.asarray(signs, dtype=np.float64).reshape(fshape)


def kink_pair(shape, W0: float, axis: int = 0, phi0: float = 1.0):
    """Static wall pair phi = -phi0 tanh(pi(x-x1)/W0) tanh(pi(x-x2)/W0) along ``axis``.

    x1 = N/4 - 1/2 and x2 = 3N/4 - 1/2, so no site sits on a zero.  Returns (phi, v=0).
    The field is mirror-symmetric about N/2 - 1/2 bit for bit (tanh is odd).
    """
    n = shape[axis]
    x = _grid(shape)[axis]
    x1, x2 = n / 4 - 0.5, 3 * n / 4 - 0.5
    a = math.pi / W0
    phi = -phi0 * np.tanh(a * (x - x1)) * np.tanh(a * (x - x2))
    return phi, np.zeros_like(phi)


def boosted_kink_pair(shape, W0: float, u: float, axis: int = 0):
    """Wall pair moving with speed u along ``axis`` at t = 0 (phi0 = 1).

    Each wall is tanh(pi gamma (x - x_i - u t)/W0) with gamma = 1/sqrt(1-u^2); the
    returned velocity is the time derivative of the product at t = 0.
    """
    n = shape[axis]
    x = _grid(shape)[axis]
    x1, x2 = n / 4 - 0.5, 3 * n / 4 - 0.5
    g = 1.0 / math.sqrt(1.0 - u * u)
    a = math.pi * g / W0
    A = np.tanh(a * (x - x1))
    B = -np.tanh(a * (x - x2))
    with np.errstate(over="ignore"):  # far from a wall cosh overflows and sech^2 is 0
        dA = -u * a / np.cosh(a * (x - x1)) ** 2
        dB = u * a / np.cosh(a * (x - x2)) ** 2
    return A * B, dA * B + A * dB


def tilted_wall_pair(shape, W0: float):
    """Wall pair along the diagonal lines x + y = N/4 - 1/2 and 3N/4 - 1/2 (mod N).

    The box must be square in (x, y).  Each wall wraps the torus once with length
    N sqrt(2), so the true A/V is 2 sqrt(2)/(N dx) (independent of z in 3D).
    """
    n = shape[0]
    assert shape[1] == n
    X = _grid(shape)
    s = (X[0] + X[1]) % n
    c1, c2 = n / 4 - 0.5, 3 * n / 4 - 0.5
    a = math.pi / (W0 * math.sqrt(2.0))  # perpendicular distance is (s - c)/sqrt(2)
    phi = -np.tanh(a * (s - c1)) * np.tanh(a * (s - c2))
    return phi, np.zeros_like(phi)


def bubble(shape, R: float, W0: float):
    """A tanh bubble of radius R centred in the box: phi < 0 inside, > 0 outside."""
    X = _grid(shape)
    c = [n / 2 - 0.5 for n in shape]
    r = np.sqrt(sum((X[i] - c[i]) ** 2 for i in range(len(shape))))
    phi = np.tanh(math.pi * (r - R) / W0)
    return phi, np.zeros_like(phi)


def plane_wave(shape, modes, amp: float, offset: float = 0.0, dx: float = 1.0):
    """offset + amp cos(k . x), k_i = 2 pi modes_i / (N_i dx).  Returns (phi, v=0, k)."""
    X = _grid(shape)
    k = [2 * math.pi * m / (n * dx) for m, n in zip(modes, shape)]
    ph = sum(k[i] * X[i] * dx for i in range(len(shape)))
    phi = offset + amp * np.cos(ph)
    return phi, np.zeros_like(phi), k

"""Seeded synthetic inputs shared by the tests and the benchmark.

This module holds no arithmetic of the method: it only draws seeded random
wave functions, perturbations and directions with numpy's PCG64 generator, so
that the oracle and the CUDA library can be fed identical inputs.  The random
numbers that the method itself draws (the SRP noise, the ring parameters) are
NOT made here: each side implements the counter-based SplitMix64 stream.
"""
import math

import numpy as np


def random_psi(n, seed, amp_jitter=0.3, shape=None):
    """Complex128 field with |psi| around 1 (jittered) and uniform random phase."""
    rng = np.random.default_rng(seed)
    shape = (n, n, n) if shape is None else shape
    mag = 1.0 + amp_jitter * rng.standard_normal(shape)
    ph = 2.0 * math.pi * rng.random(shape)
    return mag * np.exp(1j * ph)


def random_direction(n, seed, complex_valued=True):
    rng = np.random.default_rng(seed)
    if complex_valued:
        v = rng.standard_normal((n, n, n)) + 1j * rng.standard_normal((n, n, n))
    else:
        v = rng.standard_normal((n, n, n))
    return v / math.sqrt(float(np.mean(np.abs(v) ** 2)))


def smooth_psi(n, seed, nmodes=6, kmax=3, amp=0.25):
    """1 + a few low Fourier modes (band-limited, no zeros for the default amplitude)."""
    rng = np.random.default_rng(seed)
    x = 2.0 * math.pi * np.arange(n) / n
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    psi = np.ones((n, n, n), dtype=np.complex128)
    for _ in range(nmodes):
        k = rng.integers(-kmax, kmax + 1, size=3)
        c = amp / nmodes * (rng.standard_normal() + 1j * rng.standard_normal())
        psi += c * np.exp(1j * (k[0] * X + k[1] * Y + k[2] * Z))
    return psi


def grid_coords(n):
    x = 2.0 * math.pi * np.arange(n) / n
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    return X, Y, Z


def smooth_phase(n, seed, nmodes=24, kmax=4, rms=math.pi):
    """A real periodic phase field: a few random low Fourier modes scaled to the given RMS."""
    rng = np.random.default_rng(seed)
    x = 2.0 * math.pi * np.arange(n) / n
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    th = np.zeros((n, n, n))
    for _ in range(nmodes):
        k = rng.integers(-kmax, kmax + 1, size=3)
        th += rng.standard_normal() * np.cos(k[0] * X + k[1] * Y + k[2] * Z + 2.0 * math.pi * rng.random())
    return th * (rms / math.sqrt(float(np.mean(th ** 2))))

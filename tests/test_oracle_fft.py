"""Pins for the oracle FFT: brute-force DFT, numpy.fft, Parseval, round trip, closed forms."""
import itertools

import numpy as np
import pytest

from oracle import fft

SIZES = sorted({2 ** a * 3 ** b for a in range(6) for b in range(4) if 2 ** a * 3 ** b <= 48})


@pytest.mark.parametrize("n", SIZES + [5, 7, 10])
def test_fft1_matches_bruteforce(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal((3, n)) + 1j * rng.standard_normal((3, n))
    ref = fft.dft_brute(x, -1)
    got = fft.fft1(x)
    assert np.max(np.abs(got - ref)) <= 1e-13 * max(1.0, np.max(np.abs(ref)))
    back = fft.ifft1(got)
    assert np.max(np.abs(back - x)) <= 1e-13 * np.max(np.abs(x))


@pytest.mark.parametrize("shape", [(4, 6, 8), (3, 4, 2), (6, 6, 6), (8, 8, 8), (12, 12, 12)])
def test_fft3_matches_full_matrix_definition(shape):
    """3D DFT from the definition X[k] = sum_x f[x] exp(-i k . x), built as one dense matrix."""
    rng = np.random.default_rng(sum(shape))
    f = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    nz, ny, nx = shape
    pts = np.array(list(itertools.product(range(nz), range(ny), range(nx))), dtype=np.float64)
    scale = np.array([2 * np.pi / nz, 2 * np.pi / ny, 2 * np.pi / nx])
    M = np.exp(-1j * (pts * scale) @ pts.T)          # symmetric: (k * 2pi/n) . x
    ref = (M @ f.ravel()).reshape(shape)
    got = fft.fft3(f)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("n", [8, 12, 16, 24, 32])
def test_fft3_matches_numpy(n):
    rng = np.random.default_rng(100 + n)
    f = rng.standard_normal((n, n, n)) + 1j * rng.standard_normal((n, n, n))
    ref = np.fft.fftn(f)
    assert np.max(np.abs(fft.fft3(f) - ref)) <= 1e-12 * np.max(np.abs(ref))
    assert np.max(np.abs(fft.ifft3(ref) - f)) <= 1e-12 * np.max(np.abs(f))


def test_parseval_and_closed_forms():
    n = 12
    rng = np.random.default_rng(7)
    f = rng.standard_normal((n, n, n)) + 1j * rng.standard_normal((n, n, n))
    F = fft.fft3(f)
    assert abs(np.sum(np.abs(F) ** 2) / f.size - np.sum(np.abs(f) ** 2)) <= 1e-10 * np.sum(np.abs(f) ** 2)
    imp = np.zeros((n, n, n), complex)
    imp[0, 0, 0] = 1.0
    assert np.max(np.abs(fft.fft3(imp) - 1.0)) < 1e-14
    x = 2 * np.pi * np.arange(n) / n
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    mode = np.exp(1j * (2 * X - 3 * Y + 5 * Z))
    M = fft.fft3(mode)
    expect = np.zeros((n, n, n), complex)
    expect[5 % n, (-3) % n, 2] = n ** 3
    assert np.max(np.abs(M - expect)) < 1e-9

"""Oracle FFT: recursive decimation-in-time DFT for lengths 2^a * 3^b (any length works).

Test infrastructure only (see ``oracle/__init__``).

Convention (the one the pseudo-spectral scheme of Sec. 4.3 uses, with the
discrete transform standing in for the continuous one of Sec. 3.5):
    forward   X[k] = sum_j x[j] exp(-2 pi i j k / n)          (unnormalised)
    inverse   x[j] = (1/n) sum_k X[k] exp(+2 pi i j k / n)

The recursion: for a prime factor p of n, split x by residue r = j mod p,
transform each of the p sub-sequences of length m = n/p, and recombine with
X[k] = sum_r w^{r k} S_r[k mod m], w = exp(sign 2 pi i / n).  Lengths with a
prime factor other than 2 or 3 fall back to the O(n^2) definition.
"""
import numpy as np


def _dft_last(a, sign):
    n = a.shape[-1]
    if n == 1:
        return np.array(a, dtype=np.complex128, copy=True)
    p = 2 if n % 2 == 0 else (3 if n % 3 == 0 else 0)
    if p == 0:
        j = np.arange(n)
        w = np.exp(sign * 2j * np.pi * np.outer(j, j) / n)
        return np.asarray(a, dtype=np.complex128) @ w
    m = n // p
    k = np.arange(n)
    out = np.zeros(a.shape, dtype=np.complex128)
    for r in range(p):
        s = _dft_last(a[..., r::p], sign)
        out += np.tile(s, p) * np.exp(sign * 2j * np.pi * ((r * k) % n) / n)
    return out


def dft_brute(x, sign=-1):
    """O(n^2) DFT along the last axis straight from the definition (used as a pin)."""
    x = np.asarray(x, dtype=np.complex128)
    n = x.shape[-1]
    j = np.arange(n)
    return x @ np.exp(sign * 2j * np.pi * ((np.outer(j, j)) % n) / n)


def fft1(x, axis=-1):
    """Unnormalised forward DFT along one axis."""
    x = np.moveaxis(np.asarray(x, dtype=np.complex128), axis, -1)
    return np.moveaxis(_dft_last(x, -1), -1, axis)


def ifft1(x, axis=-1):
    """Inverse DFT along one axis, including the 1/n factor."""
    x = np.moveaxis(np.asarray(x, dtype=np.complex128), axis, -1)
    n = x.shape[-1]
    return np.moveaxis(_dft_last(x, +1) / n, -1, axis)


def fft3(x):
    """Unnormalised forward 3D DFT of an array indexed [z, y, x]."""
    out = np.asarray(x, dtype=np.complex128)
    for ax in (2, 1, 0):
        out = fft1(out, ax)
    return out


def ifft3(x):
    """Inverse 3D DFT (with the 1/n factor) of an array indexed [kz, ky, kx]."""
    out = np.asarray(x, dtype=np.complex128)
    for ax in (2, 1, 0):
        out = ifft1(out, ax)
    return out

"""The float32 arithmetic fact behind the kinetic factor's product order (twmul_k in the CUDA
source): a compensated complex product a * (c + i s),
applied again and again by the same small angle, gains |a|^2 steadily when a component's small
terms are first summed against its larger product alone and rounded there, and does not when the
larger product is added last.  Pure numpy emulation of float32 FMA (the exact product of two
floats fits a float64; the sum is rounded once to float32); no part of the library or the oracle."""
import numpy as np


def _fma(a, b, c):
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(np.float32)


def _split12(v):
    """hi with 12 significant bits, lo = the float remainder (the tables' hi + lo split)."""
    m, e = np.frexp(v)
    h = np.ldexp(np.round(m * 4096.0) / 4096.0, e)
    return h.astype(np.float32), (v - h).astype(np.float32)


def _mul(ax, ay, w, larger_last):
    (cx, cl), (sx, sl) = w
    re_lo = _fma(ax, cl, (-ay * sl).astype(np.float32))
    im_lo = _fma(ax, sl, (ay * cl).astype(np.float32))
    if not larger_last:   # both components in the fixed order of the FFT twiddle product
        return _fma(ax, cx, _fma(-ay, sx, re_lo)), _fma(ax, sx, _fma(ay, cx, im_lo))
    cb = np.abs(cx) >= np.abs(sx)
    re = np.where(cb, _fma(ax, cx, _fma(-ay, sx, re_lo)), _fma(-ay, sx, _fma(ax, cx, re_lo)))
    im = np.where(cb, _fma(ay, cx, _fma(ax, sx, im_lo)), _fma(ax, sx, _fma(ay, cx, im_lo)))
    return re, im


def _gain(theta, larger_last, steps=200, m=100_000, seed=3):
    rng = np.random.default_rng(seed)
    ax = rng.standard_normal(m).astype(np.float32)
    ay = rng.standard_normal(m).astype(np.float32)
    m0 = np.sum(ax.astype(np.float64) ** 2 + ay.astype(np.float64) ** 2)
    w = (_split12(np.full(m, np.cos(theta))), _split12(np.full(m, -np.sin(theta))))
    for _ in range(steps):
        ax, ay = _mul(ax, ay, w, larger_last)
    return np.sum(ax.astype(np.float64) ** 2 + ay.astype(np.float64) ** 2) / m0 - 1.0


def test_small_terms_rounded_against_the_larger_product_gain_magnitude():
    """At 2.5e-4 rad (a slow mode's kinetic phase per step) the fixed order gains ~3e-6 over 200
    steps; with the larger product added last the change is at the noise (~1e-9), as it is for
    both orders at a large angle."""
    assert _gain(2.5e-4, larger_last=False) > 1e-6
    assert abs(_gain(2.5e-4, larger_last=True)) < 2e-8
    assert abs(_gain(np.pi - 2e-4, larger_last=True)) < 2e-8
    assert abs(_gain(np.pi / 2 - 1e-4, larger_last=True)) < 2e-8
    assert abs(_gain(1.0, larger_last=False)) < 2e-8


def _nonlinear(ax, ay, coef, small_terms_first):
    """One small-phase nonlinear flow a exp(-i coef (|a|^2 - 1)) in float32, with cos - 1 and sin
    rounded once from float64 (the kernel's Taylor chains agree with them to an ulp)."""
    r2 = _fma(ax, ax, (ay * ay).astype(np.float32))
    ph = (np.float32(coef) * (r2 - np.float32(1))).astype(np.float32)
    sn = np.sin(ph.astype(np.float64)).astype(np.float32)
    cm1 = (np.cos(ph.astype(np.float64)) - 1.0).astype(np.float32)
    if small_terms_first:   # the kernel's order: a.x + (a.y sin + a.x (cos - 1)), one rounding each
        ur = _fma(ay, sn, (ax * cm1).astype(np.float32))
        ui = _fma(-ax, sn, (ay * cm1).astype(np.float32))
        return (ax + ur).astype(np.float32), (ay + ui).astype(np.float32)
    return _fma(ax, cm1, _fma(ay, sn, ax)), _fma(ay, cm1, _fma(-ax, sn, ay))


def _nonlinear_gain(dev, small_terms_first, steps=200, m=100_000, seed=5, coef=0.06):
    rng = np.random.default_rng(seed)
    r = np.sqrt(1.0 + dev * rng.uniform(-1.0, 1.0, m))
    th = rng.uniform(0.0, 2.0 * np.pi, m)
    ax, ay = (r * np.cos(th)).astype(np.float32), (r * np.sin(th)).astype(np.float32)
    m0 = np.sum(ax.astype(np.float64) ** 2 + ay.astype(np.float64) ** 2)
    for _ in range(steps):
        ax, ay = _nonlinear(ax, ay, coef, small_terms_first)
    return np.sum(ax.astype(np.float64) ** 2 + ay.astype(np.float64) ** 2) / m0 - 1.0


def test_nonlinear_small_phase_sums_its_small_terms_first():
    """Points with |a|^2 within 4e-3 of 1 at beta dt = 0.06 turn by at most 2.4e-4 rad per step.
    Adding the sine term to the component first and the shrink a (cos - 1) after it gains ~4e-6
    of the mass over 200 steps; with the two small terms summed first and the component added last
    (the kernel's order) the change is ~70x smaller."""
    old = _nonlinear_gain(4e-3, small_terms_first=False)
    new = _nonlinear_gain(4e-3, small_terms_first=True)
    assert old > 1e-6
    assert abs(new) < old / 30
    assert abs(_nonlinear_gain(0.2, small_terms_first=True)) < 1e-8

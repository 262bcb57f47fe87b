"""Pins for the oracle helicities (Sec. 3.6: eq-helicity, Hreg): the Beltrami ABC flow, the
axial velocity of a straight vortex line, mirror and conjugation symmetry, the Taylor-Green start
field (zero by symmetry, as the paper's TG table reports), and the spectra's sums."""
import math

import numpy as np
import pytest

from inputs import grid_coords, random_psi
from oracle import argle as OA
from oracle import helicity as HL
from oracle import scheme as S


def _p(n, alpha=None):
    p = S.params_from_dx_ratio(n, 1.5, 0.01)
    return p if alpha is None else S.Params(n=n, alpha=alpha, beta=p.beta, dt=p.dt)


def test_abc_flow_is_beltrami_with_the_classical_helicity():
    """v = v^(1) + v^(2) of the ABC flow: curl v^(k) = k v^(k), so curl v = v^(1) + 2 v^(2) and
    <v . curl v> = 3 (A^2 + B^2 + C^2) (the two modes are orthogonal)."""
    n = 16
    X, Y, Z = grid_coords(n)
    A, B, C = OA.ABC_DEFAULT
    v = OA.abc_velocity(X, Y, Z)
    v1 = [B * np.cos(Y) + C * np.sin(Z), C * np.cos(Z) + A * np.sin(X), A * np.cos(X) + B * np.sin(Y)]
    om = HL.curl(v)
    for j in range(3):
        assert np.max(np.abs(om[j] - (2 * v[j] - v1[j]))) < 1e-13
    assert HL.helicity_of(v) == pytest.approx(3 * (A * A + B * B + C * C), rel=1e-13)


def test_curl_of_a_gradient_vanishes():
    n = 16
    X, Y, Z = grid_coords(n)
    phi = np.sin(X + 2 * Y) * np.cos(3 * Z) + np.cos(2 * X - Z)
    v = [np.cos(X + 2 * Y) * np.cos(3 * Z) - 2 * np.sin(2 * X - Z),
         2 * np.cos(X + 2 * Y) * np.cos(3 * Z),
         -3 * np.sin(X + 2 * Y) * np.sin(3 * Z) + np.sin(2 * X - Z)]
    assert phi.shape == v[0].shape
    for c in HL.curl(v):
        assert np.max(np.abs(c)) < 1e-12


def _line_vortex_derivatives(pts, e1, e2, e3, m, winding):
    """Exact first and second derivatives of psi = (x.e1 + i s x.e2) exp(i m x.e3) (s = winding):
    a straight vortex line along e3 carrying the axial velocity 2 alpha m."""
    e2 = winding * np.asarray(e2)
    u = pts @ e1 + 1j * (pts @ e2)
    ph = np.exp(1j * m * (pts @ e3))
    a = e1 + 1j * e2                                   # grad of u
    grad = [(a[q] + 1j * m * e3[q] * u) * ph for q in range(3)]
    hess = {}
    for i in range(3):
        for j in range(i, 3):
            hess[(i, j)] = (1j * m * e3[j] * a[i] + 1j * m * e3[i] * a[j] - m * m * e3[i] * e3[j] * u) * ph
    return grad, hess


@pytest.mark.parametrize("winding", [1, -1])
def test_regularised_velocity_on_a_vortex_line_is_the_axial_velocity(winding):
    """On the core of a straight vortex line along e3 (any orientation, either winding) with the
    phase m x.e3, v_par w/|w| is the axial velocity 2 alpha m e3 (the finite part of v that the
    regularisation keeps); off the core it tends to the same value as the distance goes to 0."""
    alpha, m = 0.07, 1.7
    rng = np.random.default_rng(2)
    Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    e1, e2, e3 = Q[:, 0], Q[:, 1], np.cross(Q[:, 0], Q[:, 1])
    t = np.linspace(-2.0, 3.0, 7)
    on = t[:, None] * e3[None, :]
    grad, hess = _line_vortex_derivatives(on, e1, e2, e3, m, winding)
    vr = HL.v_reg(grad, hess, alpha)
    for q in range(3):
        assert np.max(np.abs(vr[q] - 2 * alpha * m * e3[q])) < 1e-13
    for eps in (1e-3, 1e-5):
        off = on + eps * (0.6 * e1 + 0.8 * e2)[None, :]
        grad, hess = _line_vortex_derivatives(off, e1, e2, e3, m, winding)
        vr = HL.v_reg(grad, hess, alpha)
        for q in range(3):
            assert np.max(np.abs(vr[q] - 2 * alpha * m * e3[q])) < 10 * eps


def test_w_is_the_curl_of_the_mass_current():
    """w = (2 alpha / i) grad psi* x grad psi equals curl(rho v) = curl(2 alpha Im(psi* grad psi))
    (the curl of a gradient drops out); checked on a field band-limited to |k_j| <= 3, whose
    products stay below the Nyquist wavenumber of a 16^3 grid, so that both sides are exact."""
    from inputs import smooth_psi
    from oracle.diagnostics import gradient
    n = 16
    p = _p(n)
    psi = smooth_psi(n, 5, amp=2.0)
    g = gradient(psi)
    w = HL.w_field(g, p.alpha)
    cj = HL.curl([2 * p.alpha * np.imag(np.conj(psi) * gj) for gj in g])
    for q in range(3):
        assert np.max(np.abs(w[q])) > 1e-3
        assert np.max(np.abs(w[q] - cj[q])) < 1e-12 * np.max(np.abs(w[q]))


def _mirror_x(psi):
    n = psi.shape[2]
    return psi[:, :, (-np.arange(n)) % n]


def test_helicities_are_pseudoscalars():
    """x -> -x reverses both helicities; psi -> conj(psi) (every velocity reversed) keeps them."""
    n = 16
    p = _p(n)
    psi = random_psi(n, 8, amp_jitter=0.3)
    (h, hr), _ = HL.helicities(psi, p, with_spectra=False)
    (hm, hrm), _ = HL.helicities(_mirror_x(psi), p, with_spectra=False)
    (hc, hrc), _ = HL.helicities(np.conj(psi), p, with_spectra=False)
    assert abs(h) > 1e-6 and abs(hr) > 1e-6
    assert hm == pytest.approx(-h, rel=1e-10) and hrm == pytest.approx(-hr, rel=1e-10)
    assert hc == pytest.approx(h, rel=1e-10) and hrc == pytest.approx(hr, rel=1e-10)


@pytest.mark.parametrize("steps", [0, 40])
def test_taylor_green_fields_have_no_helicity(steps):
    """The TG start field is even under x -> -x, and so is every ARGLE step driven by the TG flow,
    so both helicities vanish to round-off (the paper's TG ARGLE table prints 1e-13 and 1e-11 for
    its converged 128^3 field).  The start field's nodal lines have winding 3, the stepped ones
    are splitting: both contain symmetry planes on which grad psi is round-off, which the cut of
    the regularised velocity removes."""
    n = 32
    p = _p(n, alpha=0.05)
    psi = OA.tg_ansatz(n, 0.05, 40.0)
    if steps:
        psi = OA.argle(psi, 0.05, 40.0, 0.0125, steps, OA.velocity("tg", n))
    assert np.max(np.abs(_mirror_x(psi) - psi)) < 1e-12
    (h, hr), _ = HL.helicities(psi, p, with_spectra=False)
    assert abs(h) < 1e-10 and abs(hr) < 1e-10


def test_vortex_free_field_has_no_helicity():
    """psi = exp(i theta) with a smooth, band-limited theta: v = 2 alpha grad theta, omega = 0."""
    n = 24
    p = _p(n)
    X, Y, Z = grid_coords(n)
    psi = np.exp(0.2j * (np.sin(X) * np.cos(Y) + np.sin(Z)))
    (h, hr), _ = HL.helicities(psi, p, with_spectra=False)
    assert abs(h) < 1e-12 and abs(hr) < 1e-12


def test_spectra_add_up_to_the_totals():
    n = 16
    p = _p(n)
    psi = random_psi(n, 12, amp_jitter=0.3)
    (h, hr), (sh, shr) = HL.helicities(psi, p)
    assert len(sh) == len(shr) == int(math.floor(math.sqrt(3) * n / 2 + 0.5)) + 1
    assert np.sum(sh) == pytest.approx(h, rel=1e-10, abs=1e-14)
    assert np.sum(shr) == pytest.approx(hr, rel=1e-10, abs=1e-14)

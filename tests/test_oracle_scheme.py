"""Pins for the oracle split step (Sec. 4.3): exact solutions, invariants, identities."""
import math

import numpy as np
import pytest

from inputs import random_psi, smooth_psi
from oracle import diagnostics as D
from oracle import scheme as S


def _plane_wave(n, k, A):
    x = 2 * np.pi * np.arange(n) / n
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    return A * np.exp(1j * (k[0] * X + k[1] * Y + k[2] * Z))


def test_parameters_match_paper_table():
    """alpha = 0.05 gives beta = 40 and xi = 0.035355 (Sec. 6, parameter table, case _a)."""
    p = S.params_from_xi(128, 0.05 / math.sqrt(2.0), 1e-3)
    assert abs(p.alpha - 0.05) < 1e-15 and abs(p.beta - 40.0) < 1e-12
    assert abs(p.xi - 0.0353553) < 1e-7
    # xi k_max = (N/2) sqrt(2) alpha M with M = 1/2 (eq-scaling-choice3): 64 * sqrt(2) * 0.05 * 0.5
    assert abs(p.xi * 64 - 64 * math.sqrt(2) * 0.05 * 0.5) < 1e-12


@pytest.mark.parametrize("order", ["nkn", "knk"])
@pytest.mark.parametrize("k,A", [((1, 2, -3), 1.0), ((4, 0, -1), 0.7), ((0, 0, 0), 1.3)])
def test_plane_wave_is_exact(order, k, A):
    """Both sub-flows act exactly on plane waves: psi_m = psi_0 exp(-i omega m dt),
    omega = alpha |k|^2 + beta (|A|^2 - 1)."""
    n = 12
    p = S.params_from_dx_ratio(n, 1.5, 0.01)
    psi0 = _plane_wave(n, k, A)
    m = 25
    psi = S.evolve(psi0, p, m, order)
    om = p.alpha * sum(c * c for c in k) + p.beta * (A * A - 1.0)
    assert np.max(np.abs(psi - psi0 * np.exp(-1j * om * m * p.dt))) < 1e-12


@pytest.mark.parametrize("order", ["nkn", "knk"])
def test_linear_limit_matches_exact_propagator(order):
    """beta = 0: the scheme is the exact solution F^-1 exp(-i alpha |k|^2 t) F psi0 (numpy.fft)."""
    n = 12
    p = S.Params(n=n, alpha=0.3, beta=0.0, dt=0.02)
    psi0 = random_psi(n, 3)
    psi = S.evolve(psi0, p, 10, order)
    k = np.fft.fftfreq(n, 1.0 / n)
    k2 = k[:, None, None] ** 2 + k[None, :, None] ** 2 + k[None, None, :] ** 2
    exact = np.fft.ifftn(np.exp(-1j * p.alpha * k2 * 10 * p.dt) * np.fft.fftn(psi0))
    assert np.max(np.abs(psi - exact)) < 1e-12


def test_uniform_state_is_stationary():
    p = S.params_from_dx_ratio(8, 2.0, 0.005)
    psi = S.evolve(np.ones((8, 8, 8), complex), p, 20)
    assert np.max(np.abs(psi - 1.0)) < 1e-14


def test_dark_soliton_pair_is_stationary():
    """psi = -tanh((x-pi/2)/(sqrt2 xi)) tanh((x-3pi/2)/(sqrt2 xi)): each tanh solves
    -alpha psi'' + beta (psi^2 - 1) psi = 0 exactly, so the pair is stationary up to the
    soliton interaction (~exp(-pi/(sqrt2 xi)), 1.5e-7 here) and the O(dt^2) splitting error."""
    n, T = 128, 0.5
    errs = []
    for dt in (0.005, 0.0025):
        p = S.params_from_xi(n, 0.2 / math.sqrt(2.0), dt)
        x = 2 * np.pi * np.arange(n) / n
        a = math.sqrt(2.0) * p.xi
        prof = -np.tanh((x - 0.5 * np.pi) / a) * np.tanh((x - 1.5 * np.pi) / a)
        psi0 = prof.reshape(1, 1, n).astype(complex)
        errs.append(np.max(np.abs(S.evolve(psi0, p, int(round(T / dt))) - psi0)))
    assert errs[0] < 2e-4 and 3.8 < errs[0] / errs[1] < 4.2, errs
    # the wrong sign of the nonlinearity destroys it
    bad = S.Params(n=n, alpha=p.alpha, beta=-p.beta, dt=p.dt)
    assert np.max(np.abs(S.evolve(psi0, bad, 100) - psi0)) > 1e-2


@pytest.mark.parametrize("order", ["nkn", "knk"])
def test_bogoliubov_dispersion(order):
    """1 + eps cos(k x) oscillates at the split scheme's discrete frequency
    cos(w dt) = cos(alpha k^2 dt) - beta dt sin(alpha k^2 dt), which tends to the
    Bogoliubov omega^2 = alpha k^2 (alpha k^2 + 2 beta) (Sec. 3.2) as dt -> 0."""
    n, kk, eps = 32, 5, 1e-6
    p = S.Params(n=n, alpha=0.2, beta=5.0, dt=0.004)
    x = 2 * np.pi * np.arange(n) / n
    psi = (1.0 + eps * np.cos(kk * x)).reshape(1, 1, n).astype(complex)
    amp = []
    for _ in range(800):
        amp.append(np.real(np.fft.fft(psi[0, 0])[kk]) / n)
        psi = S.evolve(psi, p, 1, order)
    a = np.array(amp)
    c_fit = np.sum(a[1:-1] * (a[2:] + a[:-2])) / (2.0 * np.sum(a[1:-1] ** 2))
    th = p.alpha * kk * kk * p.dt
    c_scheme = math.cos(th) - p.beta * p.dt * math.sin(th)
    assert abs(c_fit - c_scheme) < 1e-9
    w_scheme = math.acos(c_scheme) / p.dt
    w_bog = math.sqrt(p.alpha * kk * kk * (p.alpha * kk * kk + 2 * p.beta))
    assert abs(w_scheme - w_bog) / w_bog < (w_bog * p.dt) ** 2
    assert 800 * p.dt * w_bog / (2 * math.pi) > 3.0          # more than three periods fitted


def test_mass_is_conserved_to_roundoff():
    n = 16
    p = S.params_from_dx_ratio(n, 1.5, 0.004)
    psi0 = random_psi(n, 11)
    m0 = D.mass(psi0)
    psi = S.evolve(psi0, p, 100)
    assert abs(D.mass(psi) - m0) / m0 < 1e-13


def test_energy_drift_is_second_order():
    """max |E - E0| over a fixed time T falls by ~4x when dt is halved."""
    n = 16
    T = 0.4
    drifts = []
    for dt in (0.02, 0.01, 0.005):
        p = S.params_from_dx_ratio(n, 2.0, dt)
        psi = smooth_psi(n, 5, amp=0.4)
        e0 = D.energy(psi, p)
        worst = 0.0
        for _ in range(int(round(T / dt))):
            psi = S.step_nkn(psi, p)
            worst = max(worst, abs(D.energy(psi, p) - e0) / e0)
        drifts.append(worst)
    slopes = [math.log2(drifts[i] / drifts[i + 1]) for i in range(2)]
    assert all(1.7 < s < 2.3 for s in slopes), (drifts, slopes)


@pytest.mark.parametrize("order", ["nkn", "knk"])
def test_time_reversibility(order):
    n = 12
    p = S.params_from_dx_ratio(n, 1.5, 0.01)
    back = S.Params(n=n, alpha=p.alpha, beta=p.beta, dt=-p.dt)
    psi0 = random_psi(n, 21)
    psi = S.evolve(S.evolve(psi0, p, 15, order), back, 15, order)
    assert np.max(np.abs(psi - psi0)) < 1e-12


def test_knk_nkn_identity():
    """KNK^m = (A o B) o NKN^(m-1) o (B o A), A = K(dt/2), B = N(dt/2)."""
    n = 12
    p = S.params_from_dx_ratio(n, 1.5, 0.01)
    psi0 = random_psi(n, 31)
    m = 6
    lhs = S.evolve(psi0, p, m, "knk")
    rhs = S.nonlinear_flow(S.kinetic_flow(psi0, p, 0.5 * p.dt), p, 0.5 * p.dt)
    rhs = S.evolve(rhs, p, m - 1, "nkn")
    rhs = S.kinetic_flow(S.nonlinear_flow(rhs, p, 0.5 * p.dt), p, 0.5 * p.dt)
    assert np.max(np.abs(lhs - rhs)) < 1e-12


def test_minus_one_is_a_global_phase():
    n = 12
    p1 = S.params_from_dx_ratio(n, 1.5, 0.01)
    p0 = S.Params(n=n, alpha=p1.alpha, beta=p1.beta, dt=p1.dt, minus_one=False)
    psi0 = random_psi(n, 41)
    m = 9
    a = S.evolve(psi0, p1, m)
    b = S.evolve(psi0, p0, m)
    assert np.max(np.abs(a - np.exp(1j * p1.beta * m * p1.dt) * b)) < 1e-12


def test_directional_flows_equal_3d_propagator():
    n = 12
    p = S.params_from_dx_ratio(n, 1.5, 0.01)
    psi0 = random_psi(n, 51)
    k = np.fft.fftfreq(n, 1.0 / n)
    k2 = k[:, None, None] ** 2 + k[None, :, None] ** 2 + k[None, None, :] ** 2
    exact = np.fft.ifftn(np.exp(-1j * p.alpha * k2 * 0.37) * np.fft.fftn(psi0))
    assert np.max(np.abs(S.kinetic_flow(psi0, p, 0.37) - exact)) < 1e-12


@pytest.mark.parametrize("order", ["nkn", "knk"])
def test_split_step_parametric_instability(order):
    """Where c = cos(alpha k^2 dt) - beta dt sin(alpha k^2 dt) falls below -1 the same discrete
    relation has no real frequency: a perturbation of the uniform state at that k grows by
    |c| + sqrt(c^2 - 1) per step -- most, 1 + beta dt to first order, at alpha k^2 dt =
    pi - atan(beta dt) -- although every sub-flow is unitary.  Just outside that band it stays
    bounded."""
    n, kk, eps, b, dt = 16, 4, 1e-9, 0.1, 2.0
    x = 2 * np.pi * np.arange(n) / n
    th = math.pi - math.atan(b)
    p = S.Params(n=n, alpha=th / (kk * kk * dt), beta=b / dt, dt=dt)
    psi = (1.0 + eps * np.cos(kk * x)).reshape(1, 1, n).astype(complex)
    amp = []
    for _ in range(61):
        amp.append(abs(np.fft.fft(psi[0, 0])[kk]) / n)
        psi = S.evolve(psi, p, 1, order)
    c = math.cos(th) - b * math.sin(th)
    assert c < -1.0
    growth = abs(c) + math.sqrt(c * c - 1.0)
    assert abs((amp[60] / amp[40]) ** (1.0 / 20) - growth) < 1e-6
    assert amp[60] < 1e-6                          # still the linear regime
    th2 = math.pi - 3.0 * b                        # outside the band: |c| < 1
    p2 = S.Params(n=n, alpha=th2 / (kk * kk * dt), beta=b / dt, dt=dt)
    psi = (1.0 + eps * np.cos(kk * x)).reshape(1, 1, n).astype(complex)
    worst = 0.0
    for _ in range(200):
        psi = S.evolve(psi, p2, 1, order)
        worst = max(worst, abs(np.fft.fft(psi[0, 0])[kk]) / n)
    assert worst < 2.0 * eps


def _unstable_shells(n, xi_over_dx, dt):
    """Integer |k|^2 on the n^3 grid (up to 3 (n/2)^2) whose discrete Bogoliubov relation has
    c < -1, for xi = xi_over_dx * dx and the paper's alpha = sqrt(2) xi, beta = 2 / alpha."""
    p = S.params_from_dx_ratio(n, xi_over_dx, dt)
    k2 = np.arange(3 * (n // 2) ** 2 + 1, dtype=np.float64)
    th = p.alpha * k2 * dt
    c = np.cos(th) - p.beta * dt * np.sin(th)
    return k2[c < -1.0]


def test_configured_time_steps_and_the_instability_band():
    """The benchmark's 256^3 run (xi = 1.5 dx, dt = 0.002) has wavenumbers in the band -- in the
    corners of the cube, |k| between 169 and 174 -- and so does the 128^3 run at dt = 0.004;
    halving either step takes every grid wavenumber out of it."""
    bad = _unstable_shells(256, 1.5, 0.002)
    assert bad.size > 0 and 169.0 < math.sqrt(bad.min()) and math.sqrt(bad.max()) < 174.0
    assert _unstable_shells(128, 1.5, 0.004).size > 0
    assert _unstable_shells(256, 1.5, 0.001).size == 0
    assert _unstable_shells(128, 1.5, 0.002).size == 0

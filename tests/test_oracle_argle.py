"""Pins of the oracle's imaginary-time (ARGLE) step and of the Taylor-Green / ABC start fields:
closed forms of the semi-implicit step, exact stationary states, the energy's closed forms and
its decrease, the Clebsch identity, the paper's winding numbers, the ABC flow's Beltrami
property."""
import math

import numpy as np
import pytest

from inputs import smooth_psi
from oracle import argle as OA
from oracle import diagnostics as OD
from oracle import fft
from oracle.scheme import Params, wavenumbers, wavenumbers_deriv


def _zero_v(n):
    z = np.zeros((n, n, n))
    return z, z, z


def test_linear_modes_follow_the_semi_implicit_factor():
    """beta = 0, v = 0: each Fourier mode is multiplied by (1 - a)/(1 + a), a = dtau alpha |k|^2 / 2
    (the half-implicit Laplacian), exactly."""
    n, alpha, dtau = 12, 0.3, 0.05
    X, Y, Z = OA.coords(n)
    modes = [((1, 0, 0), 0.7), ((2, -3, 1), 0.4 - 0.2j), ((0, 5, -6), 0.1j)]
    phi = sum(c * np.exp(1j * (kx * X + ky * Y + kz * Z)) for (kx, ky, kz), c in modes)
    out = OA.argle_step(phi, alpha, 0.0, dtau, _zero_v(n))
    ref = 0
    for (kx, ky, kz), c in modes:
        k2 = float(kx * kx + ky * ky + kz * kz)
        a = 0.5 * dtau * alpha * k2
        ref = ref + c * (1 - a) / (1 + a) * np.exp(1j * (kx * X + ky * Y + kz * Z))
    assert np.max(np.abs(out - ref)) < 1e-13


def test_uniform_state_is_stationary():
    n = 8
    phi = np.ones((n, n, n), dtype=complex)
    out = OA.argle(phi, 0.1, 20.0, 0.01, 5, _zero_v(n))
    assert np.max(np.abs(out - 1.0)) < 1e-14


@pytest.mark.parametrize("k0", [(1, -2, 3), (0, 4, 0)])
def test_plane_wave_in_matching_uniform_flow_is_stationary(k0):
    """v = 2 alpha k0 (uniform, divergence free) and phi = exp(i k0.x): alpha lap - i v.grad
    - |v|^2/(4 alpha) cancels exactly on phi, and |phi| = 1 -- for the discrete step too."""
    n, alpha, beta, dtau = 12, 0.2, 10.0, 0.02
    X, Y, Z = OA.coords(n)
    phi = np.exp(1j * (k0[0] * X + k0[1] * Y + k0[2] * Z))
    v = tuple(2.0 * alpha * k0[j] * np.ones_like(X) for j in range(3))
    out = OA.argle(phi, alpha, beta, dtau, 4, v)
    assert np.max(np.abs(out - phi)) < 1e-12
    assert abs(OA.energy_v(phi, alpha, beta, v)) < 1e-24


def test_energy_v_without_flow_is_the_gp_energy():
    """v = 0: E_v is eq-scaling-energy (band-limited field: no Nyquist content, so the first-
    derivative and Laplacian conventions agree)."""
    n, alpha, beta = 16, 0.15, 13.0
    psi = smooth_psi(n, 3)
    e = OA.energy_v(psi, alpha, beta, _zero_v(n))
    assert e == pytest.approx(OD.energy(psi, Params(n=n, alpha=alpha, beta=beta, dt=0.0)), rel=1e-12)


def test_energy_v_is_the_discrete_sum_written_out():
    """E_v against a direct evaluation: spectral gradient by an explicit Fourier series sum."""
    n, alpha, beta = 6, 0.3, 5.0
    rng = np.random.default_rng(7)
    phi = rng.normal(size=(n, n, n)) + 1j * rng.normal(size=(n, n, n))
    v = tuple(rng.normal(size=(n, n, n)) for _ in range(3))
    x = 2 * np.pi * np.arange(n) / n
    kd, kk = wavenumbers_deriv(n), wavenumbers(n)
    ph = np.fft.fftn(phi) / n ** 3            # library FFT as an independent step
    g = [np.zeros_like(phi) for _ in range(3)]
    for iz in range(n):
        for iy in range(n):
            for ix in range(n):
                c = ph[iz, iy, ix]
                e = np.exp(1j * (kk[ix] * x[None, None, :] + kk[iy] * x[None, :, None] + kk[iz] * x[:, None, None]))
                g[0] += 1j * kd[ix] * c * e
                g[1] += 1j * kd[iy] * c * e
                g[2] += 1j * kd[iz] * c * e
    t = sum(np.mean(np.abs(g[j] - 1j * v[j] * phi / (2 * alpha)) ** 2) for j in range(3))
    ref = 2 * alpha ** 2 * t + alpha * beta * np.mean((np.abs(phi) ** 2 - 1) ** 2)
    assert OA.energy_v(phi, alpha, beta, v) == pytest.approx(ref, rel=1e-12)


def test_energy_decreases_along_the_flow():
    """The step is a discrete gradient flow of E_v: from a rough start in the TG flow, E_v does
    not increase (small dtau)."""
    n, alpha, beta, dtau = 16, 0.25, 8.0, 0.01
    v = OA.velocity("tg", n)
    phi = smooth_psi(n, 11)
    e_prev = OA.energy_v(phi, alpha, beta, v)
    for _ in range(15):
        phi = OA.argle_step(phi, alpha, beta, dtau, v)
        e = OA.energy_v(phi, alpha, beta, v)
        assert e <= e_prev * (1 + 1e-12)
        e_prev = e


def test_renormalised_flow_keeps_the_mass():
    n, alpha, beta, dtau = 12, 0.2, 10.0, 0.02
    phi = OA.argle(smooth_psi(n, 2), alpha, beta, dtau, 5, OA.velocity("tg", n), renorm=0.9)
    assert float(np.mean(np.abs(phi) ** 2)) == pytest.approx(0.9, rel=1e-14)


def test_tg_clebsch_potentials_give_the_vorticity():
    """grad lambda x grad mu = curl v_TG (clebsch) where cos z != 0, by centred differences."""
    rng = np.random.default_rng(1)
    h = 1e-6
    for _ in range(20):
        x, y = rng.uniform(0, 2 * np.pi, 2)
        z = rng.uniform(-1.2, 1.2) + (np.pi if rng.random() < 0.5 else 0.0)    # away from cos z = 0

        def grad(f):
            return np.array([(f(x + h, y, z) - f(x - h, y, z)) / (2 * h), (f(x, y + h, z) - f(x, y - h, z)) / (2 * h),
                             (f(x, y, z + h) - f(x, y, z - h)) / (2 * h)])

        lam = lambda a, b, c: OA.clebsch(np.array(a), np.array(b), np.array(c))[0]   # noqa: E731
        mu = lambda a, b, c: OA.clebsch(np.array(a), np.array(b), np.array(c))[1]    # noqa: E731
        cross = np.cross(grad(lam), grad(mu))
        # curl of (sin x cos y cos z, -cos x sin y cos z, 0)
        curl = np.array([-np.cos(x) * np.sin(y) * np.sin(z), -np.sin(x) * np.cos(y) * np.sin(z),
                         2 * np.sin(x) * np.sin(y) * np.cos(z)])
        assert np.allclose(cross, curl, atol=2e-6)


@pytest.mark.parametrize("alpha,m", [(0.05, 3), (0.025, 6), (0.0125, 12), (0.00625, 25)])
def test_tg_winding_numbers_of_the_paper(alpha, m):
    """[gamma_d / 4] = [1 / (2 pi alpha)] of the paper's TG runs (3, 6, 12, 25 for N = 128..1024)."""
    assert OA.tg_winding(alpha) == m


def test_tg_ansatz_zeros_and_winding():
    """psi_e has one simple zero at the origin of the (lambda, mu) plane; psi_4 vanishes where
    (lambda, mu) = (+-1/sqrt2, 0) or (0, +-1/sqrt2); psi_4 ** m winds m times around each."""
    xi = 0.05
    assert OA.psi_e(np.array(0.0), np.array(0.0), xi) == 0
    h = 1 / math.sqrt(2)
    for cl, cm in ((h, 0.0), (-h, 0.0), (0.0, h), (0.0, -h)):
        t = np.linspace(0, 2 * np.pi, 401)
        lam, mu = cl + 0.05 * np.cos(t), cm + 0.05 * np.sin(t)
        f = OA.psi_e(lam - h, mu, xi) * OA.psi_e(lam, mu - h, xi) * OA.psi_e(lam + h, mu, xi) * OA.psi_e(lam, mu + h, xi)
        assert abs(OA.psi_e(np.array(cl - h), np.array(cm), xi) * OA.psi_e(np.array(cl), np.array(cm - h), xi)
                   * OA.psi_e(np.array(cl + h), np.array(cm), xi) * OA.psi_e(np.array(cl), np.array(cm + h), xi)) < 1e-12
        for m in (1, 3):
            wind = np.sum(np.angle((f ** m)[1:] / (f ** m)[:-1])) / (2 * np.pi)
            assert round(wind) == m and abs(wind - m) < 1e-9


def test_tg_ansatz_on_the_grid():
    """psi_ARGLE = psi_4 ** 3 at alpha = 0.05 (the TG start of the 128^3 runs): even under
    x -> 2 pi - x and y -> 2 pi - y (the mirror extension), |psi| <= 1."""
    n, alpha, beta = 32, 0.05, 40.0
    psi = OA.tg_ansatz(n, alpha, beta)
    assert np.allclose(psi, psi[:, :, (-np.arange(n)) % n]) and np.allclose(psi, psi[:, (-np.arange(n)) % n, :])
    assert np.max(np.abs(psi)) <= 1.0 + 1e-12
    assert np.isclose(psi, OA.tg_psi4(*OA.coords(n), math.sqrt(alpha / beta)) ** 3).all()


def test_abc_flow_is_beltrami_and_divergence_free():
    """Each v^(k) satisfies curl v = k v and div v = 0 (spectral derivatives, exact on the grid)."""
    n = 16
    X, Y, Z = OA.coords(n)
    A, B, C = OA.ABC_DEFAULT
    kd = wavenumbers_deriv(n)

    def d(f, axis):
        k = {0: kd[None, None, :], 1: kd[None, :, None], 2: kd[:, None, None]}[axis]
        return np.real(fft.ifft3(1j * k * fft.fft3(f)))

    for k in (1, 2):
        v = (B * np.cos(k * Y) + C * np.sin(k * Z), C * np.cos(k * Z) + A * np.sin(k * X),
             A * np.cos(k * X) + B * np.sin(k * Y))
        curl = (d(v[2], 1) - d(v[1], 2), d(v[0], 2) - d(v[2], 0), d(v[1], 0) - d(v[0], 1))
        for j in range(3):
            assert np.max(np.abs(curl[j] - k * v[j])) < 1e-12
        assert np.max(np.abs(d(v[0], 0) + d(v[1], 1) + d(v[2], 2))) < 1e-12
    vt = OA.abc_velocity(X, Y, Z)
    assert np.max(np.abs(vt[0] - (B * (np.cos(Y) + np.cos(2 * Y)) + C * (np.sin(Z) + np.sin(2 * Z))))) < 1e-14


def test_abc_ansatz_phase_is_periodic_and_follows_the_flow():
    """|phi| = 1; the phase is periodic (integer coefficients times coordinates); away from the
    jumps of its rounded coefficients its gradient is v_ABC / (2 alpha) up to the four roundings
    (at most 2 per component)."""
    n, alpha = 24, 0.05
    assert np.allclose(np.abs(OA.abc_ansatz(n, alpha)), 1.0)
    rng = np.random.default_rng(3)
    two_pi = 2 * np.pi
    pts = rng.uniform(0, two_pi, size=(200, 3))
    X, Y, Z = pts[:, 0], pts[:, 1], pts[:, 2]
    th = OA.abc_phase(X, Y, Z, alpha)
    for shift in ((two_pi, 0, 0), (0, two_pi, 0), (0, 0, two_pi)):
        d = OA.abc_phase(X + shift[0], Y + shift[1], Z + shift[2], alpha) - th
        assert np.max(np.abs(np.exp(1j * d) - 1)) < 1e-9
    v = OA.abc_velocity(X, Y, Z)
    h = 1e-7
    checked = 0
    for j, e in enumerate(np.eye(3)):
        fp = OA.abc_phase(X + h * e[0], Y + h * e[1], Z + h * e[2], alpha)
        fm = OA.abc_phase(X - h * e[0], Y - h * e[1], Z - h * e[2], alpha)
        g = (fp - fm) / (2 * h)
        # a coefficient that jumps inside the interval changes the phase by O(1): skip those points
        smooth = np.abs(g) < 1e3
        assert np.all(np.abs(g[smooth] - v[j][smooth] / (2 * alpha)) <= 2.0 + 1e-6)
        checked += int(smooth.sum())
    assert checked > 550


def test_stopping_criteria_of_a_decaying_mode():
    """beta = 0, v = 0, phi = A exp(i k.x): one step multiplies A by f = (1 - a)/(1 + a), so
    crit1 = |f - 1| |A| / dtau and, with E_v = 2 alpha^2 |A|^2 |k|^2, crit2 = |f^2 - 1| / dtau."""
    n, alpha, dtau, A = 12, 0.3, 0.05, 0.8 - 0.3j
    k = (2, -1, 3)
    X, Y, Z = OA.coords(n)
    phi = A * np.exp(1j * (k[0] * X + k[1] * Y + k[2] * Z))
    a = 0.5 * dtau * alpha * sum(c * c for c in k)
    f = (1 - a) / (1 + a)
    new = OA.argle_step(phi, alpha, 0.0, dtau, _zero_v(n))
    assert OA.residual_inf(new, phi, dtau) == pytest.approx(abs(f - 1) * abs(A) / dtau, rel=1e-12)
    assert OA.energy_change(new, phi, alpha, 0.0, dtau, _zero_v(n)) == pytest.approx(abs(f * f - 1) / dtau, rel=1e-10)


def test_converge_stops_at_the_first_checked_step_below_eps():
    """The same decaying mode: crit1 after step m is |f - 1| |f|^(m-1) |A| / dtau, a geometric
    sequence, so the first checked step below eps is known in closed form; eps <= 0 runs all
    steps and reports the last step's criteria; the stepped field is the plain loop's."""
    n, alpha, dtau, A = 8, 0.3, 0.05, 1.0
    k = (1, 2, 0)
    X, Y, Z = OA.coords(n)
    phi = A * np.exp(1j * (k[0] * X + k[1] * Y + k[2] * Z))
    a = 0.5 * dtau * alpha * sum(c * c for c in k)
    f = (1 - a) / (1 + a)
    c1 = lambda m: abs(f - 1) * abs(f) ** (m - 1) * A / dtau
    eps = 0.5 * (c1(23) + c1(24))          # first step with crit1 <= eps is 24; checked every 5: 25
    out, done, r1, r2 = OA.argle_converge(phi, alpha, 0.0, dtau, 100, _zero_v(n), eps, 5)
    assert done == 25
    assert r1 == pytest.approx(c1(25), rel=1e-10) and r2 == pytest.approx(abs(f * f - 1) / dtau, rel=1e-8)
    assert np.max(np.abs(out - OA.argle(phi, alpha, 0.0, dtau, 25, _zero_v(n)))) == 0.0
    out, done, r1, _ = OA.argle_converge(phi, alpha, 0.0, dtau, 13, _zero_v(n), 0.0, 5)
    assert done == 13 and r1 == pytest.approx(c1(13), rel=1e-10)

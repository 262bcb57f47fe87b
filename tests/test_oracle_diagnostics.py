"""Pins for the oracle diagnostics (Sec. 3.4-3.5, 4.1): closed forms and exact identities."""
import math

import numpy as np
import pytest

from inputs import grid_coords, random_psi, smooth_psi
from oracle import diagnostics as D
from oracle import fft
from oracle import scheme as S


def _p(n):
    return S.params_from_dx_ratio(n, 1.5, 0.01)


def test_plane_wave_closed_forms():
    """psi = A exp(i k.x): N = A^2, E = 2 alpha^2 A^2 |k|^2 + alpha beta (A^2-1)^2,
    u = 2 alpha A k is uniform (the k = 0 mode, incompressible), q = 0."""
    n = 12
    p = _p(n)
    X, Y, Z = grid_coords(n)
    A, k = 0.8, (2, -1, 3)
    psi = A * np.exp(1j * (k[0] * X + k[1] * Y + k[2] * Z))
    d, spec = D.full(psi, p)
    k2 = sum(c * c for c in k)
    assert abs(d["N"] - A * A) < 1e-14
    assert abs(d["E"] - (2 * p.alpha ** 2 * A * A * k2 + p.alpha * p.beta * (A * A - 1) ** 2)) < 1e-12
    assert abs(d["E_kin"] - 2 * p.alpha ** 2 * A * A * k2) < 1e-12
    assert abs(d["E_kin_i"] - d["E_kin"]) < 1e-12 and abs(d["E_kin_c"]) < 1e-12
    assert abs(d["E_q"]) < 1e-20
    assert abs(spec["E_kin_i"][0] - d["E_kin"]) < 1e-12          # all in shell 0


def test_sound_wave_is_compressible():
    """psi = exp(i eps sin x): u = 2 alpha eps cos(x) e_x, a pure gradient:
    E_kin^c = alpha^2 eps^2, E_kin^i = 0, all of it in shell 1."""
    n, eps = 32, 0.1
    p = _p(n)
    X, _, _ = grid_coords(n)
    d, spec = D.full(np.exp(1j * eps * np.sin(X)), p)
    assert abs(d["E_kin_c"] - p.alpha ** 2 * eps ** 2) < 1e-13
    assert abs(d["E_kin_i"]) < 1e-20
    assert abs(spec["E_kin_c"][1] - d["E_kin_c"]) < 1e-13


def test_density_wave_closed_form():
    """psi = 1 + a cos x (real): u = 0, q = -a sin x, E_q = alpha^2 a^2,
    E_int = alpha beta <(2 a cos x + a^2 cos^2 x)^2>."""
    n, a = 32, 0.2
    p = _p(n)
    X, _, _ = grid_coords(n)
    d, _ = D.full((1 + a * np.cos(X)).astype(complex), p)
    assert abs(d["E_kin"]) < 1e-28
    assert abs(d["E_q"] - p.alpha ** 2 * a * a) < 1e-13
    eint = p.alpha * p.beta * (2 * a * a + 3.0 / 8.0 * a ** 4)
    assert abs(d["E_int"] - eint) < 1e-13


@pytest.mark.parametrize("seed", [1, 2])
def test_energy_split_identities(seed):
    n = 12
    p = _p(n)
    psi = random_psi(n, seed, amp_jitter=0.2)
    d, spec = D.full(psi, p)
    # E = E_kin + E_q + E_int + (Nyquist part of the gradient energy)
    assert abs(d["E_kin"] + d["E_q"] + d["E_int"] + D.nyquist_gradient_energy(psi, p) - d["E"]) < 1e-10 * d["E"]
    assert abs(d["E_kin_i"] + d["E_kin_c"] - d["E_kin"]) < 1e-10 * d["E_kin"]
    for name in D.SPECTRA:
        assert abs(np.sum(spec[name]) - d[name]) < 1e-10 * abs(d[name])
    assert len(spec["E_kin_i"]) == D.nbins(n)


def test_band_limited_field_has_no_nyquist_part():
    n = 16
    p = _p(n)
    psi = smooth_psi(n, 4)
    d, _ = D.full(psi, p, with_spectra=False)
    assert abs(d["E_kin"] + d["E_q"] + d["E_int"] - d["E"]) < 1e-12 * d["E"]


def test_helmholtz_projector():
    n = 12
    rng = np.random.default_rng(9)
    kd = S.wavenumbers_deriv(n)
    kv = [kd[None, None, :], kd[None, :, None], kd[:, None, None]]
    phi = rng.standard_normal((n, n, n))
    grad = [np.real(fft.ifft3(1j * kv[j] * fft.fft3(phi))) for j in range(3)]
    ui, uc = D.helmholtz(grad)
    assert max(np.max(np.abs(c)) for c in ui) < 1e-9                   # gradient: no incompressible part
    A = [rng.standard_normal((n, n, n)) for _ in range(3)]
    Ah = [fft.fft3(a) for a in A]
    curl = [np.real(fft.ifft3(1j * (kv[1] * Ah[2] - kv[2] * Ah[1]))),
            np.real(fft.ifft3(1j * (kv[2] * Ah[0] - kv[0] * Ah[2]))),
            np.real(fft.ifft3(1j * (kv[0] * Ah[1] - kv[1] * Ah[0])))]
    ui, uc = D.helmholtz(curl)
    assert max(np.max(np.abs(c)) for c in uc) < 1e-9                   # curl: no compressible part
    u = [rng.standard_normal((n, n, n)) for _ in range(3)]
    ui, uc = D.helmholtz(u)
    cross = sum(np.sum(np.conj(ui[j]) * uc[j]) for j in range(3))
    assert abs(cross) < 1e-9 * sum(np.sum(np.abs(c) ** 2) for c in ui)   # orthogonal
    ui2, uc2 = D.helmholtz([np.real(fft.ifft3(c)) for c in ui])
    assert max(np.max(np.abs(ui2[j] - ui[j])) for j in range(3)) < 1e-9  # idempotent


def test_shells():
    assert D.nbins(64) == int(math.floor(math.sqrt(3) * 32 + 0.5)) + 1
    b = D.shell_index(8)
    assert b[0, 0, 0] == 0 and b[0, 0, 1] == 1 and b[0, 0, 4] == 4 and b[4, 4, 4] == 7
    assert b.max() == D.nbins(8) - 1


def test_zero_density_points_are_masked():
    n = 8
    p = _p(n)
    psi = random_psi(n, 3)
    psi[2, 3, 4] = 0.0
    u, q = D.hydro_fields(psi, p)
    assert all(c[2, 3, 4] == 0.0 for c in u + q)
    assert all(np.isfinite(c).all() for c in u + q)


def test_srp_start_is_vortex_free_once_resolved():
    """A smoothed random phase has no vortices: with |psi| = 1, u = 2 alpha grad(theta) is a gradient,
    so E_kin^i vanishes once the grid resolves exp(i theta) (Sec. 5.3: vortices nucleate later)."""
    from oracle import initial as OI
    n = 64
    d, _ = D.full(OI.srp_spectral(n, 1, 2.0), _p(n), with_spectra=False)
    assert d["E_kin_i"] < 1e-12 * d["E_kin_c"]


@pytest.mark.parametrize("k,amp", [((1, 0, 0), 1.0), ((2, -1, 3), 0.8)])
def test_momentum_and_mach_of_a_plane_wave(k, amp):
    """psi = A exp(i k.x): rho v = 2 alpha |A|^2 k, sqrt(rho) v = 2 alpha |A| k everywhere, so
    P = 2 alpha A^2 k and M_max = M_rms = 2 alpha A |k| / c with c = sqrt(2 alpha beta)."""
    n = 16
    p = S.Params(n=n, alpha=0.3, beta=5.0, dt=0.0)
    x = 2 * np.pi * np.arange(n) / n
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    psi = amp * np.exp(1j * (k[0] * X + k[1] * Y + k[2] * Z))
    d, _ = D.full(psi, p, with_spectra=False)
    for j, name in enumerate(("P_x", "P_y", "P_z")):
        assert d[name] == pytest.approx(2 * p.alpha * amp ** 2 * k[j], abs=1e-13)
    m = 2 * p.alpha * amp * math.sqrt(sum(c * c for c in k)) / math.sqrt(2 * p.alpha * p.beta)
    assert d["M_max"] == pytest.approx(m, rel=1e-12) and d["M_rms"] == pytest.approx(m, rel=1e-12)


def test_momentum_by_parseval():
    """<Im(psi* d_j psi)> = sum_k k~_j |F psi_k|^2 / n^2: the physical-space mean against the
    spectral sum (numpy's FFT, an independent path)."""
    n = 12
    p = S.Params(n=n, alpha=0.2, beta=10.0, dt=0.0)
    rng = np.random.default_rng(4)
    psi = rng.normal(size=(n, n, n)) + 1j * rng.normal(size=(n, n, n))
    d, _ = D.full(psi, p, with_spectra=False)
    ph = np.fft.fftn(psi)
    kd = S.wavenumbers_deriv(n)
    w = np.abs(ph) ** 2 / psi.size ** 2
    ref = [2 * p.alpha * float(np.sum(kd[None, None, :] * w)), 2 * p.alpha * float(np.sum(kd[None, :, None] * w)),
           2 * p.alpha * float(np.sum(kd[:, None, None] * w))]
    for name, r in zip(("P_x", "P_y", "P_z"), ref):
        assert d[name] == pytest.approx(r, rel=1e-12, abs=1e-14)
    assert d["M_max"] >= d["M_rms"]

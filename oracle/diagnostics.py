"""Oracle diagnostics: mass, energy, hydrodynamic split, Helmholtz split, spectra.

Test infrastructure only (see ``oracle/__init__``).

All quantities are volume means (Sec. 4.1: eq-scaling-N, eq-scaling-energy,
eq-scaling-energy-mod-rho), computed in float64.  With the unnormalised
forward DFT F and n = N^3 grid points, Parseval gives mean(|f|^2) =
sum_k |F f_k|^2 / n^2, which turns the continuous 1/(2 pi)^3 of the spectra
(Sec. 3.5) into 1/n^2 for mean-normalised energies.

Momentum <rho v> = 2 alpha <Im(psi* grad psi)> (eq-mom-total, eq-scaling-rhov) and the Mach
numbers of sqrt(rho) v (eq:Mach-Number): M_max = max |sqrt(rho) v| / c, M_rms = sqrt(2 E_kin) / c,
with the sound speed c = sqrt(2 alpha beta) (c^2 / 2 is the coefficient of (rho - 1)^2 in E).

Readings where the paper is silent:
  * first derivatives use i k~ with the Nyquist component of k~ set to zero;
    the gradient energy in E uses the Laplacian-consistent |k|^2 (Nyquist kept);
  * sqrt(rho) v and grad sqrt(rho) use u = 2 alpha Im(psi* grad psi)/|psi| and
    q = Re(psi* grad psi)/|psi|, set to zero where |psi|^2 < eps_rho = 1e-12;
  * Helmholtz projection with k~; the k = 0 mode goes to the incompressible part;
  * shells: bin b = floor(|k| + 1/2) with the true |k|, b = 0 .. floor(sqrt(3) N/2 + 1/2).
"""
import math

import numpy as np

from . import fft
from .scheme import k2_grid, wavenumbers, wavenumbers_deriv

EPS_RHO = 1e-12
NAMES = ("N", "E", "E_kin", "E_kin_i", "E_kin_c", "E_q", "E_int", "P_x", "P_y", "P_z", "M_max", "M_rms")
SPECTRA = ("E_kin_i", "E_kin_c", "E_q", "E_int")


def nbins(n):
    return int(math.floor(math.sqrt(3.0) * n / 2.0 + 0.5)) + 1


def shell_index(n):
    k = wavenumbers(n)
    kk = np.sqrt(k[:, None, None] ** 2 + k[None, :, None] ** 2 + k[None, None, :] ** 2)
    return np.floor(kk + 0.5).astype(np.int64)


def mass(psi):
    """N = <|psi|^2> (eq-scaling-N)."""
    return float(np.mean(np.abs(psi) ** 2))


def energy(psi, p):
    """E = <2 alpha^2 |grad psi|^2 + alpha beta (|psi|^2 - 1)^2> (eq-scaling-energy),
    the gradient term by Parseval with the Laplacian's |k|^2."""
    n = psi.size
    ph = fft.fft3(psi)
    grad2 = float(np.sum(k2_grid(psi.shape[0]) * np.abs(ph) ** 2)) / n ** 2
    inter = float(np.mean((np.abs(psi) ** 2 - 1.0) ** 2))
    return 2.0 * p.alpha ** 2 * grad2 + p.alpha * p.beta * inter


def gradient(psi):
    """Spectral gradient [d/dx, d/dy, d/dz] with Nyquist-zeroed wavenumbers."""
    N = psi.shape[0]
    kd = wavenumbers_deriv(N)
    ph = fft.fft3(psi)
    gx = fft.ifft3(1j * kd[None, None, :] * ph)
    gy = fft.ifft3(1j * kd[None, :, None] * ph)
    gz = fft.ifft3(1j * kd[:, None, None] * ph)
    return [gx, gy, gz]


def hydro_fields(psi, p, grad=None):
    """u = sqrt(rho) v = 2 alpha Im(psi* grad psi)/|psi| and q = grad sqrt(rho) = Re(psi* grad psi)/|psi|
    (eq-scaling-rhov, eq-scaling-energy-mod-rho), zero where |psi|^2 < EPS_RHO."""
    if grad is None:
        grad = gradient(psi)
    rho = np.abs(psi) ** 2
    mask = rho >= EPS_RHO
    amp = np.where(mask, np.sqrt(np.where(mask, rho, 1.0)), 1.0)
    u, q = [], []
    for g in grad:
        w = np.conj(psi) * g
        u.append(np.where(mask, 2.0 * p.alpha * w.imag / amp, 0.0))
        q.append(np.where(mask, w.real / amp, 0.0))
    return u, q


def helmholtz(u):
    """Split the real vector field u into compressible (curl-free) and incompressible
    (divergence-free) parts in k-space (eq:def-ekin-decomp): u^c_k = k~ (k~ . u_k) / |k~|^2."""
    N = u[0].shape[0]
    kd = wavenumbers_deriv(N)
    kv = [kd[None, None, :], kd[None, :, None], kd[:, None, None]]
    uh = [fft.fft3(c) for c in u]
    kk = kv[0] ** 2 + kv[1] ** 2 + kv[2] ** 2
    dot = kv[0] * uh[0] + kv[1] * uh[1] + kv[2] * uh[2]
    safe = np.where(kk > 0, kk, 1.0)
    coef = np.where(kk > 0, dot / safe, 0.0)
    uc = [kv[j] * coef for j in range(3)]
    ui = [uh[j] - uc[j] for j in range(3)]
    return ui, uc        # both in k-space (unnormalised DFT)


def _shell_sum(weight, bins, nb):
    return np.bincount(bins.ravel(), weights=weight.ravel(), minlength=nb)[:nb]


def full(psi, p, with_spectra=True):
    """Every diagnostic of Sec. 3.4-3.5 / 4.1 for one field.

    Returns (dict of the scalars in NAMES, dict of the spectra in SPECTRA or None).
    """
    N = psi.shape[0]
    n = psi.size
    rho = np.abs(psi) ** 2
    grad = gradient(psi)
    u, q = hydro_fields(psi, p, grad)
    ui, uc = helmholtz(u)
    out = {
        "N": float(np.mean(rho)),
        "E": energy(psi, p),
        "E_kin": float(np.mean(0.5 * (u[0] ** 2 + u[1] ** 2 + u[2] ** 2))),
        "E_kin_i": 0.5 * float(sum(np.sum(np.abs(c) ** 2) for c in ui)) / n ** 2,
        "E_kin_c": 0.5 * float(sum(np.sum(np.abs(c) ** 2) for c in uc)) / n ** 2,
        "E_q": float(np.mean(2.0 * p.alpha ** 2 * (q[0] ** 2 + q[1] ** 2 + q[2] ** 2))),
        "E_int": float(np.mean(p.alpha * p.beta * (rho - 1.0) ** 2)),
    }
    # momentum per unit volume <rho v> = 2 alpha <Im(psi* grad psi)> (eq-mom-total, eq-scaling-rhov)
    for name, g in zip(("P_x", "P_y", "P_z"), grad):
        out[name] = 2.0 * p.alpha * float(np.mean(np.imag(np.conj(psi) * g)))
    # Mach numbers (eq:Mach-Number) of sqrt(rho) v with the sound speed c = sqrt(2 alpha beta)
    c = math.sqrt(2.0 * p.alpha * p.beta)
    out["M_max"] = float(np.sqrt(np.max(u[0] ** 2 + u[1] ** 2 + u[2] ** 2))) / c
    out["M_rms"] = math.sqrt(2.0 * out["E_kin"]) / c
    if not with_spectra:
        return out, None
    nb = nbins(N)
    bins = shell_index(N)
    spec = {
        "E_kin_i": 0.5 * _shell_sum(sum(np.abs(c) ** 2 for c in ui), bins, nb) / n ** 2,
        "E_kin_c": 0.5 * _shell_sum(sum(np.abs(c) ** 2 for c in uc), bins, nb) / n ** 2,
        "E_q": 2.0 * p.alpha ** 2 * _shell_sum(sum(np.abs(fft.fft3(c)) ** 2 for c in q), bins, nb) / n ** 2,
        "E_int": p.alpha * p.beta * _shell_sum(np.abs(fft.fft3(rho - 1.0)) ** 2, bins, nb) / n ** 2,
    }
    return out, spec


def nyquist_gradient_energy(psi, p):
    """2 alpha^2 sum_k (|k|^2 - |k~|^2) |psi_k|^2 / n^2: the part of E's gradient term that
    the Nyquist-zeroed first derivatives do not see (zero for band-limited fields)."""
    N = psi.shape[0]
    n = psi.size
    kd = wavenumbers_deriv(N)
    kt2 = kd[:, None, None] ** 2 + kd[None, :, None] ** 2 + kd[None, None, :] ** 2
    ph = fft.fft3(psi)
    return 2.0 * p.alpha ** 2 * float(np.sum((k2_grid(N) - kt2) * np.abs(ph) ** 2)) / n ** 2

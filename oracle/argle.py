"""Oracle: imaginary-time (ARGLE) preparation and the Taylor-Green / ABC initial fields.

Test infrastructure only (see ``oracle/__init__``).  Float64 throughout, arrays [z, y, x] on
the periodic box [0, 2 pi]^3 with x_i = 2 pi i / N.

ARGLE (Sec. 4.2, eqn:gradient-flow): the gradient flow of the energy of a field driven by a
divergence-free external velocity v (eq-energy-num-ext-vel),
    d phi / d tau = (alpha lap - i v . grad - |v|^2 / (4 alpha) + beta - beta |phi|^2) phi,
advanced by the semi-implicit backward-Euler step of eqn:semi-backward-Euler: half of the
Laplacian implicit, everything else explicit at the old level,
    (phi' - phi) / dtau = (alpha/2) lap phi' + ((alpha/2) lap - i v . grad - |v|^2/(4 alpha)
                                               + beta - beta |phi|^2) phi,
solved exactly in Fourier space (the implicit part is diagonal):
    F phi' = [ (1 - dtau alpha |k|^2 / 2) F phi + dtau F(rest) ] / (1 + dtau alpha |k|^2 / 2),
    rest = -i v . grad phi - |v|^2/(4 alpha) phi + beta (1 - |phi|^2) phi.
Readings: the printed right-hand side applies the explicit
operator to "phi~^n", read as phi^n (the old level); first derivatives use Nyquist-zeroed
wavenumbers, the Laplacian the full |k|^2; the optional L2 renormalisation (the normalised
gradient flow the section starts from) rescales phi after each step to a prescribed mean
|phi|^2.

Stopping (eqn:crit1, eqn:crit2): ||phi^{n+1} - phi^n||_inf / dtau <= eps, and the relative
energy change |E_v(phi^{n+1}) - E_v(phi^n)| / (dtau E_v(phi^n)), which the paper reports when
the first criterion was not reached.

Energy of the driven field (eq-energy-num-ext-vel), as a volume mean:
    E_v = < 2 alpha^2 |grad phi - i v phi / (2 alpha)|^2 + alpha beta (|phi|^2 - 1)^2 >.

Taylor-Green (Sec. 5.1): v_TG = (sin x cos y cos z, -cos x sin y cos z, 0); Clebsch potentials
lambda = cos x sqrt(2 |cos z|), mu = cos y sqrt(2 |cos z|) sgn(cos z) (clebsch3d); the
one-zero field psi_e(lambda, mu) = (lambda + i mu) tanh(r / (sqrt(2) xi)) / r, r = |(lambda, mu)|
(psie); psi_4 = psi_e(lambda - 1/sqrt2, mu) psi_e(lambda, mu - 1/sqrt2) psi_e(lambda + 1/sqrt2, mu)
psi_e(lambda, mu + 1/sqrt2) (psi4); psi_ARGLE = psi_4 ** m with m = [gamma_d / 4] = floor(1 / (2 pi
alpha)) (psitot3d).  The formula is already even in x, y and z about 0 and pi, so evaluating it on
the whole box is its mirror extension.

ABC (Sec. 5.2): v = v^(1) + v^(2), v^(k) = (B cos ky + C sin kz, C cos kz + A sin kx,
A cos kx + B sin ky), (A, B, C) = (0.9, 1, 1.1)/sqrt(3) by default (ABC); the start field is
psi^(1) psi^(2), psi^(k) = psi_{A,k}^{x,y,z} psi_{B,k}^{y,z,x} psi_{C,k}^{z,x,y} with
psi_{A,k}^{x,y,z} = exp(i [A sin(kx)/(2 alpha)] y + i [A cos(kx)/(2 alpha)] z), [a] the nearest
integer (ABCphi0, ABCphi), the other two by cyclic permutation of (A, x, y, z).  Reading: a
half-integer [a] rounds away from zero (the paper does not say), with a 1e-9 window so that
the decision does not depend on the last bit of a.
"""
import math

import numpy as np

from . import fft
from .scheme import k2_grid, wavenumbers_deriv

ABC_DEFAULT = (0.9 / math.sqrt(3.0), 1.0 / math.sqrt(3.0), 1.1 / math.sqrt(3.0))


def coords(n):
    """X, Y, Z on the [z, y, x] grid."""
    x = 2.0 * math.pi * np.arange(n) / n
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    return X, Y, Z


# ---------------- external velocities ----------------

def tg_velocity(X, Y, Z):
    """v_TG (tg3d)."""
    return (np.sin(X) * np.cos(Y) * np.cos(Z), -np.cos(X) * np.sin(Y) * np.cos(Z), np.zeros_like(X))


def abc_velocity(X, Y, Z, abc=ABC_DEFAULT):
    """v_ABC = v^(1) + v^(2) (ABC)."""
    A, B, C = abc
    vx = np.zeros_like(X)
    vy = np.zeros_like(X)
    vz = np.zeros_like(X)
    for k in (1, 2):
        vx = vx + B * np.cos(k * Y) + C * np.sin(k * Z)
        vy = vy + C * np.cos(k * Z) + A * np.sin(k * X)
        vz = vz + A * np.cos(k * X) + B * np.sin(k * Y)
    return vx, vy, vz


def velocity(kind, n, abc=ABC_DEFAULT):
    X, Y, Z = coords(n)
    if kind == "tg":
        return tg_velocity(X, Y, Z)
    if kind == "abc":
        return abc_velocity(X, Y, Z, abc)
    z = np.zeros_like(X)
    return z, z, z


# ---------------- Taylor-Green start field ----------------

def clebsch(X, Y, Z):
    """lambda, mu of clebsch3d."""
    cz = np.cos(Z)
    s = np.sqrt(2.0 * np.abs(cz))
    return np.cos(X) * s, np.cos(Y) * s * np.sign(cz)


def psi_e(lam, mu, xi):
    """(lambda + i mu) tanh(r / (sqrt 2 xi)) / r (psie), 0 at r = 0."""
    r = np.sqrt(lam ** 2 + mu ** 2)
    with np.errstate(invalid="ignore", divide="ignore"):
        f = np.where(r > 0.0, np.tanh(r / (math.sqrt(2.0) * xi)) / np.where(r > 0.0, r, 1.0), 0.0)
    return (lam + 1j * mu) * f


def tg_winding(alpha):
    """m = [gamma_d / 4] with gamma_d = 2 / (pi alpha): floor(1 / (2 pi alpha))."""
    return int(math.floor(1.0 / (2.0 * math.pi * alpha)))


def tg_psi4(X, Y, Z, xi):
    lam, mu = clebsch(X, Y, Z)
    h = 1.0 / math.sqrt(2.0)
    return psi_e(lam - h, mu, xi) * psi_e(lam, mu - h, xi) * psi_e(lam + h, mu, xi) * psi_e(lam, mu + h, xi)


def tg_ansatz(n, alpha, beta):
    """psi_ARGLE of psitot3d on the n^3 grid."""
    X, Y, Z = coords(n)
    xi = math.sqrt(alpha / beta)
    return tg_psi4(X, Y, Z, xi) ** tg_winding(alpha)


# ---------------- ABC start field ----------------

ROUND_TIE = 1e-9


def _round_half_away(a):
    """Nearest integer, halves away from zero; a value within 1e-9 of a half counts as the half.
    (With the default amplitudes and alpha = 0.05, A sin(60 deg) / (2 alpha) is exactly 4.5 and
    C cos(30 deg) / (2 alpha) exactly 5.5 -- grids whose points include those angles hit the
    ties, which float64 rounding would otherwise decide either way.)"""
    return np.sign(a) * np.floor(np.abs(a) + 0.5 + ROUND_TIE)


def abc_phase(X, Y, Z, alpha, abc=ABC_DEFAULT):
    """The phase of phi(0+) = psi^(1) psi^(2) (ABCphi0 / ABCphi) at the given points."""
    A, B, C = abc
    phase = np.zeros_like(np.asarray(X, dtype=float))
    for k in (1, 2):
        # psi_{A,k}^{x,y,z}: coefficients of y and z from A and x
        phase += _round_half_away(A * np.sin(k * X) / (2 * alpha)) * Y + _round_half_away(A * np.cos(k * X) / (2 * alpha)) * Z
        # psi_{B,k}^{y,z,x}: coefficients of z and x from B and y
        phase += _round_half_away(B * np.sin(k * Y) / (2 * alpha)) * Z + _round_half_away(B * np.cos(k * Y) / (2 * alpha)) * X
        # psi_{C,k}^{z,x,y}: coefficients of x and y from C and z
        phase += _round_half_away(C * np.sin(k * Z) / (2 * alpha)) * X + _round_half_away(C * np.cos(k * Z) / (2 * alpha)) * Y
    return phase


def abc_ansatz(n, alpha, abc=ABC_DEFAULT):
    """phi(0+) of ABCphi0 on the n^3 grid."""
    X, Y, Z = coords(n)
    return np.exp(1j * abc_phase(X, Y, Z, alpha, abc))


# ---------------- ARGLE ----------------

def _grad(phi_hat, n):
    kd = wavenumbers_deriv(n)
    return [fft.ifft3(1j * kd[None, None, :] * phi_hat), fft.ifft3(1j * kd[None, :, None] * phi_hat),
            fft.ifft3(1j * kd[:, None, None] * phi_hat)]


def argle_step(phi, alpha, beta, dtau, v, renorm=None):
    """One semi-implicit backward-Euler step (eqn:semi-backward-Euler).  v = (vx, vy, vz) arrays;
    renorm: None, or the mean |phi|^2 to rescale to after the step."""
    n = phi.shape[0]
    ph = fft.fft3(phi)
    g = _grad(ph, n)
    vv = v[0] ** 2 + v[1] ** 2 + v[2] ** 2
    rest = -1j * (v[0] * g[0] + v[1] * g[1] + v[2] * g[2]) - vv / (4.0 * alpha) * phi \
        + beta * (1.0 - np.abs(phi) ** 2) * phi
    a = 0.5 * dtau * alpha * k2_grid(n)
    new = fft.ifft3(((1.0 - a) * ph + dtau * fft.fft3(rest)) / (1.0 + a))
    if renorm is not None:
        new = new * math.sqrt(renorm / float(np.mean(np.abs(new) ** 2)))
    return new


def argle(phi, alpha, beta, dtau, nsteps, v, renorm=None):
    for _ in range(nsteps):
        phi = argle_step(phi, alpha, beta, dtau, v, renorm)
    return phi


def energy_v(phi, alpha, beta, v):
    """E_v of eq-energy-num-ext-vel (volume mean; Nyquist-zeroed first derivatives)."""
    n = phi.shape[0]
    g = _grad(fft.fft3(phi), n)
    t = 0.0
    for j in range(3):
        d = g[j] - 1j * v[j] * phi / (2.0 * alpha)
        t += float(np.mean(np.abs(d) ** 2))
    return 2.0 * alpha ** 2 * t + alpha * beta * float(np.mean((np.abs(phi) ** 2 - 1.0) ** 2))


def residual_inf(phi_new, phi_old, dtau):
    """||phi^{n+1} - phi^n||_inf / dtau (eqn:crit1)."""
    return float(np.max(np.abs(phi_new - phi_old))) / dtau


def energy_change(phi_new, phi_old, alpha, beta, dtau, v):
    """|E_v(phi^{n+1}) - E_v(phi^n)| / (dtau E_v(phi^n)) (eqn:crit2)."""
    e_old = energy_v(phi_old, alpha, beta, v)
    return abs(energy_v(phi_new, alpha, beta, v) - e_old) / (dtau * e_old)


def argle_converge(phi, alpha, beta, dtau, max_steps, v, eps, check_every, renorm=None):
    """Steps until eqn:crit1 holds at a checked step or max_steps are done.

    The criteria are evaluated for every check_every-th step and for the last step; the run
    stops after the first checked step with crit1 <= eps (eps <= 0: never).  Returns
    (phi, steps_done, crit1, crit2) with the criteria of the last checked step."""
    c1 = c2 = float("nan")
    done = 0
    while done < max_steps:
        new = argle_step(phi, alpha, beta, dtau, v, renorm)
        done += 1
        if done % check_every == 0 or done == max_steps:
            c1 = residual_inf(new, phi, dtau)
            c2 = energy_change(new, phi, alpha, beta, dtau, v)
            phi = new
            if eps > 0 and c1 <= eps:
                break
        else:
            phi = new
    return phi, done, c1, c2

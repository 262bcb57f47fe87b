"""Oracle: parameters and the Strang split step of the dimensionless GP equation.

Test infrastructure only (see ``oracle/__init__``).

Equation (Sec. 4.1, eq-gpe-num):  i dpsi/dt = -alpha lap(psi) + beta (|psi|^2 - 1) psi
on the periodic box [0, 2 pi]^3 sampled at x_i = 2 pi i / N, arrays indexed [z, y, x].

Parameters (Sec. 4.1, eq-scaling-ab and eq-scaling-choice3): L = 2 pi and
alpha * beta = 1 / (2 M^2) with the reference Mach number M = 1/2, i.e.
alpha * beta = 2, and the healing length xi = sqrt(alpha / beta).  Given xi:
alpha = sqrt(2) xi and beta = 2 / alpha.

Time step (Sec. 4.3, eq:adi_looptime): exact directional kinetic sub-flows
S(s, L_j) phi = F_j^{-1}( exp(-i alpha k_j^2 s) F_j phi ) and the exact
nonlinear sub-flow S(s, N) phi = exp(-i beta |phi|^2 s) phi.  The nonlinear
flow here carries the -1 of eq-gpe-num, exp(-i beta (|phi|^2 - 1) s) phi,
unless ``minus_one=False`` selects the literal form of the splitting section;
the two differ by the global phase exp(i beta s).

Two orders of the same second-order splitting:
  KNK (the paper's eq:adi_looptime): Sx Sy Sz (dt/2) . N(dt) . Sz Sy Sx (dt/2)
  NKN: N(dt/2) . Sx Sy Sz (dt) . N(dt/2)
"""
import math
from dataclasses import dataclass

import numpy as np

from . import fft


@dataclass(frozen=True)
class Params:
    n: int
    alpha: float
    beta: float
    dt: float
    minus_one: bool = True

    @property
    def xi(self):
        return math.sqrt(self.alpha / self.beta)

    @property
    def dx(self):
        return 2.0 * math.pi / self.n


def params_from_xi(n, xi, dt, minus_one=True):
    """alpha = sqrt(2) xi, beta = 2/alpha (Sec. 4.1, eq-scaling-choice3 with M = 1/2)."""
    alpha = math.sqrt(2.0) * xi
    return Params(n=n, alpha=alpha, beta=2.0 / alpha, dt=dt, minus_one=minus_one)


def params_from_dx_ratio(n, xi_over_dx, dt, minus_one=True):
    """Healing length given as a multiple of the grid spacing dx = 2 pi / N."""
    return params_from_xi(n, xi_over_dx * 2.0 * math.pi / n, dt, minus_one)


def wavenumbers(n):
    """Integer wavenumbers of an n-point periodic grid on [0, 2 pi): 0..n/2-1, -n/2..-1."""
    k = np.arange(n, dtype=np.float64)
    k[k >= (n + 1) // 2] -= n
    return k


def wavenumbers_deriv(n):
    """Wavenumbers for first derivatives: the Nyquist entry (even n) is set to zero."""
    k = wavenumbers(n)
    if n % 2 == 0:
        k[n // 2] = 0.0
    return k


def k2_grid(n):
    """|k|^2 on the [kz, ky, kx] grid (the Nyquist entry enters as (n/2)^2)."""
    k = wavenumbers(n)
    return k[:, None, None] ** 2 + k[None, :, None] ** 2 + k[None, None, :] ** 2


# ----- sub-flows (Sec. 4.3) -----

def nonlinear_flow(phi, p, s):
    """S(s, N): pointwise phase rotation by -beta (|phi|^2 - 1) s; |phi| is unchanged."""
    rho = np.abs(phi) ** 2
    v = rho - 1.0 if p.minus_one else rho
    return np.exp(-1j * p.beta * v * s) * phi


def kinetic_flow_axis(phi, p, s, axis):
    """S(s, L_j): 1D transform along one axis, multiply by exp(-i alpha k_j^2 s), inverse."""
    n = phi.shape[axis]
    k = wavenumbers(n)
    shape = [1, 1, 1]
    shape[axis] = n
    mult = np.exp(-1j * p.alpha * (k ** 2) * s).reshape(shape)
    return fft.ifft1(mult * fft.fft1(phi, axis), axis)


def kinetic_flow(phi, p, s):
    """S(s,Lx) S(s,Ly) S(s,Lz): the three directional flows (they commute exactly)."""
    for axis in (2, 1, 0):
        phi = kinetic_flow_axis(phi, p, s, axis)
    return phi


def step_knk(psi, p):
    """One step in the paper's order (eq:adi_looptime): kinetic dt/2, nonlinear dt, kinetic dt/2."""
    phi = psi
    for axis in (2, 1, 0):            # S(dt/2, Lx), then Ly, then Lz
        phi = kinetic_flow_axis(phi, p, 0.5 * p.dt, axis)
    phi = nonlinear_flow(phi, p, p.dt)
    for axis in (0, 1, 2):            # S(dt/2, Lz), then Ly, then Lx
        phi = kinetic_flow_axis(phi, p, 0.5 * p.dt, axis)
    return phi


def step_nkn(psi, p):
    """One step in the nonlinear-outside order: N(dt/2), kinetic dt, N(dt/2)."""
    phi = nonlinear_flow(psi, p, 0.5 * p.dt)
    phi = kinetic_flow(phi, p, p.dt)
    return nonlinear_flow(phi, p, 0.5 * p.dt)


def evolve(psi, p, nsteps, order="nkn", callback=None):
    """Apply ``nsteps`` steps one by one; ``callback(step_index, psi)`` after each."""
    step = step_nkn if order == "nkn" else step_knk
    psi = np.asarray(psi, dtype=np.complex128)
    for m in range(nsteps):
        psi = step(psi, p)
        if callback is not None:
            callback(m + 1, psi)
    return psi

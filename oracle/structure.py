"""Oracle: longitudinal velocity structure functions.

Test infrastructure only (see ``oracle/__init__``).  Float64, arrays [z, y, x] on the periodic
box [0, 2 pi]^3.

strfunc-def (Sec. 3.5): along the unit vector e_j,
    S^p_j(r) = < ((v(x + r e_j) - v(x)) . e_j)^p >,
a volume mean over the grid, for separations r = s dx, dx = 2 pi / N, s = 0 .. N/2 (on the
periodic grid S^p_j(N dx - r) = (-1)^p S^p_j(r), so those shifts carry all of it).

Readings where the paper is silent:
  * v is the superfluid velocity of eq-scaling-rhov, v = 2 alpha Im(psi* grad psi) / |psi|^2,
    with the spectral gradient of the other diagnostics (Nyquist-zeroed wavenumbers) and v = 0
    where |psi|^2 < eps_rho = 1e-12 (the same cut as sqrt(rho) v);
  * the integral is the volume mean, like the energies;
  * the order p is a positive integer.
"""
import numpy as np

from .diagnostics import EPS_RHO, gradient


def velocity(psi, p, grad=None):
    """v_j = 2 alpha Im(psi* d_j psi) / |psi|^2 (eq-scaling-rhov), 0 where |psi|^2 < EPS_RHO."""
    if grad is None:
        grad = gradient(psi)
    rho = np.abs(psi) ** 2
    mask = rho >= EPS_RHO
    safe = np.where(mask, rho, 1.0)
    return [np.where(mask, 2.0 * p.alpha * np.imag(np.conj(psi) * g) / safe, 0.0) for g in grad]


# array axis of each direction j = x, y, z on the [z, y, x] grid
_AXIS = (2, 1, 0)


def structure_function(v, order):
    """S^order_j(s dx) for j = 0, 1, 2 (x, y, z) and s = 0 .. N/2: array [3, N/2 + 1].

    v: the three velocity components.  Each separation is the definition written out: the
    field shifted by s points in +e_j (np.roll by -s brings v(x + s dx e_j) to x), the
    difference of the j-th components, its power, the mean."""
    n = v[0].shape[0]
    ns = n // 2 + 1
    out = np.zeros((3, ns))
    for j in range(3):
        vj = v[j]
        for s in range(ns):
            d = np.roll(vj, -s, axis=_AXIS[j]) - vj
            out[j, s] = float(np.mean(d ** order))
    return out


def separations(n):
    """r = s 2 pi / N for s = 0 .. N/2."""
    return 2.0 * np.pi * np.arange(n // 2 + 1) / n

"""Oracle: helicity and regularised helicity of a GP field.

Test infrastructure only (see ``oracle/__init__``).  Float64, arrays [z, y, x] on the periodic
box [0, 2 pi]^3; all integrals are volume means, like the energies.  In the dimensionless units
of Sec. 4.1 the quantum hbar / m becomes 2 alpha (v = 2 alpha grad theta, eq-scaling-rhov).

eq-helicity:   H = < v . omega >,  omega = curl v.
Sec. 3.6 (regularised helicity, after Clark di Leoni et al.):
    w       = (2 alpha / i) grad psi* x grad psi                           (a real vector)
    v_par   = 2 alpha w_i [ (d_i d_j psi) d_j psi* - (d_i d_j psi*) d_j psi ]
              / ( 2 i |w| (d_l psi)(d_l psi*) )
    v_reg   = v_par w / |w|
    H_reg   = < v_reg . omega >                                                   (Hreg)
Helicity spectra: H(k) and H_reg(k) are the shell sums (shell floor(|k| + 1/2)) of
Re(conj(F v) . F omega) / n^2 and Re(conj(F v_reg) . F omega) / n^2, so that they add up to
H and H_reg (Parseval with the unnormalised DFT F and n grid points).

Readings where the paper is silent:
  * v is the velocity of the structure functions and diagnostics: 2 alpha Im(psi* grad psi) /
    |psi|^2, 0 where |psi|^2 < 1e-12; omega is its spectral curl (i k~ x F v, the
    Nyquist-zeroed wavenumbers of every first derivative);
  * the second derivatives d_i d_j psi are -k~_i k~_j F psi (the first derivative applied twice);
  * v_reg = 0 where |w| <= W_CUT 4 alpha <|grad psi|^2> (W_CUT = 1e-5): v_par has no limit where
    grad psi vanishes (at a stagnation point it grows like 1/|grad psi|, and w/|w| has no
    direction), and on symmetry planes the gradient is only round-off there.  Since
    |w| <= 2 alpha |grad psi|^2 the one cut also removes those points.  Near a vortex line
    |w| is of the order of 4 alpha |grad psi|^2, far above the cut; in the smooth flow between
    the lines w = grad rho x v is small, and so is omega, so the cut points add nothing there.
"""
import numpy as np

from . import fft
from .diagnostics import gradient, nbins, shell_index
from .scheme import wavenumbers_deriv
from .structure import velocity

W_CUT = 1e-5


def _kvec(n):
    kd = wavenumbers_deriv(n)
    return [kd[None, None, :], kd[None, :, None], kd[:, None, None]]


def curl_hat(vh):
    """F(curl v) = i k~ x F v for the spectra vh[0..2] of a vector field."""
    k = _kvec(vh[0].shape[0])
    return [1j * (k[1] * vh[2] - k[2] * vh[1]),
            1j * (k[2] * vh[0] - k[0] * vh[2]),
            1j * (k[0] * vh[1] - k[1] * vh[0])]


def curl(v):
    wh = curl_hat([fft.fft3(c) for c in v])
    return [np.real(fft.ifft3(c)) for c in wh]


def helicity_of(v):
    """< v . curl v > of a real vector field (eq-helicity)."""
    om = curl(v)
    return float(np.mean(v[0] * om[0] + v[1] * om[1] + v[2] * om[2]))


def hessian(psi):
    """d_i d_j psi for i <= j as a dict {(i, j): array}, i, j in 0 (x), 1 (y), 2 (z)."""
    ph = fft.fft3(psi)
    k = _kvec(psi.shape[0])
    return {(i, j): fft.ifft3(-k[i] * k[j] * ph) for i in range(3) for j in range(i, 3)}


def w_field(grad, alpha):
    """w = (2 alpha / i) grad psi* x grad psi, returned as its real part (the imaginary part
    vanishes identically: the cross product of a vector and its conjugate is imaginary)."""
    a = [np.conj(g) for g in grad]
    b = grad
    c = [a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]]
    return [np.real(2.0 * alpha / 1j * cj) for cj in c]


def v_parallel(grad, hess, alpha, wcut=0.0):
    """v_par and w from first and second derivatives (pointwise; any array shape).

    grad: [d_x psi, d_y psi, d_z psi];  hess: {(i, j): d_i d_j psi} for i <= j.
    Returns (v_par, w), v_par = 0 where |w| <= wcut or |grad psi|^2 = 0."""
    w = w_field(grad, alpha)
    H = lambda i, j: hess[(min(i, j), max(i, j))]
    num = 0.0
    for i in range(3):
        t = 0.0
        for j in range(3):
            t = t + H(i, j) * np.conj(grad[j]) - np.conj(H(i, j)) * grad[j]
        num = num + w[i] * t
    wn = np.sqrt(w[0] ** 2 + w[1] ** 2 + w[2] ** 2)
    g2 = np.real(sum(g * np.conj(g) for g in grad))
    den = 2j * wn * g2
    ok = (wn > wcut) & (g2 > 0)
    vpar = np.where(ok, np.real(2.0 * alpha * num / np.where(ok, den, 1.0)), 0.0)
    return vpar, w


def v_reg(grad, hess, alpha, wcut=0.0):
    """v_par w / |w| (0 where |w| <= wcut)."""
    vpar, w = v_parallel(grad, hess, alpha, wcut)
    wn = np.sqrt(w[0] ** 2 + w[1] ** 2 + w[2] ** 2)
    safe = np.where(wn > wcut, wn, 1.0)
    return [np.where(wn > wcut, vpar * wc / safe, 0.0) for wc in w]


def w_cut(grad, alpha):
    """W_CUT 4 alpha <|grad psi|^2>."""
    return W_CUT * 4.0 * alpha * float(np.mean(sum(np.abs(g) ** 2 for g in grad)))


def helicities(psi, p, with_spectra=True):
    """(H, H_reg) and, with_spectra, (H(k), H_reg(k)) over the shells 0 .. nbins(N) - 1."""
    n = psi.shape[0]
    grad = gradient(psi)
    v = velocity(psi, p, grad)
    vh = [fft.fft3(c) for c in v]
    omh = curl_hat(vh)
    om = [np.real(fft.ifft3(c)) for c in omh]
    H = float(np.mean(v[0] * om[0] + v[1] * om[1] + v[2] * om[2]))
    vr = v_reg(grad, hessian(psi), p.alpha, w_cut(grad, p.alpha))
    Hr = float(np.mean(vr[0] * om[0] + vr[1] * om[1] + vr[2] * om[2]))
    if not with_spectra:
        return (H, Hr), None
    nb = nbins(n)
    bins = shell_index(n).ravel()
    vrh = [fft.fft3(c) for c in vr]
    dens = [sum(np.real(np.conj(a[j]) * omh[j]) for j in range(3)) / float(psi.size) ** 2 for a in (vh, vrh)]
    spec = [np.bincount(bins, weights=d.ravel(), minlength=nb)[:nb] for d in dens]
    return (H, Hr), (spec[0], spec[1])

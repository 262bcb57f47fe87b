"""Oracle adjoint: vector-Jacobian products of the split step and of E_kin^i.

Test infrastructure only (see ``oracle/__init__``).  The paper has no adjoint;
this is the transpose of its split step (Sec. 4.3) under the real inner product
<a, b> = Re sum_x conj(a_x) b_x, derived from the sub-flows:

  kinetic  K(s) = F^-1 exp(-i alpha |k|^2 s) F is unitary, so VJP_K(s)(lam) = K(-s) lam.
  nonlinear N(s): psi_out = exp(-i phi) psi, phi = beta s (|psi|^2 - 1) (or beta s |psi|^2);
           VJP_N(lam) = exp(+i phi) lam + 2 beta s Im(conj(lam) psi_out) psi.

A step's VJP applies the sub-flow VJPs in reverse order at the intermediate
states of the forward step.  The functional is the incompressible kinetic
energy of the final state, J = E_kin^i(psi_T) (Sec. 3.4, eq:def-ekin-decomp),
with |psi| regularised as sqrt(|psi|^2 + eps_J) inside u = sqrt(rho) v so that J
is differentiable at vortex cores; its gradient (the adjoint's final value) is

  lam_T = (2 alpha / n) sum_j [ -i w_j d_j psi - d_j(i w_j psi) - w_j Im(psi* d_j psi) psi / |psi|_eps^2 ],
  w_j = u^i_j / |psi|_eps,

with d_j the Nyquist-zeroed spectral derivative (d_j^T = -d_j).  For psi_0 = exp(i theta):
dJ/dtheta = -Im(conj(lam_0) psi_0).
"""
import numpy as np

from . import fft
from .diagnostics import helmholtz
from .scheme import kinetic_flow, nonlinear_flow, wavenumbers_deriv

EPS_J = 1e-6


def vjp_nonlinear(psi_in, lam, p, s):
    rho = np.abs(psi_in) ** 2
    phi = p.beta * s * ((rho - 1.0) if p.minus_one else rho)
    psi_out = np.exp(-1j * phi) * psi_in
    return np.exp(1j * phi) * lam + 2.0 * p.beta * s * np.imag(np.conj(lam) * psi_out) * psi_in


def vjp_kinetic(lam, p, s):
    return kinetic_flow(lam, p, -s)


def vjp_step(psi_n, lam_next, p, order="nkn"):
    """lam_n from lam_{n+1} for one step taken from state psi_n."""
    if order == "nkn":
        a = nonlinear_flow(psi_n, p, 0.5 * p.dt)
        b = kinetic_flow(a, p, p.dt)
        lb = vjp_nonlinear(b, lam_next, p, 0.5 * p.dt)
        la = vjp_kinetic(lb, p, p.dt)
        return vjp_nonlinear(psi_n, la, p, 0.5 * p.dt)
    a = kinetic_flow(psi_n, p, 0.5 * p.dt)
    lb = vjp_kinetic(lam_next, p, 0.5 * p.dt)
    la = vjp_nonlinear(a, lb, p, p.dt)
    return vjp_kinetic(la, p, 0.5 * p.dt)


def _grad(psi):
    N = psi.shape[0]
    kd = wavenumbers_deriv(N)
    kv = [kd[None, None, :], kd[None, :, None], kd[:, None, None]]
    ph = fft.fft3(psi)
    return [fft.ifft3(1j * kv[j] * ph) for j in range(3)], kv


def _deriv(f, kv_j):
    return fft.ifft3(1j * kv_j * fft.fft3(f))


def ekin_i_reg(psi, p, eps=EPS_J):
    """J(psi) = E_kin^i with u = 2 alpha Im(psi* grad psi) / sqrt(|psi|^2 + eps)."""
    g, _ = _grad(psi)
    amp = np.sqrt(np.abs(psi) ** 2 + eps)
    u = [2.0 * p.alpha * np.imag(np.conj(psi) * gj) / amp for gj in g]
    ui, _ = helmholtz(u)
    n = psi.size
    return 0.5 * float(sum(np.sum(np.abs(c) ** 2) for c in ui)) / n ** 2


def ekin_i_reg_grad(psi, p, eps=EPS_J):
    """lam_T = dJ/dpsi in the Re<conj(lam), dpsi> convention."""
    g, kv = _grad(psi)
    amp2 = np.abs(psi) ** 2 + eps
    amp = np.sqrt(amp2)
    u = [2.0 * p.alpha * np.imag(np.conj(psi) * gj) / amp for gj in g]
    ui_hat, _ = helmholtz(u)
    ui = [np.real(fft.ifft3(c)) for c in ui_hat]
    lam = np.zeros_like(psi)
    for j in range(3):
        w = ui[j] / amp
        lam += (-1j * w * g[j]
                - _deriv(1j * w * psi, kv[j])
                - w * np.imag(np.conj(psi) * g[j]) * psi / amp2)
    return (2.0 * p.alpha / psi.size) * lam


def forward_states(psi0, p, nsteps, order="nkn"):
    from .scheme import step_knk, step_nkn
    step = step_nkn if order == "nkn" else step_knk
    states = [np.asarray(psi0, dtype=np.complex128)]
    for _ in range(nsteps):
        states.append(step(states[-1], p))
    return states


def gradient_theta(theta, p, nsteps, order="nkn", eps=EPS_J):
    """dJ/dtheta for J = E_kin^i(psi_T), psi_0 = exp(i theta); returns (J, grad)."""
    psi0 = np.exp(1j * np.asarray(theta, dtype=np.float64))
    states = forward_states(psi0, p, nsteps, order)
    lam = ekin_i_reg_grad(states[-1], p, eps)
    for m in range(nsteps - 1, -1, -1):
        lam = vjp_step(states[m], lam, p, order)
    return ekin_i_reg(states[-1], p, eps), -np.imag(np.conj(lam) * psi0)

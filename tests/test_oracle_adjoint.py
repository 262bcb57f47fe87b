"""Pins for the oracle adjoint: dot-product tests and finite differences in float64."""
import math

import numpy as np
import pytest

from inputs import random_direction, random_psi
from oracle import adjoint as A
from oracle import initial as I
from oracle import scheme as S


def _inner(a, b):
    return float(np.real(np.sum(np.conj(a) * b)))


@pytest.mark.parametrize("order", ["nkn", "knk"])
@pytest.mark.parametrize("minus_one", [True, False])
def test_step_vjp_dot_product(order, minus_one):
    """<lam, J dpsi> = <VJP(lam), dpsi>, with J dpsi by central differences (h = 1e-6)."""
    n = 8
    p0 = S.params_from_dx_ratio(n, 1.5, 0.02)
    p = S.Params(n, p0.alpha, p0.beta, p0.dt, minus_one)
    step = S.step_nkn if order == "nkn" else S.step_knk
    psi = random_psi(n, 1)
    dpsi = random_direction(n, 2)
    lam = random_direction(n, 3)
    h = 1e-6
    jvp = (step(psi + h * dpsi, p) - step(psi - h * dpsi, p)) / (2 * h)
    lhs = _inner(lam, jvp)
    rhs = _inner(A.vjp_step(psi, lam, p, order), dpsi)
    assert abs(lhs - rhs) < 1e-7 * abs(rhs)


def test_ekin_i_gradient_matches_finite_differences():
    n = 8
    p = S.params_from_dx_ratio(n, 1.5, 0.02)
    psi = random_psi(n, 5, amp_jitter=0.2)
    lam = A.ekin_i_reg_grad(psi, p)
    for seed in (6, 7):
        v = random_direction(n, seed)
        h = 1e-5
        fd = (A.ekin_i_reg(psi + h * v, p) - A.ekin_i_reg(psi - h * v, p)) / (2 * h)
        assert abs(fd - _inner(lam, v)) < 1e-6 * abs(fd)


def test_theta_gradient_matches_finite_differences():
    """dJ/dtheta of J = E_kin^i(psi_T) through 6 steps from an SRP phase; h = 1e-4, float64."""
    n, m = 12, 6
    p = S.params_from_dx_ratio(n, 1.5, 0.004)
    theta = I.srp_theta(n, 0, 3.0)
    J0, g = A.gradient_theta(theta, p, m)
    assert J0 > 0
    for seed in range(4):
        v = np.real(random_direction(n, 100 + seed, complex_valued=False))
        h = 1e-4
        jp = A.ekin_i_reg(S.evolve(np.exp(1j * (theta + h * v)), p, m), p)
        jm = A.ekin_i_reg(S.evolve(np.exp(1j * (theta - h * v)), p, m), p)
        fd = (jp - jm) / (2 * h)
        assert abs(fd - float(np.sum(g * v))) < 1e-6 * abs(fd)

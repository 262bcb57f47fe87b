"""Configuration 5 (128^3, xi = 1.5 dx, dt = 0.004, SRP start with k0 = 4, gradient of the final
incompressible kinetic energy with respect to the initial phase, checkpoints every 20 steps).

The flow amplifies perturbations of its start quickly: a 4e-8 relative perturbation grows ~10x per
20 steps at first (to ~1e-4 after 100 steps), and the gradient's norm grows with it (~1e-4 after 20
steps, ~1e2 after 100, ~1e5 after 400).  At 400 steps a float64 run from the float32-rounded start
already gives a different gradient, and no float64 finite difference resolves the linear response.
These tests separate the adjoint's own arithmetic from that sensitivity:
  * the float32 and the float64 adjoints run along the SAME trajectory (the float32 run's
    checkpoints, upcast, and the same final cotangent), 400 steps: they agree to 1e-3;
  * centred finite differences in float64 on 16 seeded directions match the float64 adjoint to
    1e-3 at 20 steps and at 100 steps (where the start's sensitivity reaches 1e-4), with h scaled
    to the measured amplification A of a start perturbation over the horizon, h =
    10^floor(log10(1e-4 / A)): 1e-5 at 20 steps, 1e-8 at 100.  The configuration's h = 1e-4 is
    outside the linear regime already at 20 steps (measured worst error 1.1e-3 over the 16
    directions; 0.6 to 2.8 at 100 steps); the difference converges as h^2 to the adjoint value
    as h shrinks, at every horizon where float64 can still resolve it."""
import math

import numpy as np
import pytest

from inputs import random_direction
from oracle import initial as OI

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2003_03590_gb300 import GP_FP32, GP_FP64, Plan, field_params  # noqa: E402

N, DT, EVERY, STEPS, EPS = 128, 0.004, 20, 400, 1e-6


def _theta():
    return torch.from_numpy(OI.srp_theta(N, 0, 4.0)).cuda()


def _plan(prec):
    return Plan(field_params(N, DT, xi_over_dx=1.5, precision=prec))


def _rel(a, b):
    return float(torch.linalg.vector_norm((a - b).double()) / torch.linalg.vector_norm(b.double()))


def _forward(plan, theta, steps):
    psi0 = plan.psi_from_phase(0, theta)
    psi = psi0.clone()
    ckpts, done = [], 0
    while done < steps:
        k = min(EVERY, steps - done)
        ckpts.append((psi.clone(), k))
        plan.step([psi], k)
        done += k
    return psi0, psi, ckpts


def _backward(plan, psi0, ckpts, lam):
    for state, k in reversed(ckpts):
        plan.adjoint_step(0, state, lam, k)
    return plan.phase_grad(0, psi0, lam)


def test_fp32_and_fp64_adjoints_agree_along_the_same_trajectory():
    p32, p64 = _plan(GP_FP32), _plan(GP_FP64)
    th = _theta()
    psi0_32, psiT_32, ck32 = _forward(p32, th.float(), STEPS)
    lam32, _ = p32.ekin_i_grad(0, psiT_32, EPS)
    g32 = _backward(p32, psi0_32, ck32, lam32)
    # the float64 adjoint on the float32 trajectory: its checkpoints and final state, upcast
    lam64, _ = p64.ekin_i_grad(0, psiT_32.to(torch.complex128), EPS)
    ck64 = [(s.to(torch.complex128), k) for s, k in ck32]
    g64 = _backward(p64, p64.psi_from_phase(0, th.float().double()), ck64, lam64)
    e = _rel(g32, g64)
    print("config 5, 400 steps, same trajectory: float32 vs float64 adjoint gradient", e)
    assert e < 1e-3, e


def _sensitivity_horizon(p64, th, limit=1e-4):
    """Largest multiple of 20 steps (<= 400) at which the float64 flow from the start perturbed by
    4e-8 (relative, a float32 rounding) stays within `limit` of the unperturbed flow."""
    rng = np.random.default_rng(5)
    a = p64.psi_from_phase(0, th)
    b = a * (1.0 + 4e-8 * torch.from_numpy(rng.standard_normal(a.shape)).cuda())
    horizon, curve = 0, []
    for m in range(EVERY, STEPS + 1, EVERY):
        p64.step([a], EVERY)
        p64.step([b], EVERY)
        r = _rel(b, a)
        curve.append((m, r))
        if r <= limit:
            horizon = m
        else:
            break
    return horizon, curve


def test_finite_differences_at_two_horizons():
    p64 = _plan(GP_FP64)
    th = _theta()
    M100, curve = _sensitivity_horizon(p64, th)
    print("float64 sensitivity to a 4e-8 start perturbation (steps, rel L2):", curve)
    assert M100 >= 60, curve
    amp = dict(curve)

    def J(t, M):
        psi = p64.psi_from_phase(0, t)
        p64.step([psi], M)
        return p64.ekin_i_grad(0, psi, EPS)[1]

    def h_of(M):   # the difference stays in the flow's linear regime: h A(M) <= 1e-4
        return 10.0 ** math.floor(math.log10(1e-4 / max(amp[M] / 4e-8, 1.0)))

    for M, h in ((EVERY, h_of(EVERY)), (M100, h_of(M100))):
        psi0, psiT, ck = _forward(p64, th, M)
        lam, _ = p64.ekin_i_grad(0, psiT, EPS)
        g = _backward(p64, psi0, ck, lam)
        worst = 0.0
        for seed in range(16):
            v = torch.from_numpy(np.real(random_direction(N, 900 + seed, complex_valued=False))).cuda()
            fd = (J(th + h * v, M) - J(th - h * v, M)) / (2 * h)
            an = float((g * v).sum())
            worst = max(worst, abs(fd - an) / abs(an))
        print(f"finite differences vs adjoint at {M} steps, h = {h:.0e}, 16 directions: worst relative error {worst:.2e}")
        assert worst < 1e-3, (M, h, worst)

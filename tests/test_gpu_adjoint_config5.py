"""Configuration 5: 128^3, xi = 1.5 dx, SRP start with k0 = 4, gradient of the final incompressible
kinetic energy with respect to the initial phase, 400 steps, checkpoints every 20 steps, float32
and float64 through the checkpointed adjoint.

The configuration leaves dt open.  dt = 0.002 is used: at 0.004 the grid's wavenumbers
|k| = 85..87 lie in the split step's instability band (alpha |k|^2 dt just below pi, where
cos(alpha k^2 dt) - beta dt sin(alpha k^2 dt) < -1), and the scheme itself amplifies any
perturbation there by up to 1 + beta dt per step: a 4e-8 perturbation of the start grows ~10x per
20 steps, the gradient's norm grows to ~1e5 by 400 steps, and neither a float32/float64 comparison
nor a float64 finite difference can resolve it (test_in_the_instability_band).  At dt = 0.002 the
whole grid is outside the band (alpha |k|^2 dt <= 2.56 < 3.06):
  * the flow's response to a 4e-8 start perturbation stays ~4e-8 over the 400 steps;
  * the float32 and float64 adjoints along one trajectory (the float32 run's checkpoints, upcast)
    agree to 1e-3, and the two precisions' gradients on their own trajectories to 2e-3 (measured
    1.3e-3: the float32 forward run's rounding near the vortex cores, where E_kin^i's 1/|psi| makes
    the functional steep);
  * centred finite differences in float64 on 16 seeded directions match the float64 adjoint to 1e-3
    with h = 1e-5 (the configuration's h = 1e-4: 4e-4 to 4.5e-3, the O(h^2) truncation of the
    difference itself; the error falls 100-fold per decade of h)."""
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

N, EVERY, STEPS, EPS = 128, 20, 400, 1e-6
DT_STABLE, DT_BAND = 0.002, 0.004


def _theta():
    return torch.from_numpy(OI.srp_theta(N, 0, 4.0)).cuda()


def _plan(prec, dt):
    return Plan(field_params(N, dt, xi_over_dx=1.5, precision=prec))


def _rel(a, b):
    return float(torch.linalg.vector_norm((a - b).to(torch.complex128)) / torch.linalg.vector_norm(b.to(torch.complex128)))


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


def _gradient(plan, theta, steps):
    psi0, psiT, ck = _forward(plan, theta, steps)
    lam, _ = plan.ekin_i_grad(0, psiT, EPS)
    return _backward(plan, psi0, ck, lam)


def _sensitivity(p64, th, steps):
    """(steps, relative L2 response) of the float64 flow to a 4e-8 relative perturbation of the start."""
    rng = np.random.default_rng(5)
    a = p64.psi_from_phase(0, th)
    b = a * (1.0 + 4e-8 * torch.from_numpy(rng.standard_normal(a.shape)).cuda())
    curve = []
    for m in range(EVERY, steps + 1, EVERY):
        p64.step([a], EVERY)
        p64.step([b], EVERY)
        curve.append((m, _rel(b, a)))
    return curve


def _same_trajectory(dt, th):
    p32, p64 = _plan(GP_FP32, dt), _plan(GP_FP64, dt)
    psi0_32, psiT_32, ck32 = _forward(p32, th.float(), STEPS)
    lam32, _ = p32.ekin_i_grad(0, psiT_32, EPS)
    g32 = _backward(p32, psi0_32, ck32, lam32)
    lam64, _ = p64.ekin_i_grad(0, psiT_32.to(torch.complex128), EPS)
    ck64 = [(s.to(torch.complex128), k) for s, k in ck32]
    g64 = _backward(p64, p64.psi_from_phase(0, th.float().double()), ck64, lam64)
    return _rel(g32, g64)


def test_config5_at_a_stable_step():
    th = _theta()
    p64, p32 = _plan(GP_FP64, DT_STABLE), _plan(GP_FP32, DT_STABLE)
    a, b = p64.coefficients()
    assert a * 3 * (N / 2) ** 2 * DT_STABLE < math.pi - 2 * b * DT_STABLE
    curve = _sensitivity(p64, th, STEPS)
    print("dt = 0.002: response to a 4e-8 start perturbation", curve[::5])
    assert max(r for _, r in curve) < 1e-7
    e_same = _same_trajectory(DT_STABLE, th)
    g64 = _gradient(p64, th, STEPS)
    g32 = _gradient(p32, th.float(), STEPS).double()
    e_own = _rel(g32, g64)
    print("dt = 0.002, 400 steps: fp32 vs fp64 adjoint, same trajectory", e_same, "own trajectories", e_own)
    assert e_same < 1e-3 and e_own < 2e-3, (e_same, e_own)

    def J(t):
        psi = p64.psi_from_phase(0, t)
        p64.step([psi], STEPS)
        return p64.ekin_i_grad(0, psi, EPS)[1]

    worst = {1e-4: 0.0, 1e-5: 0.0}
    for seed in range(16):
        v = torch.from_numpy(np.real(random_direction(N, 900 + seed, complex_valued=False))).cuda()
        an = float((g64 * v).sum())
        for h in worst:
            fd = (J(th + h * v) - J(th - h * v)) / (2 * h)
            worst[h] = max(worst[h], abs(fd - an) / abs(an))
    print("dt = 0.002, 400 steps, 16 directions: worst relative error of the finite difference", worst)
    assert worst[1e-5] < 1e-3, worst


def test_in_the_instability_band():
    """dt = 0.004: the start's 4e-8 perturbation is amplified ~10x per 20 steps.  The adjoint is
    still the exact derivative of the scheme: float32 and float64 adjoints along one trajectory
    agree over 400 steps, and finite differences match it at 20 and 100 steps once h is scaled to
    the amplification A over the horizon, h = 10^floor(log10(1e-4 / A))."""
    th = _theta()
    p64 = _plan(GP_FP64, DT_BAND)
    curve = _sensitivity(p64, th, 120)
    print("dt = 0.004: response to a 4e-8 start perturbation", curve)
    amp = dict(curve)
    assert amp[100] > 100 * amp[20]
    e_same = _same_trajectory(DT_BAND, th)
    print("dt = 0.004, 400 steps: fp32 vs fp64 adjoint, same trajectory", e_same)
    assert e_same < 1e-3

    def J(t, M):
        psi = p64.psi_from_phase(0, t)
        p64.step([psi], M)
        return p64.ekin_i_grad(0, psi, EPS)[1]

    for M in (20, 100):
        h = 10.0 ** math.floor(math.log10(1e-4 / max(amp[M] / 4e-8, 1.0)))
        g = _gradient(p64, th, M)
        worst = 0.0
        for seed in range(16):
            v = torch.from_numpy(np.real(random_direction(N, 900 + seed, complex_valued=False))).cuda()
            fd = (J(th + h * v, M) - J(th - h * v, M)) / (2 * h)
            an = float((g * v).sum())
            worst = max(worst, abs(fd - an) / abs(an))
        print(f"dt = 0.004: finite differences vs adjoint at {M} steps, h = {h:.0e}: worst relative error {worst:.2e}")
        assert worst < 1e-3, (M, h, worst)

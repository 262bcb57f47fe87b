"""GPU split step (fused float32 and plain float64 paths) against the float64 CPU oracle."""
import math

import numpy as np
import pytest

from inputs import random_psi, smooth_psi
from oracle import scheme as OS
from tests._util import rel_l2, to_gpu, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2003_03590_gb300 import GP_FP32, GP_FP64, GP_SPLIT_KNK, GP_SPLIT_NKN, Plan, field_params  # noqa: E402

SMALL = [8, 12, 16, 24, 32, 48, 64]


def _oracle_params(plan, dt, minus_one=True):
    a, b = plan.coefficients()
    return OS.Params(n=plan.n(), alpha=a, beta=b, dt=dt, minus_one=minus_one)


def _run(n, prec, split, steps, psi0, dt=0.004, minus_one=True):
    plan = Plan(field_params(n, dt, xi_over_dx=1.5, precision=prec, split=split, minus_one=minus_one))
    dtype = np.complex128 if prec == GP_FP64 else np.complex64
    start = psi0.astype(dtype)
    psi = to_gpu(start, dtype)
    plan.step([psi], steps)
    ref = OS.evolve(start.astype(np.complex128), _oracle_params(plan, dt, minus_one), steps,
                    "nkn" if split == GP_SPLIT_NKN else "knk")
    return to_np(psi), ref


@pytest.mark.parametrize("n", SMALL + [96])
@pytest.mark.parametrize("split", [GP_SPLIT_NKN, GP_SPLIT_KNK])
def test_fp32_fused_step_per_step_parity(n, split):
    psi0 = random_psi(n, n, amp_jitter=0.2)
    got, ref = _run(n, GP_FP32, split, 1, psi0)
    assert rel_l2(got, ref) < 1e-5


@pytest.mark.parametrize("n", SMALL)
@pytest.mark.parametrize("steps", [1, 2, 7])
def test_fp32_merged_steps(n, steps):
    """Several steps in one call (half steps merged, graph-replayed cycle for >= 5 steps)."""
    psi0 = random_psi(n, 100 + n, amp_jitter=0.2)
    got, ref = _run(n, GP_FP32, GP_SPLIT_NKN, steps, psi0)
    assert rel_l2(got, ref) < 1e-5 * steps


@pytest.mark.parametrize("n", SMALL + [96])
@pytest.mark.parametrize("split", [GP_SPLIT_NKN, GP_SPLIT_KNK])
def test_fp64_plain_step_parity(n, split):
    psi0 = random_psi(n, 7 * n, amp_jitter=0.2)
    got, ref = _run(n, GP_FP64, split, 3, psi0)
    assert rel_l2(got, ref) < 1e-12


@pytest.mark.parametrize("prec", [GP_FP32, GP_FP64])
def test_literal_nonlinearity_flag(prec):
    n = 16
    psi0 = random_psi(n, 5)
    got, ref = _run(n, prec, GP_SPLIT_NKN, 4, psi0, minus_one=False)
    assert rel_l2(got, ref) < (1e-5 if prec == GP_FP32 else 1e-12)


@pytest.mark.parametrize("n", [16, 64])
def test_plane_wave_exact_on_gpu(n):
    x = 2 * np.pi * np.arange(n) / n
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    k, A, dt, m = (3, -2, 5), 0.9, 0.003, 40
    psi0 = A * np.exp(1j * (k[0] * X + k[1] * Y + k[2] * Z))
    for prec, tol in ((GP_FP64, 1e-11), (GP_FP32, 2e-5)):
        plan = Plan(field_params(n, dt, xi_over_dx=1.5, precision=prec))
        a, b = plan.coefficients()
        om = a * sum(c * c for c in k) + b * (A * A - 1)
        dtype = np.complex128 if prec == GP_FP64 else np.complex64
        psi = to_gpu(psi0, dtype)
        plan.step([psi], m)
        assert np.max(np.abs(to_np(psi) - psi0 * np.exp(-1j * om * m * dt))) < tol


def test_zero_steps_and_mass():
    n = 32
    plan = Plan(field_params(n, 0.004, xi_over_dx=1.5))
    psi0 = random_psi(n, 3).astype(np.complex64)
    psi = to_gpu(psi0, np.complex64)
    plan.step([psi], 0)
    assert np.array_equal(to_np(psi), psi0.astype(np.complex128))
    plan.step([psi], 50)
    m0 = np.mean(np.abs(psi0.astype(np.complex128)) ** 2)
    assert abs(np.mean(np.abs(to_np(psi)) ** 2) - m0) / m0 < 2e-7


@pytest.mark.parametrize("n,bound", [(64, 1e-6), (96, 5e-6)])
def test_fp32_mass_drift_over_1000_steps(n, bound):
    """Mass is conserved exactly by both sub-flows.  In float32 what is left is round-off: the
    rounding of the few Fourier modes that hold most of the mass does not average over grid
    points, so N(t) random-walks (measured excursions 2e-7..3e-6 over 1000 steps here, changing
    sign and size with any change of the arithmetic); the systematic part is tested below."""
    plan = Plan(field_params(n, 0.002, xi_over_dx=1.5))
    psi = plan.init_srp(0, plan.empty(), seed=0, mode=0, p0=4.0, p1=math.pi)
    m0 = plan.diagnostics(0, psi, spectra=False)[0]["N"]
    worst = 0.0
    for _ in range(10):
        plan.step([psi], 100)
        m = plan.diagnostics(0, psi, spectra=False)[0]["N"]
        worst = max(worst, abs(m - m0) / m0)
    assert worst < bound, worst


@pytest.mark.parametrize("n", [32, 48, 64, 96, 128, 192])
def test_fp32_transforms_have_no_mass_bias(n):
    """The float32 transforms and kinetic factor must not change the mass systematically.  With
    beta ~ 0 a step is a forward 3D FFT, the kinetic factor and an inverse FFT; alpha must be
    non-zero: without the kinetic factor the round trip reaches a fixed point of its own rounding
    after a step or two and no drift can show.  On a random field whose mass is spread over all
    modes the unbiased (hi + lo) twiddles and factors keep the drift at the level of the rounding
    random walk (measured <= ~5e-7 over 1000 steps); a float-rounded twiddle or a lost
    compensation term (as radix-3 lengths once had) drifts ~1e-5..1e-4 over the same steps, as a
    float32 FFT with float32 twiddles does."""
    plan = Plan(field_params(n, 0.002, alpha=0.05, beta=1e-300))
    psi = to_gpu(random_psi(n, 1, amp_jitter=0.1), np.complex64)
    m0 = plan.diagnostics(0, psi, spectra=False)[0]["N"]
    plan.step([psi], 1000)
    m = plan.diagnostics(0, psi, spectra=False)[0]["N"]
    print(n, m / m0 - 1)
    assert abs(m - m0) / m0 < 2e-6


@pytest.mark.parametrize("n", [128, 256])
def test_large_grid_one_step(n):
    """Full per-step parity at the large grids on a smooth field (one oracle step)."""
    psi0 = smooth_psi(n, 9, nmodes=8, kmax=6, amp=0.3)
    got, ref = _run(n, GP_FP32, GP_SPLIT_NKN, 1, psi0, dt=0.002)
    assert rel_l2(got, ref) < 1e-5


@pytest.mark.parametrize("n", [128, 192])
def test_white_field_one_step(n):
    """One step of a field with every Fourier mode populated (random phase, jittered modulus) at
    the lengths between the small grids and 256: 128 (radix 16 x 8) and 192 (three passes with a
    radix-3 one), every butterfly and twiddle carrying data."""
    psi0 = random_psi(n, 31, amp_jitter=0.2)
    got, ref = _run(n, GP_FP32, GP_SPLIT_NKN, 1, psi0, dt=0.002)
    assert rel_l2(got, ref) < 1e-5


@pytest.mark.parametrize("n", [512, 1024])
def test_largest_grids_plane_wave_and_linear_limit(n):
    """At 512^3 / 1024^3 (no full oracle step): plane waves are exact for the scheme, so every
    point is known; a superposition checks the linear limit mode by mode."""
    dt, m = 0.001, 3
    plan = Plan(field_params(n, dt, xi_over_dx=1.5))
    a, b = plan.coefficients()
    idx = torch.arange(n, device="cuda", dtype=torch.float64) * (2 * math.pi / n)
    k = (7, -n // 2 + 1, n // 4)
    ph = (k[0] * idx[None, None, :] + k[1] * idx[None, :, None] + k[2] * idx[:, None, None])
    psi = torch.polar(torch.ones_like(ph), ph).to(torch.complex64).contiguous()
    del ph
    plan.step([psi], m)
    om = a * sum(c * c for c in k)
    # sample points checked against the exact value
    rng = np.random.default_rng(n)
    pts = rng.integers(0, n, size=(2000, 3))
    ti = torch.as_tensor(pts, device="cuda")
    got = psi[ti[:, 0], ti[:, 1], ti[:, 2]].cpu().numpy()
    x = 2 * np.pi * pts / n
    exact = np.exp(1j * (k[0] * x[:, 2] + k[1] * x[:, 1] + k[2] * x[:, 0] - om * m * dt))
    assert np.max(np.abs(got - exact)) < 5e-5
    mass = float((psi.abs() ** 2).double().mean())
    assert abs(mass - 1.0) < 1e-6


def test_time_reversal_on_gpu():
    n = 32
    psi0 = random_psi(n, 77, amp_jitter=0.2)
    for prec, tol in ((GP_FP64, 1e-11), (GP_FP32, 1e-5)):
        dtype = np.complex128 if prec == GP_FP64 else np.complex64
        fwd = Plan(field_params(n, 0.004, xi_over_dx=1.5, precision=prec))
        bwd = Plan(field_params(n, -0.004, xi_over_dx=1.5, precision=prec))
        psi = to_gpu(psi0, dtype)
        fwd.step([psi], 10)
        bwd.step([psi], 10)
        assert rel_l2(to_np(psi), psi0.astype(dtype)) < tol


def test_long_run_256_fp32_vs_fp64():
    """256^3, xi = 1.5 dx, dt = 0.002 (the configured step), 40 vortex rings, 1000 steps.

    At this dt the grid's corner wavenumbers |k| = 169..174 lie in the split step's instability
    band (alpha |k|^2 dt just below pi, where cos(alpha k^2 dt) - beta dt sin(alpha k^2 dt) < -1):
    the scheme itself amplifies any perturbation there by up to 1 + beta dt = 1.077 per step, so
    the float64 path started from the float32-rounded initial state (a perturbation of ~4e-8)
    drifts from the float64 path by ~0.5 (relative L2) after 1000 steps, and no float32 trajectory
    can stay within 1e-3 of float64 that long (at dt = 0.001, outside the band, it stays within
    3e-5: test_1000_steps_fp32_vs_fp64_at_a_stable_step).  What is checked here:
      * the float32 error is the injected rounding carried by that same amplification: it stays
        below 100x the float64-vs-float64 separation while the latter is small;
      * within the first 350 steps it stays below 1e-3;
      * the mass drifts by less than 1e-6 over the 1000 steps."""
    n, dt = 256, 0.002
    p32 = Plan(field_params(n, dt, xi_over_dx=1.5, precision=GP_FP32))
    p64 = Plan(field_params(n, dt, xi_over_dx=1.5, precision=GP_FP64))
    a, b = p32.coefficients()
    xi = math.sqrt(a / b)
    ref = p64.init_rvr(0, p64.empty(), seed=0, mode=0, count=40, p0=4 * xi, p1=12 * xi)
    f32 = ref.to(torch.complex64)
    f64 = f32.to(torch.complex128)
    m0 = p32.diagnostics(0, f32, spectra=False)[0]["N"]

    def rel(x, y):
        return float(torch.linalg.vector_norm(x.to(torch.complex128) - y) / torch.linalg.vector_norm(y))

    worst = 0.0
    for k in range(20):
        for plan, f in ((p32, f32), (p64, f64), (p64, ref)):
            plan.step([f], 50)
        m = p32.diagnostics(0, f32, spectra=False)[0]["N"]
        worst = max(worst, abs(m - m0) / m0)
        e32, sens = rel(f32, f64), rel(f64, ref)
        if sens < 1e-2:
            assert e32 < 100 * sens + 1e-6, (50 * (k + 1), e32, sens)
        if 50 * (k + 1) <= 350:
            assert e32 < 1e-3, (50 * (k + 1), e32)
    assert worst < 1e-6, worst

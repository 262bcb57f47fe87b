"""GPU longitudinal structure functions (Sec. 3.5, strfunc-def) against the float64 oracle, a
closed form at the benchmark grid sizes, and the argument checks of the C ABI."""
import math

import numpy as np
import pytest

from inputs import grid_coords, random_psi
from oracle import scheme as OS
from oracle import structure as OSF
from tests._util import to_gpu

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2003_03590_gb300 import GP_FP32, GP_FP64, GPError, Plan, field_params  # noqa: E402


def _plan(n, prec):
    return Plan(field_params(n, 0.004, xi_over_dx=1.5, precision=prec))


def _dtype(prec):
    return np.complex128 if prec == GP_FP64 else np.complex64


def _scale(ref_even, order):
    """Size of the terms behind S^order: max over s of S^(2m)^(order / 2m), 2m the even order >= order."""
    return float(np.max(np.abs(ref_even))) ** (order / (order + (order % 2)))


@pytest.mark.parametrize("prec", [GP_FP64, GP_FP32])
@pytest.mark.parametrize("n", [12, 16, 24, 48])
def test_structure_functions_match_oracle(n, prec):
    plan = _plan(n, prec)
    a, b = plan.coefficients()
    psi = random_psi(n, 40 + n, amp_jitter=0.25).astype(_dtype(prec))
    v = OSF.velocity(psi.astype(np.complex128), OS.Params(n=n, alpha=a, beta=b, dt=0.004))
    tol = 1e-11 if prec == GP_FP64 else 1e-4
    for order in (1, 2, 3, 4, 8):
        got = plan.structure_function(0, to_gpu(psi, _dtype(prec)), order)
        ref = OSF.structure_function(v, order)
        scale = _scale(OSF.structure_function(v, order + (order % 2)), order)
        assert got.shape == ref.shape
        assert np.all(got[:, 0] == 0.0)
        assert np.max(np.abs(got - ref)) <= tol * scale, (order, np.max(np.abs(got - ref)), scale)


@pytest.mark.parametrize("n", [256, 512])
def test_structure_function_closed_form_at_benchmark_sizes(n):
    """psi = A(y) exp(i a cos(k x)): v = (-2 alpha a k sin(k x), 0, 0) exactly (band-limited to
    round-off), so S^2_x(r) = (2 alpha a k)^2 (1 - cos k r) and S^2_y = S^2_z = 0; the float32
    path at the sizes the benchmark runs (many tiles of pencils, all three staging layouts)."""
    plan = _plan(n, GP_FP32)
    alpha, _ = plan.coefficients()
    a, k = 0.15, 3
    x = torch.arange(n, dtype=torch.float64, device="cuda") * (2 * math.pi / n)
    amp = 0.8 * (1 + 0.2 * torch.cos(x))[None, :, None]                      # varies along y
    psi = (amp * torch.exp(1j * a * torch.cos(k * x))[None, None, :]).expand(n, n, n)
    psi = psi.to(torch.complex64).contiguous()
    got = plan.structure_function(0, psi, 2)
    r = 2 * math.pi * np.arange(n // 2 + 1) / n
    want = (2 * alpha * a * k) ** 2 * (1 - np.cos(k * r))
    peak = (2 * alpha * a * k) ** 2 * 2
    assert np.max(np.abs(got[0] - want)) <= 2e-5 * peak
    assert np.max(np.abs(got[1:])) <= 2e-5 * peak


def test_structure_function_large_separation_against_mean_square():
    """strfunc-verif on a float64 field: S^2_j(r) = 2 <v_j^2> - 2 C_j(r) exactly (Wiener-Khinchin,
    C from torch's FFT of the oracle velocity), which tends to 2 <v_j^2> when C decays."""
    n = 32
    plan = _plan(n, GP_FP64)
    a, b = plan.coefficients()
    psi = random_psi(n, 77, amp_jitter=0.2)
    got = plan.structure_function(0, to_gpu(psi, np.complex128), 2)
    v = OSF.velocity(psi, OS.Params(n=n, alpha=a, beta=b, dt=0.004))
    for j, ax in enumerate((2, 1, 0)):
        f = np.fft.fft(v[j], axis=ax)
        c = np.mean(np.moveaxis(np.real(np.fft.ifft(np.abs(f) ** 2, axis=ax)), ax, 0).reshape(n, -1), axis=1) / n
        want = 2 * np.mean(v[j] ** 2) - 2 * c[: n // 2 + 1]
        assert np.max(np.abs(got[j] - want)) <= 1e-11 * np.max(np.abs(want))


def test_structure_function_rejects_bad_arguments():
    plan = _plan(16, GP_FP32)
    psi = torch.ones((16, 16, 16), dtype=torch.complex64, device="cuda")
    for order in (0, 9):
        with pytest.raises(GPError):
            plan.structure_function(0, psi, order)
    bad = psi.clone()
    bad[3, 4, 5] = float("nan")
    with pytest.raises(GPError):
        plan.structure_function(0, bad, 2)

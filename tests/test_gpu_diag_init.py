"""GPU diagnostics and initial conditions against the float64 CPU oracle."""
import math

import numpy as np
import pytest

from inputs import random_psi, smooth_psi
from oracle import diagnostics as OD
from oracle import initial as OI
from oracle import scheme as OS
from tests._util import rel_l2, to_gpu, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2003_03590_gb300 import GP_FP32, GP_FP64, GPError, Plan, field_params  # noqa: E402


def _plan(n, prec, dt=0.004, ratio=1.5):
    return Plan(field_params(n, dt, xi_over_dx=ratio, precision=prec))


def _oparams(plan):
    a, b = plan.coefficients()
    return OS.Params(n=plan.n(), alpha=a, beta=b, dt=0.004)


@pytest.mark.parametrize("n", [16, 24, 32, 48])
@pytest.mark.parametrize("prec", [GP_FP32, GP_FP64])
def test_diagnostics_parity(n, prec):
    plan = _plan(n, prec)
    dtype = np.complex128 if prec == GP_FP64 else np.complex64
    psi0 = random_psi(n, n, amp_jitter=0.25).astype(dtype)
    d, spec = plan.diagnostics(0, to_gpu(psi0, dtype))
    ref, rspec = OD.full(psi0.astype(np.complex128), _oparams(plan))
    tol = 1e-10 if prec == GP_FP64 else 2e-5
    for k in ref:
        assert abs(d[k] - ref[k]) <= tol * max(abs(ref[k]), 1e-3 * abs(ref["E"])), (k, d[k], ref[k])
    for k in rspec:
        scale = max(np.max(np.abs(rspec[k])), 1e-30)
        assert np.max(np.abs(spec[k] - rspec[k])) <= tol * 10 * scale, k


def test_diagnostics_sound_wave_and_srp():
    n = 32
    plan = _plan(n, GP_FP64)
    p = _oparams(plan)
    x = 2 * np.pi * np.arange(n) / n
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    d, _ = plan.diagnostics(0, to_gpu(np.exp(0.1j * np.sin(X)), np.complex128))
    assert abs(d["E_kin_c"] - p.alpha ** 2 * 0.01) < 1e-12 and abs(d["E_kin_i"]) < 1e-18
    # SRP at t = 0 is vortex free: once resolved (48^3, k0 = 2) its kinetic energy is compressible
    n = 48
    plan = _plan(n, GP_FP64)
    psi = OI.srp_spectral(n, 1, 2.0)
    d, _ = plan.diagnostics(0, to_gpu(psi, np.complex128))
    assert d["E_kin_c"] > 1e6 * max(d["E_kin_i"], 1e-300)


@pytest.mark.parametrize("prec", [GP_FP32, GP_FP64])
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_momentum_and_mach_of_a_plane_wave(prec, axis):
    """psi = exp(i m x_j): rho = 1 and v = 2 alpha m e_j everywhere, so P = 2 alpha m e_j,
    M_max = M_rms = 2 alpha m / sqrt(2 alpha beta) exactly (eq-mom-total, eq:Mach-Number)."""
    n, m = 32, 3
    plan = _plan(n, prec)
    a, b = plan.coefficients()
    dtype = np.complex128 if prec == GP_FP64 else np.complex64
    x = 2 * np.pi * np.arange(n) / n
    grids = np.meshgrid(x, x, x, indexing="ij")       # [z, y, x]
    coord = grids[2 - axis]
    d, _ = plan.diagnostics(0, to_gpu(np.exp(1j * m * coord), dtype))
    tol = 1e-12 if prec == GP_FP64 else 2e-6
    want = [0.0, 0.0, 0.0]
    want[axis] = 2 * a * m
    for j, name in enumerate(("P_x", "P_y", "P_z")):
        assert abs(d[name] - want[j]) <= tol * 2 * a * m, (name, d[name], want[j])
    mach = 2 * a * m / math.sqrt(2 * a * b)
    assert d["M_max"] == pytest.approx(mach, rel=10 * tol)
    assert d["M_rms"] == pytest.approx(mach, rel=10 * tol)


def test_momentum_is_odd_under_conjugation_and_mach_even():
    """psi -> conj(psi) reverses every velocity: P -> -P, the Mach numbers stay."""
    n = 32
    plan = _plan(n, GP_FP64)
    psi = random_psi(n, 5, amp_jitter=0.25)
    d, _ = plan.diagnostics(0, to_gpu(psi, np.complex128))
    c, _ = plan.diagnostics(0, to_gpu(np.conj(psi), np.complex128))
    for name in ("P_x", "P_y", "P_z"):
        assert abs(d[name] + c[name]) <= 1e-12 * max(abs(d[name]), 1e-3 * d["E"]), name
    for name in ("M_max", "M_rms"):
        assert c[name] == pytest.approx(d[name], rel=1e-12), name


def test_diagnostics_rejects_nonfinite():
    n = 16
    plan = _plan(n, GP_FP32)
    psi = random_psi(n, 1).astype(np.complex64)
    psi[3, 4, 5] = np.nan
    with pytest.raises(GPError) as e:
        plan.diagnostics(0, to_gpu(psi, np.complex64))
    assert e.value.status == 6


@pytest.mark.parametrize("prec", [GP_FP32, GP_FP64])
@pytest.mark.parametrize("n,k0", [(24, 3.0), (64, 4.0)])
def test_init_srp_spectral(prec, n, k0):
    plan = _plan(n, prec)
    psi = plan.init_srp(0, plan.empty(), seed=5, mode=0, p0=k0, p1=math.pi)
    ref = OI.srp_spectral(n, 5, k0)
    assert rel_l2(to_np(psi), ref) < (1e-12 if prec == GP_FP64 else 2e-7)


def test_init_srp_spectral_is_reproducible():
    """The RMS normalisation is a sum formed in a fixed order: the same seed gives the same
    field bit for bit, call after call (checked at 256^3, where the sum spans many blocks)."""
    plan = _plan(256, GP_FP32)
    a = plan.init_srp(0, plan.empty(), seed=3, mode=0, p0=8.0, p1=math.pi)
    b = plan.init_srp(0, plan.empty(), seed=3, mode=0, p0=8.0, p1=math.pi)
    c = plan.init_srp(0, plan.empty(), seed=4, mode=0, p0=8.0, p1=math.pi)
    plan.sync()
    assert torch.equal(a, b)
    assert not torch.equal(a, c)


@pytest.mark.parametrize("n,nr", [(16, 4), (48, 4), (24, 3)])
def test_init_srp_spline(n, nr):
    plan = _plan(n, GP_FP64)
    K = 8 * math.pi
    psi = plan.init_srp(0, plan.empty(), seed=2, mode=1, p0=K, p1=nr)
    ref = OI.srp_spline(n, 2, K, nr)
    assert rel_l2(to_np(psi), ref) < 1e-12


@pytest.mark.parametrize("prec", [GP_FP32, GP_FP64])
def test_init_rvr_rings(prec):
    n = 32
    plan = _plan(n, prec)
    a, b = plan.coefficients()
    xi = math.sqrt(a / b)
    psi = plan.init_rvr(0, plan.empty(), seed=0, mode=0, count=40, p0=4 * xi, p1=12 * xi)
    ref = OI.rvr_tanh(n, 0, xi, 40, 4 * xi, 12 * xi)
    assert rel_l2(to_np(psi), ref) < (1e-12 if prec == GP_FP64 else 2e-7)


def test_init_rvr_rings_config_size_sampled():
    """256^3 with 40 rings: sampled points against the oracle's pointwise product."""
    n = 256
    plan = _plan(n, GP_FP32, dt=0.002)
    a, b = plan.coefficients()
    xi = math.sqrt(a / b)
    psi = plan.init_rvr(0, plan.empty(), seed=0, mode=0, count=40, p0=4 * xi, p1=12 * xi)
    rng = np.random.default_rng(0)
    pts = rng.integers(0, n, size=(4000, 3))
    ti = torch.as_tensor(pts, device="cuda")
    got = psi[ti[:, 0], ti[:, 1], ti[:, 2]].cpu().numpy().astype(np.complex128)
    R, c, nv = OI.rvr_rings(0, 40, 4 * xi, 12 * xi)
    xyz = np.stack([pts[:, 2], pts[:, 1], pts[:, 0]], axis=1) * (2 * np.pi / n)
    ref = OI.rvr_tanh_points(xyz, xi, R, c, nv)
    assert np.max(np.abs(got - ref)) < 2e-6


@pytest.mark.parametrize("n", [16, 24])
def test_init_rvr_pade_pairs(n):
    plan = _plan(n, GP_FP64, ratio=2.0)
    a, b = plan.coefficients()
    xi = math.sqrt(a / b)
    psi = plan.init_rvr(0, plan.empty(), seed=3, mode=1, count=3, p0=0.5 * math.pi, p1=math.pi)
    ref = OI.rvr_pade(n, 3, xi, 3)
    assert rel_l2(to_np(psi), ref) < 1e-11


def test_psi_from_phase_and_invalid_calls():
    n = 16
    plan = _plan(n, GP_FP32)
    th = torch.rand((n, n, n), device="cuda") * 6
    psi = plan.psi_from_phase(0, th)
    assert torch.allclose(psi, torch.polar(torch.ones_like(th), th), atol=2e-7)
    with pytest.raises(GPError) as e:
        plan.init_srp(0, psi, seed=1, mode=1, p0=1.0, p1=5)     # 16 % 5 != 0
    assert e.value.status == 1
    with pytest.raises(GPError):
        plan.init_rvr(0, psi, seed=1, mode=7)

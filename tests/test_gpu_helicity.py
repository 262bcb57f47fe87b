"""GPU helicity and regularised helicity (Sec. 3.6: eq-helicity, Hreg) against the float64 oracle,
their mirror antisymmetry at the benchmark grid size, and the argument checks of the C ABI.
(The paper's values for the prepared ABC and TG fields are checked with the ARGLE tests.)"""
import numpy as np
import pytest

from inputs import random_psi, smooth_psi
from oracle import helicity as OH
from oracle import scheme as OS
from oracle import structure as OSF
from oracle.diagnostics import gradient
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


def _integrand_scale(psi, p):
    """<|v| |omega|>: the size of the terms whose mean the helicities are."""
    v = OSF.velocity(psi, p, gradient(psi))
    om = OH.curl(v)
    return float(np.mean(np.sqrt(sum(c * c for c in v)) * np.sqrt(sum(c * c for c in om))))


@pytest.mark.parametrize("prec", [GP_FP64, GP_FP32])
@pytest.mark.parametrize("n,kind", [(16, "random"), (24, "smooth"), (32, "random"), (48, "smooth")])
def test_helicities_match_oracle(n, kind, prec):
    plan = _plan(n, prec)
    a, b = plan.coefficients()
    p = OS.Params(n=n, alpha=a, beta=b, dt=0.004)
    psi = (random_psi(n, 60 + n, amp_jitter=0.3) if kind == "random" else smooth_psi(n, 60 + n, amp=2.0))
    psi = psi.astype(_dtype(prec))
    got, gspec = plan.helicity(0, to_gpu(psi, _dtype(prec)))
    (h, hr), (sh, shr) = OH.helicities(psi.astype(np.complex128), p)
    scale = _integrand_scale(psi.astype(np.complex128), p)
    tol = 1e-10 if prec == GP_FP64 else 2e-4
    print(n, kind, prec, got, (h, hr), scale)
    assert abs(got["H"] - h) <= tol * scale
    assert abs(got["H_reg"] - hr) <= tol * scale
    assert np.max(np.abs(gspec["H"] - sh)) <= tol * scale
    assert np.max(np.abs(gspec["H_reg"] - shr)) <= tol * scale
    assert np.sum(gspec["H"]) == pytest.approx(got["H"], rel=1e-9, abs=1e-12 * scale)


def _mirror_x(psi):
    n = psi.shape[2]
    return psi[:, :, (-np.arange(n)) % n]


@pytest.mark.parametrize("n", [64, 256])
def test_helicities_are_pseudoscalars_at_size(n):
    """x -> -x reverses both helicities and every shell of their spectra; psi -> conj(psi) keeps
    them: float32 path at the benchmark size (the oracle cannot run there; the symmetry holds at
    any size)."""
    plan = _plan(n, GP_FP32)
    psi = smooth_psi(n, 5, nmodes=24, kmax=6, amp=2.5).astype(np.complex64)
    d, s = plan.helicity(0, to_gpu(psi, np.complex64))
    m, sm = plan.helicity(0, to_gpu(np.ascontiguousarray(_mirror_x(psi)), np.complex64))
    c, sc = plan.helicity(0, to_gpu(np.conj(psi), np.complex64))
    for k in ("H", "H_reg"):
        scale = float(np.sum(np.abs(s[k])))      # bounds |H| and every shell
        assert abs(d[k]) > 1e-2 * scale
        assert abs(m[k] + d[k]) <= 1e-4 * scale, (k, d[k], m[k])
        assert abs(c[k] - d[k]) <= 1e-4 * scale, (k, d[k], c[k])
        assert np.max(np.abs(sm[k] + s[k])) <= 1e-4 * scale


def test_helicity_rejects_bad_arguments():
    plan = _plan(16, GP_FP32)
    psi = torch.ones((16, 16, 16), dtype=torch.complex64, device="cuda")
    bad = psi.clone()
    bad[1, 2, 3] = float("inf")
    with pytest.raises(GPError):
        plan.helicity(0, bad)
    d, _ = plan.helicity(0, psi)
    assert d["H"] == 0.0 and d["H_reg"] == 0.0

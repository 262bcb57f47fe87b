"""gp_diagnostics_noalloc -- the diagnostics for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc: an application whose caching allocator already owns the
device's memory, or a monitoring hook in a latency-critical loop where an allocation would stall
every stream.  For them the library offers one entry point that works entirely in fixed device
arrays reserved when the library is loaded (fields up to 64^3).  This file checks, through the C
ABI, that it gives the same energies, mass and spectra as the plan-based gp_diagnostics and as the
float64 oracle on consecutive calls (each call reuses the arrays the one before left behind; the
sequence 32, 64, 48 fills the arrays to their limit and then shrinks), and that a size above its
limit is refused.  It is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

from inputs import random_psi
from oracle import diagnostics as OD
from oracle import scheme as OS

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2003_03590_gb300 import GP_FP32, Plan, _lib, field_params  # noqa: E402

TOL = 2e-5   # the tolerance of the float32 diagnostics parity tests


def _noalloc(n, alpha, beta, psi, nbins):
    L = _lib.load()
    d = _lib.Diag()
    spec = np.zeros(4 * nbins)
    st = L.gp_diagnostics_noalloc(n, alpha, beta, ctypes.c_void_p(psi.data_ptr()), ctypes.byref(d),
                                  spec.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), nbins,
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, {k: getattr(d, k) for k in _lib.DIAG_NAMES}, spec.reshape(4, nbins)


def _close(got, ref, spec, rspec, what):
    for k in ref:
        assert abs(got[k] - ref[k]) <= TOL * max(abs(ref[k]), 1e-3 * abs(ref["E"])), (what, k, got[k], ref[k])
    for q, name in enumerate(("E_kin_i", "E_kin_c", "E_q", "E_int")):
        scale = max(np.max(np.abs(rspec[name])), 1e-30)
        assert np.max(np.abs(spec[q] - rspec[name])) <= 10 * TOL * scale, (what, name)


def test_noalloc_matches_plan_diagnostics_and_oracle_on_consecutive_calls():
    for call, (n, seed) in enumerate(((32, 11), (32, 12), (64, 14), (48, 13))):
        plan = Plan(field_params(n, 0.004, xi_over_dx=1.5, precision=GP_FP32))
        alpha, beta = plan.coefficients()
        psi_np = random_psi(n, seed, amp_jitter=0.25).astype(np.complex64)
        psi = torch.from_numpy(psi_np).cuda()
        ref, rspec = plan.diagnostics(0, psi)
        nb = plan.nbins()
        st, got, spec = _noalloc(n, alpha, beta, psi, nb)
        assert st == 0, (call, _lib.STATUS.get(st))
        _close(got, ref, spec, rspec, f"call {call}: plan")
        oref, ospec = OD.full(psi_np.astype(np.complex128), OS.Params(n=n, alpha=alpha, beta=beta, dt=0.004))
        _close(got, {k: oref[k] for k in ref if k in oref}, spec, ospec, f"call {call}: oracle")


def test_noalloc_refuses_sizes_beyond_its_arrays():
    psi = torch.zeros((96, 96, 96), dtype=torch.complex64, device="cuda")
    st, _, _ = _noalloc(96, 0.1, 20.0, psi, 100)
    assert _lib.STATUS[st] == "GP_ERR_UNSUPPORTED_SIZE"

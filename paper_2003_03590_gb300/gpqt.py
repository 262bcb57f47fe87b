"""Python binding of the C ABI (include/gp.h): argument marshalling only.

Every operation runs in libgpqt.so's CUDA kernels; torch provides device
memory and the stream.  Fields are contiguous torch tensors on the GPU,
complex64 for GP_FP32 plans and complex128 for GP_FP64 plans, shaped
(N, N, N) and indexed [z, y, x].
"""
import ctypes
import math

import numpy as np
import torch

from . import _lib
from ._lib import (DIAG_NAMES, GP_FLOW_ABC, GP_FLOW_NONE, GP_FLOW_TG, GP_FP32, GP_FP64, GP_SPLIT_KNK, GP_SPLIT_NKN,
                   OP_PLANE, SUPPORTED_N, VARIANT_PLAIN,
                   VARIANT_TMA, VARIANT_TMA_2STAGE, VARIANT_TMA_GROUPS, VARIANT_TMA_ONE, Diag, FieldParams,
                   GPError)


def field_params(n, dt, xi=None, xi_over_dx=None, alpha=0.0, beta=0.0, precision=GP_FP32, split=GP_SPLIT_NKN,
                 minus_one=True):
    """Parameters of one field; give xi, or xi_over_dx (xi = ratio * 2 pi / N), or alpha and beta."""
    if xi is None and xi_over_dx is not None:
        xi = xi_over_dx * 2.0 * math.pi / n
    return FieldParams(n=n, xi=float(xi or 0.0), alpha=float(alpha), beta=float(beta), dt=float(dt),
                       precision=int(precision), split=int(split), nonlin_minus_one=1 if minus_one else 0)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


class Plan:
    """A gp_plan: one or more fields (a ragged batch) advanced together on one CUDA stream."""

    def __init__(self, fields, stream=None):
        self._lib = _lib.load()
        if isinstance(fields, FieldParams):
            fields = [fields]
        self.fields = list(fields)
        arr = (FieldParams * len(self.fields))(*self.fields)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = ctypes.c_void_p()
        st = self._lib.gp_plan_create(arr, len(self.fields), ctypes.c_void_p(stream.cuda_stream), ctypes.byref(h))
        if st != 0:
            raise GPError(st, "gp_plan_create failed")
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.gp_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != 0:
            msg = self._lib.gp_last_error(self._h)
            raise GPError(st, msg.decode() if msg else "")

    # ---- properties
    def n(self, field=0):
        return self.fields[field].n

    def dtype(self, field=0):
        return torch.complex128 if self.fields[field].precision == GP_FP64 else torch.complex64

    def real_dtype(self, field=0):
        return torch.float64 if self.fields[field].precision == GP_FP64 else torch.float32

    def coefficients(self, field=0):
        a, b = ctypes.c_double(), ctypes.c_double()
        self._check(self._lib.gp_plan_coefficients(self._h, field, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def nbins(self, field=0):
        return self._lib.gp_plan_nbins(self._h, field)

    def empty(self, field=0):
        n = self.n(field)
        return torch.empty((n, n, n), dtype=self.dtype(field), device="cuda")

    def _field(self, t, field):
        n = self.n(field)
        if not (t.is_cuda and t.is_contiguous() and t.dtype == self.dtype(field) and tuple(t.shape) == (n, n, n)):
            raise ValueError(f"field {field}: need a contiguous CUDA {self.dtype(field)} tensor of shape {(n, n, n)}")
        return t

    # ---- C ABI calls
    def init_srp(self, field, psi, seed, mode=0, p0=4.0, p1=math.pi):
        self._check(self._lib.gp_init_srp(self._h, field, _ptr(self._field(psi, field)), seed, mode, p0, p1))
        return psi

    def init_rvr(self, field, psi, seed, mode=0, count=40, p0=0.0, p1=0.0):
        self._check(self._lib.gp_init_rvr(self._h, field, _ptr(self._field(psi, field)), seed, mode, count, p0, p1))
        return psi

    # ---- imaginary-time preparation (see gp.h)
    @staticmethod
    def _abc_arg(abc):
        if abc is None:
            return None, None
        arr = (ctypes.c_double * 3)(*[float(a) for a in abc])
        return ctypes.cast(arr, ctypes.c_void_p), arr

    def init_tg(self, field, psi):
        """Taylor-Green start field psi_ARGLE (Sec. 5.1) into psi."""
        self._check(self._lib.gp_init_tg(self._h, field, _ptr(self._field(psi, field))))
        return psi

    def init_abc(self, field, psi, abc=None):
        """ABC start field (Sec. 5.2); abc = (A, B, C) or None for (0.9, 1, 1.1)/sqrt(3)."""
        ptr, _keep = self._abc_arg(abc)
        self._check(self._lib.gp_init_abc(self._h, field, _ptr(self._field(psi, field)), ptr))
        return psi

    def argle(self, field, psi, flow, dtau, nsteps, abc=None, renorm=False, energy=True):
        """nsteps imaginary-time (ARGLE) steps in place; returns E_v after them (or None)."""
        ptr, _keep = self._abc_arg(abc)
        e = ctypes.c_double()
        self._check(self._lib.gp_argle(self._h, field, _ptr(self._field(psi, field)), int(flow), ptr, float(dtau),
                                       int(nsteps), 1 if renorm else 0, ctypes.byref(e) if energy else None))
        return e.value if energy else None

    def argle_converge(self, field, psi, flow, dtau, max_steps, eps, check_every=100, abc=None, renorm=False,
                       energy=True):
        """ARGLE steps in place until ||phi^{n+1} - phi^n||_inf / dtau <= eps at a checked step (every
        check_every steps and the last) or max_steps; returns (steps_done, crit1, crit2, E_v or None)."""
        ptr, _keep = self._abc_arg(abc)
        done, c1, c2, e = ctypes.c_int(), ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        self._check(self._lib.gp_argle_converge(self._h, field, _ptr(self._field(psi, field)), int(flow), ptr,
                                                float(dtau), int(max_steps), 1 if renorm else 0, float(eps),
                                                int(check_every), ctypes.byref(done), ctypes.byref(c1),
                                                ctypes.byref(c2), ctypes.byref(e) if energy else None))
        return done.value, c1.value, c2.value, (e.value if energy else None)

    def psi_from_phase(self, field, theta, out=None):
        if out is None:
            out = self.empty(field)
        theta = theta.contiguous()
        if theta.dtype != self.real_dtype(field) or not theta.is_cuda:
            raise ValueError("theta must be a CUDA tensor of the plan's real dtype")
        self._check(self._lib.gp_psi_from_phase(self._h, field, _ptr(theta), _ptr(self._field(out, field))))
        return out

    def step(self, psis, nsteps):
        if isinstance(psis, torch.Tensor):
            psis = [psis]
        if len(psis) != len(self.fields):
            raise ValueError("one tensor per field")
        arr = (ctypes.c_void_p * len(psis))(*[self._field(t, i).data_ptr() for i, t in enumerate(psis)])
        self._check(self._lib.gp_step(self._h, arr, int(nsteps)))
        return psis

    def step_host(self, arrays, nsteps):
        """Step host-resident fields (numpy arrays or CPU tensors, pinned if possible) in place."""
        if not isinstance(arrays, (list, tuple)):
            arrays = [arrays]
        ptrs = []
        for i, a in enumerate(arrays):
            n = self.n(i)
            if isinstance(a, torch.Tensor):
                if a.is_cuda or not a.is_contiguous() or a.dtype != self.dtype(i) or a.numel() != n ** 3:
                    raise ValueError("host tensors must be contiguous CPU tensors of the plan's dtype")
                ptrs.append(a.data_ptr())
            else:
                want = np.complex128 if self.fields[i].precision == GP_FP64 else np.complex64
                if a.dtype != want or not a.flags.c_contiguous or a.size != n ** 3:
                    raise ValueError("host arrays must be C-contiguous of the plan's dtype")
                ptrs.append(a.ctypes.data)
        arr = (ctypes.c_void_p * len(ptrs))(*ptrs)
        self._check(self._lib.gp_step_host(self._h, arr, int(nsteps)))
        return arrays

    def diagnostics(self, field, psi, spectra=True):
        d = Diag()
        nb = self.nbins(field)
        spec = np.zeros(4 * nb) if spectra else None
        sp = spec.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if spectra else None
        self._check(self._lib.gp_diagnostics(self._h, field, _ptr(self._field(psi, field)), ctypes.byref(d), sp, nb))
        out = {k: getattr(d, k) for k in DIAG_NAMES}
        if not spectra:
            return out, None
        spec = spec.reshape(4, nb)
        return out, {"E_kin_i": spec[0], "E_kin_c": spec[1], "E_q": spec[2], "E_int": spec[3]}

    def structure_function(self, field, psi, order=2):
        """S^order along x, y, z at the separations s 2 pi / N, s = 0 .. N/2: array [3, N/2 + 1]."""
        ns = self.n(field) // 2 + 1
        out = np.zeros(3 * ns)
        self._check(self._lib.gp_structure_function(self._h, field, _ptr(self._field(psi, field)), int(order),
                                                    out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ns))
        return out.reshape(3, ns)

    def helicity(self, field, psi, spectra=True):
        """({"H", "H_reg"}, {"H": H(k), "H_reg": H_reg(k)} or None) of the field (see gp.h)."""
        h, hr = ctypes.c_double(), ctypes.c_double()
        nb = self.nbins(field)
        spec = np.zeros(2 * nb) if spectra else None
        sp = spec.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if spectra else None
        self._check(self._lib.gp_helicity(self._h, field, _ptr(self._field(psi, field)), ctypes.byref(h),
                                          ctypes.byref(hr), sp, nb))
        out = {"H": h.value, "H_reg": hr.value}
        if not spectra:
            return out, None
        return out, {"H": spec[:nb].copy(), "H_reg": spec[nb:].copy()}

    def adjoint_step(self, field, psi_n, lam, nsteps):
        self._check(self._lib.gp_adjoint_step(self._h, field, _ptr(self._field(psi_n, field)),
                                              _ptr(self._field(lam, field)), int(nsteps)))
        return lam

    def ekin_i_grad(self, field, psi, eps=1e-6, lam=None):
        if lam is None:
            lam = self.empty(field)
        J = ctypes.c_double()
        self._check(self._lib.gp_ekin_i_grad(self._h, field, _ptr(self._field(psi, field)),
                                             _ptr(self._field(lam, field)), float(eps), ctypes.byref(J)))
        return lam, J.value

    def autotune(self, cache_path=None):
        """Pick the fastest float32 sweep kernel per grid length and sweep kind (see gp.h)."""
        path = None if cache_path is None else str(cache_path).encode()
        self._check(self._lib.gp_plan_autotune(self._h, path))
        return self

    def sweep_variant(self, n, axis, op):
        return self._lib.gp_plan_sweep_variant(self._h, n, axis, op)

    def sync(self):
        """Wait for the plan's stream; raises GPError(GP_ERR_TIMEOUT) if a sweep kernel gave up a
        bounded wait since the last check."""
        self._check(self._lib.gp_plan_sync(self._h))
        return self

    def test_timeout(self, tiles):
        """Make the next fused-kernel launch skip its first `tiles` tiles (a test of the bounded
        waits: the launch ends with the status word set; see gp.h)."""
        self._check(self._lib.gp_plan_test_timeout(self._h, int(tiles)))
        return self

    def set_sweep_variant(self, n, axis, op, variant):
        """Choose the kernel of one sweep kind by hand (see gp.h); returns self."""
        self._check(self._lib.gp_plan_set_sweep_variant(self._h, n, axis, op, variant))
        return self

    def set_fused_batch(self, on=True):
        """Advance every field of a step call in one persistent launch (see gp.h); returns self."""
        self._check(self._lib.gp_plan_set_fused_batch(self._h, 1 if on else 0))
        return self

    def phase_grad(self, field, psi, lam):
        n = self.n(field)
        g = torch.empty((n, n, n), dtype=self.real_dtype(field), device="cuda")
        self._check(self._lib.gp_phase_grad(self._h, field, _ptr(self._field(psi, field)),
                                            _ptr(self._field(lam, field)), _ptr(g)))
        return g


def profile(plan, enable=True):
    plan._check(plan._lib.gp_profile(plan._h, 1 if enable else 0))


def profile_read(plan, max_kinds=64):
    names = ctypes.create_string_buffer(64 * max_kinds)
    launches = (ctypes.c_longlong * max_kinds)()
    ms = (ctypes.c_double * max_kinds)()
    k = plan._lib.gp_profile_read(plan._h, max_kinds, names, launches, ms)
    if k < 0:
        raise GPError(4, "gp_profile_read failed")
    out = {}
    for q in range(k):
        nm = names.raw[64 * q:64 * (q + 1)].split(b"\0", 1)[0].decode()
        out[nm] = (int(launches[q]), float(ms[q]))
    return out


def launch_count(plan):
    return int(plan._lib.gp_launch_count(plan._h))


class GPEvolve(torch.autograd.Function):
    """psi_T = S^nsteps(exp(i theta)) with a checkpointed adjoint backward.

    Forward keeps the state every ``every`` steps; backward recomputes each
    segment from its checkpoint inside gp_adjoint_step and pulls the cotangent
    back through it, then returns dJ/dtheta = -Im(conj(lam_0) psi_0).
    The plan must hold a single field.
    """

    @staticmethod
    def forward(ctx, theta, plan, nsteps, every):
        psi0 = plan.psi_from_phase(0, theta.detach())
        psi = psi0.clone()
        ckpts = []
        done = 0
        while done < nsteps:
            k = min(every, nsteps - done)
            ckpts.append((psi.clone(), k))
            plan.step([psi], k)
            done += k
        ctx.plan = plan
        ctx.ckpts = ckpts
        ctx.save_for_backward(psi0)
        return psi

    @staticmethod
    def backward(ctx, grad_psi):
        (psi0,) = ctx.saved_tensors
        lam = grad_psi.contiguous().clone()
        for state, k in reversed(ctx.ckpts):
            ctx.plan.adjoint_step(0, state, lam, k)
        return ctx.plan.phase_grad(0, psi0, lam), None, None, None


class IncompressibleKineticEnergy(torch.autograd.Function):
    """J = E_kin^i(psi) with |psi| regularised by eps inside sqrt(rho) v; backward uses gp_ekin_i_grad."""

    @staticmethod
    def forward(ctx, psi, plan, eps):
        lam, J = plan.ekin_i_grad(0, psi.detach().contiguous(), eps)
        ctx.save_for_backward(lam)
        return torch.tensor(J, dtype=torch.float64, device=psi.device)

    @staticmethod
    def backward(ctx, gJ):
        (lam,) = ctx.saved_tensors
        return lam * gJ.to(lam.real.dtype), None, None

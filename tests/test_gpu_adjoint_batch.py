"""GPU adjoint and gradient against the oracle and finite differences; batched and host-buffer paths."""
import math

import numpy as np
import pytest

from inputs import random_direction, random_psi
from oracle import adjoint as OA
from oracle import initial as OI
from oracle import scheme as OS
from tests._util import rel_l2, to_gpu, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2003_03590_gb300 import (GP_FP32, GP_FP64, GP_SPLIT_KNK, GP_SPLIT_NKN, GPEvolve,  # noqa: E402
                                    IncompressibleKineticEnergy, Plan, field_params)
from paper_2003_03590_gb300.gpqt import (OP_PLANE, VARIANT_PLAIN, VARIANT_TMA, VARIANT_TMA_2STAGE,  # noqa: E402
                                         VARIANT_TMA_ONE)


def _op(plan, dt):
    a, b = plan.coefficients()
    return OS.Params(n=plan.n(), alpha=a, beta=b, dt=dt)


@pytest.mark.parametrize("prec", [GP_FP64, GP_FP32])
@pytest.mark.parametrize("split", [GP_SPLIT_NKN, GP_SPLIT_KNK])
def test_adjoint_segment_matches_oracle(prec, split):
    n, dt, m = 16, 0.004, 5
    plan = Plan(field_params(n, dt, xi_over_dx=1.5, precision=prec, split=split))
    dtype = np.complex128 if prec == GP_FP64 else np.complex64
    psi0 = random_psi(n, 1, amp_jitter=0.2).astype(dtype)
    lam_T = random_direction(n, 2).astype(dtype)
    lam = to_gpu(lam_T, dtype)
    plan.adjoint_step(0, to_gpu(psi0, dtype), lam, m)
    p = _op(plan, dt)
    order = "nkn" if split == GP_SPLIT_NKN else "knk"
    states = OA.forward_states(psi0.astype(np.complex128), p, m, order)
    ref = lam_T.astype(np.complex128)
    for k in range(m - 1, -1, -1):
        ref = OA.vjp_step(states[k], ref, p, order)
    assert rel_l2(to_np(lam), ref) < (1e-11 if prec == GP_FP64 else 2e-5)


@pytest.mark.parametrize("prec", [GP_FP64, GP_FP32])
def test_ekin_i_gradient_matches_oracle(prec):
    n = 24
    plan = Plan(field_params(n, 0.004, xi_over_dx=1.5, precision=prec))
    dtype = np.complex128 if prec == GP_FP64 else np.complex64
    psi = random_psi(n, 4, amp_jitter=0.2).astype(dtype)
    lam, J = plan.ekin_i_grad(0, to_gpu(psi, dtype), 1e-6)
    p = _op(plan, 0.004)
    Jr = OA.ekin_i_reg(psi.astype(np.complex128), p)
    lr = OA.ekin_i_reg_grad(psi.astype(np.complex128), p)
    tol = 1e-11 if prec == GP_FP64 else 5e-5
    assert abs(J - Jr) < tol * Jr
    assert rel_l2(to_np(lam), lr) < tol


def test_autograd_gradient_vs_finite_differences_fp64():
    """dJ/dtheta through the checkpointed adjoint, FP64, vs centred differences (h = 1e-4)."""
    n, dt, m = 16, 0.004, 12
    plan = Plan(field_params(n, dt, xi_over_dx=1.5, precision=GP_FP64))
    # k0 = 2 keeps psi away from zero here (with k0 = 3 a vortex core forms, where the O(h^2) error
    # of the h = 1e-4 difference reaches 2e-2: the oracle shows the same)
    theta0 = torch.from_numpy(OI.srp_theta(n, 0, 2.0)).cuda()
    theta = theta0.clone().requires_grad_(True)
    psiT = GPEvolve.apply(theta, plan, m, 4)
    J = IncompressibleKineticEnergy.apply(psiT, plan, 1e-6)
    J.backward()
    g = theta.grad.detach()

    def Jof(th):
        psi = plan.psi_from_phase(0, th)
        plan.step([psi], m)
        return plan.ekin_i_grad(0, psi, 1e-6)[1]

    # h = 1e-4 (the configuration's check, relative error <= 1e-3) and h = 1e-5 (tighter: the
    # state holds near-zeros of psi, where the O(h^2) error of h = 1e-4 is ~1e-4)
    for seed in range(3):
        v = torch.from_numpy(np.real(random_direction(n, 50 + seed, complex_valued=False))).cuda()
        an = float((g * v).sum())
        for h, tol in ((1e-4, 1e-3), (1e-5, 1e-6)):
            fd = (Jof(theta0 + h * v) - Jof(theta0 - h * v)) / (2 * h)
            assert abs(fd - an) < tol * abs(fd), (seed, h, fd, an)
    # and against the oracle's adjoint gradient
    Jr, gr = OA.gradient_theta(theta0.cpu().numpy(), _op(plan, dt), m)
    assert abs(float(J) - Jr) < 1e-10 * Jr
    assert rel_l2(g.cpu().numpy(), gr) < 1e-8


def test_autograd_fp32_vs_fp64_adjoint():
    n, dt, m = 32, 0.004, 20
    th = torch.from_numpy(OI.srp_theta(n, 1, 4.0))
    grads = []
    for prec, rdt in ((GP_FP64, torch.float64), (GP_FP32, torch.float32)):
        plan = Plan(field_params(n, dt, xi_over_dx=1.5, precision=prec))
        t = th.to(rdt).cuda().requires_grad_(True)
        J = IncompressibleKineticEnergy.apply(GPEvolve.apply(t, plan, m, 5), plan, 1e-6)
        J.backward()
        grads.append(t.grad.double().cpu().numpy())
    assert rel_l2(grads[1], grads[0]) < 1e-3


def test_batched_ragged_plan_matches_single_plans_bitwise():
    dt = 0.004
    sizes = [16] * 3 + [24] * 2 + [32] * 2
    fields = [field_params(n, dt, xi_over_dx=1.5) for n in sizes]
    batch = Plan(fields)
    psis = [to_gpu(random_psi(n, 10 + i), np.complex64) for i, n in enumerate(sizes)]
    singles = [p.clone() for p in psis]
    batch.step(psis, 9)
    for i, n in enumerate(sizes):
        Plan(field_params(n, dt, xi_over_dx=1.5)).step([singles[i]], 9)
        assert torch.equal(psis[i], singles[i]), i


def test_batched_ragged_ensemble_against_the_oracle():
    """The configuration-4 size classes (64^3, 96^3 with radix-3 passes, 128^3, two fields each,
    xi = 1.5 dx, dt = 0.004, SRP starts made by the oracle) advanced together by one plan: one
    step and three steps of every field match the oracle to 1e-5 per step."""
    dt = 0.004
    sizes = [64, 64, 96, 96, 128, 128]
    batch = Plan([field_params(n, dt, xi_over_dx=1.5) for n in sizes])
    starts = [OI.srp_spectral(n, 40 + i, 4.0).astype(np.complex64).astype(np.complex128) for i, n in enumerate(sizes)]
    for steps in (1, 3):
        psis = [to_gpu(x, np.complex64) for x in starts]
        batch.step(psis, steps)
        batch.sync()
        for i, n in enumerate(sizes):
            p = OS.params_from_dx_ratio(n, 1.5, dt)
            ref = OS.evolve(starts[i], p, steps)
            assert rel_l2(to_np(psis[i]), ref) < 1e-5 * steps, (n, i, steps)


@pytest.mark.parametrize("split", [GP_SPLIT_NKN, GP_SPLIT_KNK])
def test_fused_plane_kernel_matches_separate_sweeps_bitwise(split):
    """The fused plane kernel (forward y, x with K, inverse y of every z-plane in one launch,
    synchronised per plane through global counters) computes exactly what the three separate
    sweeps compute: same arithmetic, only the schedule differs."""
    dt = 0.004
    sizes = [32, 32, 48, 64, 96, 128, 192, 256]
    fused = Plan([field_params(n, dt, xi_over_dx=1.5, split=split) for n in sizes])
    two = Plan([field_params(n, dt, xi_over_dx=1.5, split=split) for n in sizes])
    one = Plan([field_params(n, dt, xi_over_dx=1.5, split=split) for n in sizes])
    sep = Plan([field_params(n, dt, xi_over_dx=1.5, split=split) for n in sizes])
    for n in set(sizes):
        assert fused.sweep_variant(n, 1, OP_PLANE) == VARIANT_TMA       # the default
        two.set_sweep_variant(n, 1, OP_PLANE, VARIANT_TMA_2STAGE)      # two stages, twiddles via L1
        one.set_sweep_variant(n, 1, OP_PLANE, VARIANT_TMA_ONE)         # one CTA per SM (another lag)
        sep.set_sweep_variant(n, 1, OP_PLANE, VARIANT_PLAIN)
    fa = [to_gpu(random_psi(n, 70 + i), np.complex64) for i, n in enumerate(sizes)]
    fb = [f.clone() for f in fa]
    fc = [f.clone() for f in fa]
    fd = [f.clone() for f in fa]
    for steps in (5, 9):                    # the second call replays the captured cycle
        fused.step(fa, steps)
        sep.step(fb, steps)
        two.step(fc, steps)
        one.step(fd, steps)
        for p in (fused, sep, two, one):
            p.sync()                        # no bounded wait gave up
        for i, (x, y, z, w) in enumerate(zip(fa, fb, fc, fd)):
            assert torch.equal(x, y), sizes[i]
            assert torch.equal(z, y), sizes[i]
            assert torch.equal(w, y), sizes[i]


def test_bounded_wait_gives_up_and_reports_timeout():
    """Tiles whose inputs never complete: the fused kernel's waits give up (about a second), the
    launch ends, the status word reads as GP_ERR_TIMEOUT at the next check, and the plan and the
    CUDA context stay usable."""
    from paper_2003_03590_gb300 import GPError
    n = 32
    plan = Plan(field_params(n, 0.004, xi_over_dx=1.5))
    assert plan.sweep_variant(n, 1, OP_PLANE) == VARIANT_TMA
    psi = to_gpu(random_psi(n, 5), np.complex64)
    plan.test_timeout(1)                     # the first tile of plane 0 is never processed
    plan.step([psi], 1)
    with pytest.raises(GPError) as err:
        plan.sync()
    assert err.value.status == 5             # GP_ERR_TIMEOUT
    # usable afterwards: a clean step on a fresh field, checked against a fresh plan
    good = to_gpu(random_psi(n, 6), np.complex64)
    ref = good.clone()
    plan.step([good], 2)
    plan.sync()
    Plan(field_params(n, 0.004, xi_over_dx=1.5)).step([ref], 2)
    torch.cuda.synchronize()
    assert torch.equal(good, ref)


def test_two_stage_strided_kernels_bitwise():
    """The y and z TMA kernels with two shared-memory stages (one more CTA per SM) compute what
    the three-stage kernels compute."""
    dt = 0.004
    sizes = [32, 48, 64, 96, 128, 192, 256]
    ref = Plan([field_params(n, dt, xi_over_dx=1.5) for n in sizes])
    two = Plan([field_params(n, dt, xi_over_dx=1.5) for n in sizes])
    for n in sizes:
        for p in (ref, two):
            p.set_sweep_variant(n, 1, OP_PLANE, VARIANT_PLAIN)   # y sweeps as separate launches
        for axis, op in ((2, 3), (2, 4), (2, 5), (1, 1), (1, 2)):
            two.set_sweep_variant(n, axis, op, VARIANT_TMA_2STAGE)
    fa = [to_gpu(random_psi(n, 90 + i), np.complex64) for i, n in enumerate(sizes)]
    fb = [f.clone() for f in fa]
    ref.step(fa, 5)
    two.step(fb, 5)
    ref.sync()
    two.sync()
    for i, (x, y) in enumerate(zip(fa, fb)):
        assert torch.equal(x, y), sizes[i]


@pytest.mark.parametrize("n", [512, 1024])
def test_fused_plane_kernel_large_lengths_bitwise(n):
    """Lengths above 256: two TMA boxes per pencil, 8 or 4 pencils per tile."""
    dt = 0.001
    fused = Plan(field_params(n, dt, xi_over_dx=1.5))
    sep = Plan(field_params(n, dt, xi_over_dx=1.5)).set_sweep_variant(n, 1, OP_PLANE, VARIANT_PLAIN)
    g = torch.Generator(device="cuda").manual_seed(n)
    re = torch.rand((n, n, n), device="cuda", generator=g, dtype=torch.float32)
    im = torch.rand((n, n, n), device="cuda", generator=g, dtype=torch.float32)
    x = torch.complex(re - 0.5, im - 0.5)
    del re, im
    y = x.clone()
    fused.step([x], 2)
    sep.step([y], 2)
    fused.sync()
    sep.sync()
    assert torch.equal(x, y)


@pytest.mark.parametrize("n", [512, 1024])
def test_every_sweep_variant_bitwise_at_large_lengths(n):
    """Every kernel variant of every sweep kind of the step (TMA pipelined, one CTA per SM, plain
    one-tile-per-CTA with register caps, two stages, two compute groups per CTA, wide z tiles at 512)
    runs the same arithmetic: two steps agree bitwise with the default kernels."""
    from paper_2003_03590_gb300.gpqt import VARIANT_TMA_GROUPS
    dt = 0.001
    kinds = [(2, 4), (2, 3), (2, 5), (2, 1), (2, 2), (1, 1), (1, 2), (0, 6)]
    g = torch.Generator(device="cuda").manual_seed(n + 1)
    re = torch.rand((n, n, n), device="cuda", generator=g, dtype=torch.float32)
    im = torch.rand((n, n, n), device="cuda", generator=g, dtype=torch.float32)
    x0 = torch.complex(re - 0.5, im - 0.5)
    del re, im
    ref = x0.clone()
    Plan(field_params(n, dt, xi_over_dx=1.5)).step([ref], 2)
    for v in (VARIANT_TMA_ONE, VARIANT_PLAIN, VARIANT_TMA_2STAGE, VARIANT_TMA_GROUPS):
        plan = Plan(field_params(n, dt, xi_over_dx=1.5)).set_sweep_variant(n, 1, OP_PLANE, VARIANT_PLAIN)
        for a, o in kinds:
            if v == VARIANT_TMA_2STAGE and a == 0:
                continue
            plan.set_sweep_variant(n, a, o, v)
        x = x0.clone()
        plan.step([x], 2)
        plan.sync()
        assert torch.equal(x, ref), v
        del plan, x
    # the fused plane kernel: TMA stages, one CTA per SM, two stages, several compute groups
    for v in (VARIANT_TMA, VARIANT_TMA_ONE, VARIANT_TMA_2STAGE, VARIANT_TMA_GROUPS):
        plan = Plan(field_params(n, dt, xi_over_dx=1.5)).set_sweep_variant(n, 1, OP_PLANE, v)
        x = x0.clone()
        plan.step([x], 2)
        plan.sync()
        assert torch.equal(x, ref), ("plane", v)
        del plan, x
    torch.cuda.empty_cache()


def test_plans_stepped_from_two_host_threads():
    """Two plans on their own streams, stepped from two host threads at once (the library's
    per-launch argument blocks, tensor maps included, are per host thread): each field equals
    the same steps taken alone."""
    import threading
    n, steps = 128, 6
    starts = [to_gpu(random_psi(n, 90 + i), np.complex64) for i in range(2)]
    refs = []
    for x in starts:
        r = x.clone()
        Plan(field_params(n, 0.002, xi_over_dx=1.5)).step([r], steps)
        refs.append(r)
    torch.cuda.synchronize()
    plans = [Plan(field_params(n, 0.002, xi_over_dx=1.5), stream=torch.cuda.Stream()) for _ in range(2)]
    fields = [x.clone() for x in starts]
    torch.cuda.synchronize()
    errors = []

    def run(i):
        try:
            for _ in range(5):   # several calls: the first ones launch directly, later ones replay graphs
                plans[i].step([fields[i]], steps)
                plans[i].sync()
                fields[i].copy_(starts[i])
                torch.cuda.current_stream().synchronize()
            plans[i].step([fields[i]], steps)
            plans[i].sync()
        except Exception as e:  # noqa: BLE001 -- reported below
            errors.append(e)

    threads = [threading.Thread(target=run, args=(i,)) for i in range(2)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    torch.cuda.synchronize()
    assert not errors, errors
    for x, r in zip(fields, refs):
        assert torch.equal(x, r)


def test_host_buffer_step_matches_device_step():
    n = 32
    plan = Plan(field_params(n, 0.004, xi_over_dx=1.5))
    psi0 = random_psi(n, 8).astype(np.complex64)
    host = torch.from_numpy(psi0.copy()).pin_memory()
    plan.step_host([host], 6)
    dev = to_gpu(psi0, np.complex64)
    plan.step([dev], 6)
    assert torch.equal(host, dev.cpu())


def test_mixed_precision_batch():
    fields = [field_params(16, 0.004, xi_over_dx=1.5, precision=GP_FP64),
              field_params(16, 0.004, xi_over_dx=1.5, precision=GP_FP32)]
    plan = Plan(fields)
    psi0 = random_psi(16, 3)
    a = to_gpu(psi0, np.complex128)
    b = to_gpu(psi0, np.complex64)
    plan.step([a, b], 5)
    assert rel_l2(to_np(b), to_np(a)) < 5e-6


def test_repeated_call_replays_whole_run_graph_bitwise():
    """A gp_step call repeated with the same fields and step count replays one captured graph of
    the whole run; its result is bitwise the result of the launches it replaces."""
    dt = 0.004
    sizes = [16, 16, 24]
    a = Plan([field_params(n, dt, xi_over_dx=1.5) for n in sizes])
    b = Plan([field_params(n, dt, xi_over_dx=1.5) for n in sizes])
    fa = [to_gpu(random_psi(n, 40 + i), np.complex64) for i, n in enumerate(sizes)]
    fb = [f.clone() for f in fa]
    from paper_2003_03590_gb300.gpqt import launch_count
    for _ in range(3):                      # calls 2 and 3 of plan a replay the whole-run graph
        l0 = launch_count(a)
        a.step(fa, 7)
        # two groups (16^3 x2, 24^3); lengths without TMA kernels take 4 sweeps per step, + 1
        per_step = [2 if a.sweep_variant(n, 1, OP_PLANE) == VARIANT_TMA else 4 for n in (16, 24)]
        assert launch_count(a) - l0 == sum(k * 7 + 1 for k in per_step)
    other = [f.clone() for f in fa]
    for _ in range(3):                      # alternating field sets: never the whole-run graph
        b.step(fb, 7)
        b.step(other, 7)
    torch.cuda.synchronize()
    for x, y in zip(fa, fb):
        assert torch.equal(x, y)


def test_autotune_picks_variants_and_caches(tmp_path):
    dt = 0.004
    sizes = [32, 48]
    cache = tmp_path / "tune.json"
    tuned = Plan([field_params(n, dt, xi_over_dx=1.5) for n in sizes]).autotune(cache)
    text = cache.read_text()
    assert text.count("|") >= 2 * 8 * 3          # 8 sweep kinds per length, 3 separators per key
    for n in sizes:
        for axis, op in ((2, 3), (1, 1), (1, 2)):
            assert tuned.sweep_variant(n, axis, op) in (0, 1, 2, 3)
        assert tuned.sweep_variant(n, 0, 6) in (0, 1, 2)
        assert tuned.sweep_variant(n, 1, OP_PLANE) in (VARIANT_TMA, VARIANT_TMA_ONE, VARIANT_PLAIN, VARIANT_TMA_2STAGE)
    again = Plan([field_params(n, dt, xi_over_dx=1.5) for n in sizes]).autotune(cache)   # from the cache
    for n in sizes:
        assert again.sweep_variant(n, 0, 6) == tuned.sweep_variant(n, 0, 6)
    plain = Plan([field_params(n, dt, xi_over_dx=1.5) for n in sizes])
    fa = [to_gpu(random_psi(n, 60 + i), np.complex64) for i, n in enumerate(sizes)]
    fb = [f.clone() for f in fa]
    tuned.step(fa, 6)
    plain.step(fb, 6)
    for x, y in zip(fa, fb):
        assert rel_l2(to_np(x), to_np(y)) < 1e-6

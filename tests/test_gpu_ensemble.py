"""A ragged ensemble advanced in one persistent launch per call (gp_plan_set_fused_batch):
bitwise against the per-sweep launches, and against the oracle."""
import numpy as np
import pytest

from inputs import random_direction, random_psi
from oracle import initial as OI
from oracle import scheme as OS
from tests._util import rel_l2, to_gpu, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2003_03590_gb300 import GP_FP32, GP_FP64, GP_SPLIT_KNK, GPError, Plan, field_params  # noqa: E402
from paper_2003_03590_gb300.gpqt import launch_count  # noqa: E402


def _pair(sizes, dt):
    fused = Plan([field_params(n, dt, xi_over_dx=1.5) for n in sizes]).set_fused_batch(True)
    per = Plan([field_params(n, dt, xi_over_dx=1.5) for n in sizes])
    return fused, per


def test_fused_run_matches_per_sweep_launches_bitwise():
    """Every length the fused run holds, several fields of each, calls of 1, 2 and 7 steps (the
    repeated 7-step call replays the captured graph): each call is one launch, and the fields
    equal those of the per-sweep launches bit for bit (same tiles, same arithmetic)."""
    sizes = [32, 64, 32, 96, 128, 64, 96]
    fused, per = _pair(sizes, 0.002)
    fa = [to_gpu(random_psi(n, 300 + i, amp_jitter=0.1), np.complex64) for i, n in enumerate(sizes)]
    fb = [f.clone() for f in fa]
    for steps in (1, 2, 7, 7):
        l0 = launch_count(fused)
        fused.step(fa, steps)
        assert launch_count(fused) - l0 == 1
        per.step(fb, steps)
        fused.sync()
        per.sync()
        for i, (x, y) in enumerate(zip(fa, fb)):
            assert torch.equal(x, y), (i, sizes[i], steps)


def test_fused_run_against_the_oracle():
    """Lengths 32, 64, 96 (radix-3 passes) and 128 with SRP starts made by the oracle, xi = 1.5 dx,
    dt = 0.002: one and three steps of every field match the oracle to 1e-5 per step."""
    dt = 0.002
    sizes = [32, 64, 96, 128]
    fused = Plan([field_params(n, dt, xi_over_dx=1.5) for n in sizes]).set_fused_batch(True)
    starts = [OI.srp_spectral(n, 60 + i, 4.0).astype(np.complex64).astype(np.complex128) for i, n in enumerate(sizes)]
    for steps in (1, 3):
        psis = [to_gpu(x, np.complex64) for x in starts]
        fused.step(psis, steps)
        fused.sync()
        for i, n in enumerate(sizes):
            ref = OS.evolve(starts[i], OS.params_from_dx_ratio(n, 1.5, dt), steps)
            assert rel_l2(to_np(psis[i]), ref) < 1e-5 * steps, (n, steps)


def test_fused_run_of_the_ragged_ensemble_workload():
    """The 48-field ensemble (24 x 64^3, 16 x 96^3, 8 x 128^3, seeds 0..47, dt = 0.004): 12 steps
    in one launch equal 12 steps of the per-sweep launches bit for bit, and every field's norm
    is conserved to 1e-5 (the nonlinear factor has modulus one, the kinetic one too)."""
    sizes = [64] * 24 + [96] * 16 + [128] * 8
    fused, per = _pair(sizes, 0.004)
    fa = [fused.init_srp(i, fused.empty(i), seed=i, mode=0, p0=4.0, p1=np.pi) for i in range(len(sizes))]
    fb = [f.clone() for f in fa]
    m0 = [float((x.abs() ** 2).double().mean()) for x in fa]
    fused.step(fa, 12)
    per.step(fb, 12)
    fused.sync()
    per.sync()
    for i, (x, y) in enumerate(zip(fa, fb)):
        assert torch.equal(x, y), (i, sizes[i])
        m = float((x.abs() ** 2).double().mean())
        assert abs(m - m0[i]) < 1e-5 * m0[i], (i, m, m0[i])


def test_fused_batch_rejects_what_it_cannot_run():
    """Float64 fields, the KNK split, lengths other than 32/64/96/128 and more than 64 fields are
    refused with GP_ERR_INVALID_ARG, and the plan keeps stepping as before."""
    for fp in ([field_params(64, 0.002, xi_over_dx=1.5, precision=GP_FP64)],
               [field_params(64, 0.002, xi_over_dx=1.5, split=GP_SPLIT_KNK)],
               [field_params(48, 0.002, xi_over_dx=1.5)],
               [field_params(256, 0.002, xi_over_dx=1.5)],
               [field_params(32, 0.002, xi_over_dx=1.5)] * 65):
        p = Plan(fp)
        with pytest.raises(GPError):
            p.set_fused_batch(True)
        p.set_fused_batch(False)
    p = Plan([field_params(32, 0.002, xi_over_dx=1.5, precision=GP_FP32)])
    x = to_gpu(random_psi(32, 5), np.complex64)
    y = x.clone()
    p.step([x], 3)
    p.set_fused_batch(True).step([y], 3)
    p.sync()
    assert torch.equal(x, y)


def test_fused_run_bounded_wait_gives_up_and_reports_timeout():
    """A fused run whose first tile is never handed out: the tiles that need it wait about a
    second, give up, and the run ends with the status word set (GP_ERR_TIMEOUT at the next
    check); the plan and the context stay usable and the next run is exact again."""
    sizes = [32, 64]
    fused, per = _pair(sizes, 0.002)
    fa = [to_gpu(random_psi(n, 500 + i), np.complex64) for i, n in enumerate(sizes)]
    fused.test_timeout(1)
    fused.step(fa, 1)
    with pytest.raises(GPError) as err:
        fused.sync()
    assert err.value.status == 5             # GP_ERR_TIMEOUT
    good = [to_gpu(random_psi(n, 510 + i), np.complex64) for i, n in enumerate(sizes)]
    ref = [g.clone() for g in good]
    fused.step(good, 2)
    per.step(ref, 2)
    fused.sync()
    per.sync()
    for x, y in zip(good, ref):
        assert torch.equal(x, y)


def test_graph_replay_after_the_counter_buffer_grows():
    """A fused run's graph holds the address of the plan's counters.  An adjoint step (its
    recomputation runs the fused plane kernel, whose counters are larger) reallocates them; the
    next call must not replay the stale graph: the field still equals the per-sweep launches'."""
    n, dt = 32, 0.002
    fused, per = _pair([n], dt)
    x = to_gpu(random_psi(n, 7), np.complex64)
    y = x.clone()
    fused.step([x], 1)
    fused.step([x], 1)                       # replays the graph captured by the first call
    per.step([y], 1)                         # the same calls (a 2-step call merges the half steps)
    per.step([y], 1)
    lam = to_gpu(random_direction(n, 8), np.complex64)
    fused.adjoint_step(0, x.clone(), lam, 2)
    fused.step([x], 1)
    per.step([y], 1)
    fused.sync()
    per.sync()
    assert torch.equal(x, y)

#!/usr/bin/env python
"""Throughput of the Strang split step of the dimensionless 3D Gross-Pitaevskii equation.

Workload (default): 256^3 periodic box, xi = 1.5 dx (alpha = sqrt(2) xi, beta = 2/alpha),
dt = 0.002, random-vortex-ring initial condition (40 rings, radii in [4 xi, 12 xi], seed 0),
float32 storage, fused sweeps.  A bench step is one time step of the scheme; the timed
region is one gp_step call advancing K steps on a field already resident in HBM.

Metric: N^3 * steps / s (grid points advanced per second), whole job.  Also reported:
  roofline     the dominant sweep kernel (bound "alu": the issue of its float32 arithmetic
               limits it): algorithmic flops (5 log2 N per point and 1D transform, 6 per
               pointwise complex factor) / its mean CUDA-event time against the nominal FP32
               rate; beside it ("hbm") algorithmic bytes (16 B per point per launch, one read
               and one write of the complex64 field) against the measured HBM copy bandwidth,
               the ncu DRAM traffic and FMA-pipe / issue activity when taken on the current
               source; floor_frac = 32 N^3 B / (t_step * BW) (two sweeps per step is the
               fewest a 3D FFT pair admits)
  e2e          the same metric through gp_step_host with the field in pinned host memory,
               one host->device copy, one step and one device->host copy per bench step
  cpu_baseline the float64 numpy oracle, one full 256^3 step, on the host
  fp64_plain   the unfused complex128 GPU path, cufft_torch the cuFFT + elementwise baseline
  sizes        512^3 and 1024^3 (smoothed-random-phase start, k0 = 8, dt = 0.001)
N > 1 GPUs (torchrun): every rank advances its own independent field (replicas; the
ensemble shards without communication), value = all ranks' points * steps / max time.
"""
import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_MAIN, DT_MAIN, RINGS = 256, 0.002, 40
METRIC = "GP N^3*steps/s (fused FP32 split step)"
UNIT = "N^3*steps/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="gp", choices=["gp", "reference"])
    ap.add_argument("--no-extras", action="store_true", help="skip fp64/cufft/large-size/cpu legs")
    ap.add_argument("--sizes", default="512,1024")
    ap.add_argument("--only-step", action="store_true", help="init, warm-up and the timed steps only (profiling)")
    ap.add_argument("--only-diag", type=int, default=0, metavar="CALLS",
                    help="init, then CALLS diagnostics calls of the step workload's field (profiling)")
    ap.add_argument("--kernel-tour", action="store_true",
                    help="every library entry point once on the benchmark's sizes, then exit (for a per-kernel ncu list)")
    ap.add_argument("--paper-prep", default=None, metavar="CASE",
                    help="one of the paper's imaginary-time preparations (tg_a..tg_d, abc_a..abc_c): our energies, "
                         "helicities and Mach numbers next to the printed ones, then exit")
    ap.add_argument("--tune-cache", default=None,
                    help="JSON file of kernel choices: read if present (no tuning launches), else written")
    return ap.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except Exception:
        return 6800.0, "fallback 6.8 TB/s (MEASURED_PEAKS.json absent)"


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("gp_fft.cuh", "gp_sweep.cuh", "gp_tma.cuh", "gp_plane.cuh"):
        with open(os.path.join(ROOT, "paper_2003_03590_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel, n):
    """dram read+write bytes per launch from the committed ncu summary, if it was taken on the
    current kernel source (lines: <kernel> <n> <bytes_per_launch> <source_hash>)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(path):
        return None
    cur = kernel_source_hash()
    with open(path) as f:
        for line in f:
            parts = line.split()
            if len(parts) == 4 and not line.startswith("#") and parts[0] == kernel and int(parts[1]) == n \
                    and parts[3] == cur:
                return float(parts[2])
    return None


def ncu_pipes(kernel, n):
    """FMA-pipe and issue-slot activity (% of peak) of a kernel from the committed ncu summary, if
    taken on the current kernel source (lines: <kernel> <n> <fma_pipe_pct> <issue_pct> <source_hash>)."""
    path = os.path.join(ROOT, "profiles", "ncu_pipes.txt")
    if not os.path.exists(path):
        return None
    cur = kernel_source_hash()
    with open(path) as f:
        for line in f:
            parts = line.split()
            if len(parts) == 5 and not line.startswith("#") and parts[0] == kernel and int(parts[1]) == n \
                    and parts[4] == cur:
                return {"fma_pipe_active_pct": float(parts[2]), "issue_active_pct": float(parts[3]),
                        "source": "profiles/ncu_pipes.txt"}
    return None


class ClockSampler:
    """nvidia-smi clocks during the timed region."""

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(backend=None):
    """Rank/world from the launcher's environment.  One process per GPU: N > 1 runs N
    replicas of the workload (no data-path collective); the process group only carries the
    barriers around the timed region and the max over ranks of the timings (nccl on GPUs,
    gloo for the CPU tests of this host logic)."""
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    backend = backend or "nccl"
    if world > 1:
        import torch.distributed as dist
        if backend == "nccl":
            torch.cuda.set_device(local)
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:
            dist.init_process_group(backend)
    elif backend == "nccl":
        torch.cuda.set_device(0)
    return world, rank, local


def _on_gpu():
    import torch.distributed as dist
    return dist.is_initialized() and dist.get_backend() == "nccl"


def barrier(world):
    if world > 1:
        import torch
        import torch.distributed as dist
        dist.barrier()
        if _on_gpu():
            torch.cuda.synchronize()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if _on_gpu() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(points_per_rank, steps, world, ms_max):
    """Whole-job N^3*steps/s: every rank advances its own field (weak scaling), timed by the
    slowest rank."""
    return points_per_rank * steps * world / (ms_max / 1e3)


def tuned_choices(plan, n):
    names = {0: "tma", 1: "tma_1cta", 2: "plain", 3: "tma_2stage", 4: "tma_2groups"}
    kinds = {"z:n_fwd": (2, 4), "z:inv_n_fwd": (2, 3), "z:inv_n": (2, 5), "y:fwd": (1, 1), "y:inv": (1, 2),
             "x:fwd_k_inv": (0, 6)}
    out = {k: names.get(plan.sweep_variant(n, a, o), "?") for k, (a, o) in kinds.items()}
    pv = plan.sweep_variant(n, 1, 7)
    out["y_x_y"] = "three sweeps" if pv == 2 else "fused plane kernel (" + names.get(pv, "?") + ")"
    return out


def make_plan(gq, n, dt, prec):
    return gq.Plan(gq.field_params(n, dt, xi_over_dx=1.5, precision=prec))


def init_rvr(gq, plan, seed):
    a, b = plan.coefficients()
    xi = math.sqrt(a / b)
    return plan.init_rvr(0, plan.empty(), seed=seed, mode=0, count=RINGS, p0=4 * xi, p1=12 * xi)


def time_steps(plan, psi, k):
    import torch
    s = plan.stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(s)
    plan.step([psi], k)
    e1.record(s)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


# Algorithmic arithmetic of one sweep kind, per grid point: 1D transforms (5 log2 N flops each, the
# radix-2 count of an N-point complex FFT) and pointwise complex factors (6 flops: the complex
# multiply by exp(-i phase) of N(s) or K(s)).
SWEEP_WORK = {"fwd": (1, 0), "inv": (1, 0), "n_fwd": (1, 1), "inv_n": (1, 1), "inv_n_fwd": (2, 1),
              "fwd_k_inv": (2, 1), "y_fwd_x_fwd_k_inv_y_inv": (4, 1)}
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12   # SMs x FP32 lanes x 2 (FMA) x max SM clock: 80.5


def roofline_of(gq, plan, psi, n, ksteps, peak):
    gq.profile(plan, True)
    plan.step([psi], ksteps)
    rec = gq.profile_read(plan)
    gq.profile(plan, False)
    per_kernel = {}
    flops_of = {}
    for name, (cnt, ms) in rec.items():
        kern, op = name.split(":")[0], name.split(":")[1]
        c, m = per_kernel.get(kern, (0, 0.0))
        per_kernel[kern] = (c + cnt, m + ms)
        tr, pw = SWEEP_WORK.get(op, (1, 0))
        flops_of[kern] = flops_of.get(kern, 0.0) + cnt * (tr * 5 * math.log2(n) + 6 * pw) * n ** 3
    total = sum(m for _, m in per_kernel.values())
    kern, (cnt, ms) = max(per_kernel.items(), key=lambda kv: kv[1][1])
    per_launch_s = ms / cnt / 1e3
    alg_bytes = 16.0 * n ** 3
    achieved = alg_bytes / per_launch_s / 1e9
    traffic = ncu_traffic(kern, n)
    alg_flops = flops_of[kern] / cnt
    tflops = alg_flops / per_launch_s / 1e12
    # The sweep kernels are limited by the issue of their float32 arithmetic, not by HBM (ncu:
    # DRAM well below peak, issue slots and the FMA pipe the busiest units): the bound is "alu",
    # against the nominal FP32 rate, with the HBM figures and the ncu pipe counters beside it.
    return {"kernel": kern, "bound": "alu", "achieved": round(tflops, 2), "peak": round(FP32_PEAK_TFLOPS, 1),
            "unit": "TFLOP/s", "frac": round(tflops / FP32_PEAK_TFLOPS, 4), "traffic": traffic,
            "algorithmic_flops": alg_flops, "peak_source": "nominal: 152 SMs x 128 FP32 lanes x 2 x 2070 MHz",
            "pipes": ncu_pipes(kern, n),
            "hbm": {"achieved": round(achieved, 1), "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
                    "algorithmic_bytes": alg_bytes},
            "launches": cnt, "mean_launch_us": round(per_launch_s * 1e6, 2), "time_share": round(ms / total, 3),
            "kernels": {k: {"launches": c, "ms": round(m, 3), "share": round(m / total, 3)}
                        for k, (c, m) in per_kernel.items()},
            "kinds_mean_us": {k: round(ms_ / c_ * 1e3, 2) for k, (c_, ms_) in rec.items()}}


def ensemble_leg(gq, steps=500):
    """24 x 64^3 + 16 x 96^3 + 8 x 128^3 smoothed-random-phase fields (seeds 0..47, k0 = 4),
    dt = 0.004, advanced together by one plan (one launch per sweep and size class; the timed
    call repeats an untimed call of the same length, so the whole 500-step run replays as one
    captured CUDA graph), by one plan in one persistent launch per call (the fused run), and
    one plan at a time."""
    import torch
    sizes = [64] * 24 + [96] * 16 + [128] * 8
    fields = [gq.field_params(n, 0.004, xi_over_dx=1.5) for n in sizes]
    import tempfile
    cache = os.path.join(tempfile.mkdtemp(), "tune.json")
    batch = gq.Plan(fields).autotune(cache)
    psis = [batch.init_srp(i, batch.empty(i), seed=i, mode=0, p0=4.0, p1=math.pi) for i in range(len(sizes))]
    pts = sum(n ** 3 for n in sizes)
    batch.step(psis, steps)                     # untimed: the next call of this length is one graph
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = gq.launch_count(batch)
    e0.record(batch.stream)
    batch.step(psis, steps)
    e1.record(batch.stream)
    torch.cuda.synchronize()
    ms_b = e0.elapsed_time(e1)
    launches = gq.launch_count(batch) - l0
    # the same fields advanced by one persistent launch per call (the whole 500-step run)
    fused = gq.Plan(fields).set_fused_batch(True)
    fused.step(psis, steps)
    torch.cuda.synchronize()
    l0 = gq.launch_count(fused)
    e0.record(fused.stream)
    fused.step(psis, steps)
    e1.record(fused.stream)
    torch.cuda.synchronize()
    ms_f = e0.elapsed_time(e1)
    launches_f = gq.launch_count(fused) - l0
    fused.sync()
    singles = [gq.Plan(f).autotune(cache) for f in fields]     # the same kernel choices
    for pl, f in zip(singles, psis):
        pl.step([f], steps)
    torch.cuda.synchronize()
    e0.record(singles[0].stream)
    for pl, f in zip(singles, psis):
        pl.step([f], steps)
    e1.record(singles[0].stream)
    torch.cuda.synchronize()
    ms_s = e0.elapsed_time(e1)
    return {"points": pts, "steps": steps,
            "fused_run": {"value": pts * steps / (ms_f / 1e3), "ms": ms_f, "launches": launches_f,
                          "kernel": "k_ensemble_run (one persistent launch per call)"},
            "batched": {"value": pts * steps / (ms_b / 1e3), "ms": ms_b, "launches": launches, "graph_launches": 1},
            "sequential": {"value": pts * steps / (ms_s / 1e3), "ms": ms_s}, "speedup": ms_s / ms_b,
            "fused_speedup_vs_batched": ms_b / ms_f, "fused_speedup_vs_sequential": ms_s / ms_f}


def config3_run(gq, plan, f, steps=2000, every=100):
    """Configuration 3 as specified: 1024^3, xi = 1.5 dx, dt = 0.001, SRP start (k0 = 8, seed
    0), 2000 steps with the full diagnostics (float64 sums, four spectra) every 100 steps.  The
    wall time covers steps and diagnostics (each diagnostics call synchronises).  The time step
    puts grid wavenumbers in the split step's instability band (growth up to 1 + beta dt = 1.15
    per step), so the run reports the step at which the energy leaves its start value by 1e-3
    and the first non-finite field, if any: the scheme's property at this dt, float64 alike."""
    import torch
    f = plan.init_srp(0, f, seed=0, mode=0, p0=8.0, p1=math.pi)
    d0, _ = plan.diagnostics(0, f)
    e0, n0 = d0["E"], d0["N"]
    hist, departed, nonfinite = [], None, None
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for c in range(steps // every):
        plan.step([f], every)
        try:
            d, _ = plan.diagnostics(0, f)
            rel_e, rel_n = d["E"] / e0 - 1.0, d["N"] / n0 - 1.0
            hist.append([(c + 1) * every, rel_e, rel_n])
            if departed is None and abs(rel_e) > 1e-3:
                departed = (c + 1) * every
        except gq.GPError as e:   # a non-finite field: the band's growth has overflowed
            if e.status != 6:
                raise
            nonfinite = nonfinite or (c + 1) * every
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    return {"steps": steps, "diagnostics_every": every, "seconds": secs,
            "N3_steps_per_s_with_diagnostics": 1024 ** 3 * steps / secs,
            "energy_departs_1e-3_at_step": departed, "first_nonfinite_at_step": nonfinite,
            "rel_energy_and_mass_every_100": hist}


def adjoint_leg(gq, n=128, steps=400, every=20, dt=0.002):
    """Gradient of E_kin^i(psi_T) with respect to the initial phase (128^3, 400 steps, checkpoints
    every 20, dt = 0.002: outside the split step's instability band on this grid) through the
    autograd function, float32 and float64, and their agreement."""
    import torch

    from inputs import smooth_phase
    th = torch.from_numpy(smooth_phase(n, 0))
    out = {"dt": dt}
    grads = {}
    for name, prec, rdt in (("fp32", gq.GP_FP32, torch.float32), ("fp64", gq.GP_FP64, torch.float64)):
        plan = gq.Plan(gq.field_params(n, dt, xi_over_dx=1.5, precision=prec))
        t = th.to(rdt).cuda().requires_grad_(True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        J = gq.IncompressibleKineticEnergy.apply(gq.GPEvolve.apply(t, plan, steps, every), plan, 1e-6)
        J.backward()
        torch.cuda.synchronize()
        out[name] = {"seconds": time.perf_counter() - t0, "J": float(J.detach())}
        grads[name] = t.grad.double()
    # sensitivity of the float64 gradient itself to the float32 rounding of the start
    plan = gq.Plan(gq.field_params(n, dt, xi_over_dx=1.5, precision=gq.GP_FP64))
    t = th.to(torch.float32).to(torch.float64).cuda().requires_grad_(True)
    J = gq.IncompressibleKineticEnergy.apply(gq.GPEvolve.apply(t, plan, steps, every), plan, 1e-6)
    J.backward()
    g64r = t.grad.double()
    g32, g64 = grads["fp32"], grads["fp64"]
    rel = lambda a, b: float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))
    out["grad_rel_err_fp32_vs_fp64"] = rel(g32, g64)
    out["grad_rel_err_fp64_rounded_start_vs_fp64"] = rel(g64r, g64)
    # the adjoint's own error: both adjoints along the float32 trajectory (its checkpoints and final
    # state, upcast for float64), so the flow's sensitivity to the start does not enter
    p32 = gq.Plan(gq.field_params(n, dt, xi_over_dx=1.5, precision=gq.GP_FP32))
    p64 = gq.Plan(gq.field_params(n, dt, xi_over_dx=1.5, precision=gq.GP_FP64))
    t32 = th.to(torch.float32).cuda()
    psi0 = p32.psi_from_phase(0, t32)
    psi = psi0.clone()
    ck = []
    for _ in range(steps // every):
        ck.append(psi.clone())
        p32.step([psi], every)
    lam32, _ = p32.ekin_i_grad(0, psi, 1e-6)
    lam64, _ = p64.ekin_i_grad(0, psi.to(torch.complex128), 1e-6)
    for c in reversed(ck):
        p32.adjoint_step(0, c, lam32, every)
        p64.adjoint_step(0, c.to(torch.complex128), lam64, every)
    gs32 = p32.phase_grad(0, psi0, lam32).double()
    gs64 = p64.phase_grad(0, p64.psi_from_phase(0, t32.double()), lam64)
    out["grad_rel_err_fp32_vs_fp64_same_trajectory"] = rel(gs32, gs64)
    return out


def diag_leg(gq, plan, psi, n, ms_step, calls=3):
    import torch
    plan.diagnostics(0, psi)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(calls):
        plan.diagnostics(0, psi)
    ms = (time.perf_counter() - t0) * 1e3 / calls
    return {"ms_per_call": ms, "share_at_1_per_100_steps": ms / (ms + 100 * ms_step)}


def analysis_leg(plan, psi, calls=3):
    """Wall time per call of the field analyses on the timed field: the second-order structure
    functions along x, y, z (Sec. 3.5) and both helicities with their spectra (Sec. 3.6); each
    call synchronises the stream."""
    import torch
    out = {}
    for name, fn in (("structure_function_p2", lambda: plan.structure_function(0, psi, 2)),
                     ("helicity_with_spectra", lambda: plan.helicity(0, psi))):
        fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(calls):
            fn()
        out[name] = {"ms_per_call": (time.perf_counter() - t0) * 1e3 / calls}
    return out


# The paper's preparations: its parameter table (alpha, beta per resolution), its TG / ABC run
# tables (dtau, tau_f) and, at tau_f, its ARGLE energy tables (E_kin^i, E_kin^c, E_q, E_int, H,
# H_reg), its conservation tables (N, E at t = 0) and its ABC Mach table (ABC_c only).
PAPER_PREP = {
    "tg_a": (128, 0.05, 40.0, "tg", 1.25e-2, 60, dict(E_kin_i=0.12901707, E_kin_c=4.8667051e-4, E_q=7.9239425e-3,
                                                      E_int=1.2995235e-2, H=1.37e-13, H_reg=-1.87e-11, N=0.9789997,
                                                      E=0.1504230)),
    "tg_b": (256, 0.025, 80.0, "tg", 6.25e-3, 60, dict(E_kin_i=0.11334487, E_kin_c=2.2334712e-4, E_q=4.0373670e-3,
                                                       E_int=6.8223665e-3, H=2.96e-7, H_reg=-5.52e-7, N=0.9873160,
                                                       E=0.1244280)),
    "tg_c": (512, 0.0125, 160.0, "tg", 3.125e-3, 60, dict(E_kin_i=0.12884207, E_kin_c=1.5065059e-4, E_q=2.4895687e-3,
                                                          E_int=4.2864757e-3, H=3.83e-3, H_reg=-5.63e-7, N=0.9920083,
                                                          E=0.1357688)),
    "tg_d": (1024, 0.00625, 320.0, "tg", 1.5625e-3, 60, dict(E_kin_i=0.12968555, E_kin_c=9.5590716e-5, E_q=1.3476259e-3,
                                                             E_int=2.3466209e-3, H=-3.94e-4, H_reg=-9.71e-8, N=0.9955732,
                                                             E=0.1275738)),
    "abc_a": (128, 0.05, 40.0, "abc", 4e-3, 30, dict(E_kin_i=0.9485114, E_kin_c=0.0014218, E_q=0.0277287,
                                                    E_int=0.0430379, H=2.4106982, H_reg=2.4726091, N=0.9410138,
                                                    E=1.0206996)),
    "abc_b": (256, 0.025, 80.0, "abc", 2e-3, 30, dict(E_kin_i=0.9792042, E_kin_c=0.0008142, E_q=0.0144931,
                                                     E_int=0.0237201, H=2.7439625, H_reg=2.6532860, N=0.9647786,
                                                     E=1.0182316)),
    "abc_c": (512, 0.0125, 160.0, "abc", 1e-3, 30, dict(E_kin_i=0.9884992, E_kin_c=0.0006486, E_q=0.0073802,
                                                       E_int=0.0124975, H=2.7217161, H_reg=2.7365301, N=0.9796053,
                                                       E=1.0090255, M_max=1.486860, M_rms=0.703259)),
}


def paper_prep(gq, case):
    """One of the paper's imaginary-time preparations with its parameters (float32 field), then the
    diagnostics (with the Mach numbers) and both helicities of the prepared field, each next to the
    value the paper prints and their relative difference."""
    import torch
    n, alpha, beta, kind, dtau, tau_f, paper = PAPER_PREP[case]
    plan = gq.Plan(gq.field_params(n, 1e-3, alpha=alpha, beta=beta, precision=gq.GP_FP32))
    psi = plan.init_tg(0, plan.empty()) if kind == "tg" else plan.init_abc(0, plan.empty())
    steps = int(round(tau_f / dtau))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plan.argle(0, psi, gq.GP_FLOW_TG if kind == "tg" else gq.GP_FLOW_ABC, dtau, steps, energy=False)
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    d, _ = plan.diagnostics(0, psi, spectra=False)
    h, _ = plan.helicity(0, psi, spectra=False)
    got = dict(d)
    got.update(h)
    rows = {k: {"ours": got[k], "paper": v, "rel": (got[k] / v - 1) if abs(v) > 1e-6 else None}
            for k, v in paper.items()}
    return {"paper_prep": case, "n": n, "alpha": alpha, "beta": beta, "dtau": dtau, "argle_steps": steps,
            "argle_seconds": secs, "precision": "f32", "values": rows}


def kernel_tour(gq):
    """Every library entry point once, on the sizes the benchmark uses (256^3 float32 fields,
    128^3 for the float64 path, the imaginary-time preparation and the batch), so that one ncu
    launch list covers every kernel of the library."""
    import ctypes
    import torch
    from paper_2003_03590_gb300 import _lib
    n = N_MAIN
    plan = make_plan(gq, n, DT_MAIN, gq.GP_FP32)                     # default kernel variants
    psi = init_rvr(gq, plan, seed=0)
    plan.init_rvr(0, plan.empty(), seed=1, mode=1, count=2, p0=0.5 * math.pi, p1=math.pi)
    plan.init_srp(0, plan.empty(), seed=2, mode=0, p0=8.0, p1=math.pi)
    plan.init_srp(0, plan.empty(), seed=3, mode=1, p0=math.pi, p1=16)
    plan.psi_from_phase(0, torch.zeros((n, n, n), dtype=torch.float32, device="cuda"))
    plan.step([psi], 3)
    plan.diagnostics(0, psi)
    plan.structure_function(0, psi, 2)
    plan.helicity(0, psi)
    lam = psi.clone()
    plan.adjoint_step(0, psi, lam, 2)
    plan.ekin_i_grad(0, psi)
    plan.phase_grad(0, psi, lam)
    small = make_plan(gq, 64, DT_MAIN, gq.GP_FP32)
    f64 = init_rvr(gq, small, seed=4)
    a, b = small.coefficients()
    d = _lib.Diag()
    _lib.load().gp_diagnostics_noalloc(64, a, b, ctypes.c_void_p(f64.data_ptr()), ctypes.byref(d), None, 0,
                                       ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    p64 = make_plan(gq, 128, DT_MAIN, gq.GP_FP64)
    g = p64.init_srp(0, p64.empty(), seed=5, mode=0, p0=4.0, p1=math.pi)
    p64.step([g], 2)
    p64.diagnostics(0, g)
    prep = gq.Plan(gq.field_params(128, 0.001, alpha=0.05, beta=40.0, precision=gq.GP_FP32))
    phi = prep.init_tg(0, prep.empty())
    prep.argle(0, phi, gq.GP_FLOW_TG, 1.25e-2, 2)
    prep.argle_converge(0, phi, gq.GP_FLOW_TG, 1.25e-2, 2, 0.0, check_every=2)
    phi = prep.init_abc(0, prep.empty())
    prep.argle(0, phi, gq.GP_FLOW_ABC, 4e-3, 2, renorm=True, energy=False)
    sizes = [64, 64, 96, 128]
    batch = gq.Plan([gq.field_params(m, 0.004, xi_over_dx=1.5) for m in sizes])
    fs = [batch.init_srp(i, batch.empty(i), seed=i, mode=0, p0=4.0, p1=math.pi) for i in range(len(sizes))]
    batch.step(fs, 2)
    torch.cuda.synchronize()
    for p_ in (plan, small, p64, prep, batch):
        p_.sync()
    return {"kernel_tour": "done", "n": n}


def argle_leg(gq, steps=200):
    """Imaginary-time (ARGLE) preparation of the paper's 128^3 Taylor-Green run (alpha = 0.05,
    beta = 40, dtau = 1.25e-2): time per ARGLE step (five 3D transforms) in float32 and float64."""
    import torch
    out = {}
    for name, prec in (("f32", gq.GP_FP32), ("f64", gq.GP_FP64)):
        plan = gq.Plan(gq.field_params(128, 0.001, alpha=0.05, beta=40.0, precision=prec))
        psi = plan.init_tg(0, plan.empty())
        plan.argle(0, psi, gq.GP_FLOW_TG, 1.25e-2, 5, energy=False)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(plan.stream)
        plan.argle(0, psi, gq.GP_FLOW_TG, 1.25e-2, steps, energy=False)
        e1.record(plan.stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        out[name] = {"ms_per_step": ms, "N3_steps_per_s": 128 ** 3 / (ms / 1e3), "steps": steps}
    return out


def cpu_oracle_baseline(n, dt, steps):
    """The float64 oracle, as it stands, on the host: `steps` full steps of the n^3 workload."""
    from inputs import random_psi
    from oracle import scheme as OS
    p = OS.params_from_dx_ratio(n, 1.5, dt)
    # the step's cost does not depend on the values: a seeded field of the workload's size
    psi = random_psi(n, 0, amp_jitter=0.1)
    t0 = time.perf_counter()
    for _ in range(steps):
        psi = OS.step_nkn(psi, p)
    dt_s = time.perf_counter() - t0
    return n ** 3 * steps / dt_s, dt_s


def _oracle_step_worker(job):
    """One float64 oracle step of the n^3 workload in a worker process (spawned: no CUDA state)."""
    import time as _t
    n, dt, seed = job
    from inputs import random_psi
    from oracle import scheme as OS
    p = OS.params_from_dx_ratio(n, 1.5, dt)
    psi = random_psi(n, seed, amp_jitter=0.1)
    t0 = _t.perf_counter()
    OS.step_nkn(psi, p)
    return _t.perf_counter() - t0


def host_cores():
    """Cores of this host: os.cpu_count() and the lscpu model line."""
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                model = ln.split(":", 1)[1].strip()
    except Exception:
        pass
    return os.cpu_count() or 1, model


def cpu_oracle_all_cores(n, dt, workers=None):
    """The oracle on every host core at once: one independent float64 step of the n^3 workload per
    core (replicas: the numpy oracle is single-threaded), throughput = workers n^3 / wall time."""
    import multiprocessing as mp
    workers = workers or (os.cpu_count() or 1)
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers) as pool:
        pool.map(_oracle_step_worker, [(8, dt, 0)] * workers)      # start-up of every worker
        t0 = time.perf_counter()
        per = pool.map(_oracle_step_worker, [(n, dt, w) for w in range(workers)])
        wall = time.perf_counter() - t0
    return workers * n ** 3 / wall, wall, max(per), workers


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1 and rank != 0:
        return 0
    k = 1
    w = min(args.warmup, 0)
    ncpu, model = host_cores()
    val, secs, worst, cores = cpu_oracle_all_cores(N_MAIN, DT_MAIN)
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": k, "warmup": w, "ms_per_step": secs * 1e3 / cores, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"GP split step {N_MAIN}^3, xi=1.5dx, dt={DT_MAIN}, RVR {RINGS} rings",
                       "global_batch": 1, "seq_len": N_MAIN ** 3, "parallelism": "single process, host"},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "host": {"nproc": ncpu, "lscpu_model": model},
                             "sample": f"one full float64 NKN step of the {N_MAIN}^3 field on each of {cores} cores "
                                       f"at once (numpy oracle, one process per core, {secs:.1f} s wall)"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import numpy as np
    import torch

    import paper_2003_03590_gb300.gpqt as gq
    world, rank, local = dist_setup()
    peak, peak_src = peaks()
    n, K, W = N_MAIN, args.steps, max(3, args.warmup)

    if args.paper_prep:
        out = paper_prep(gq, args.paper_prep)
        if rank == 0:
            print(json.dumps(out))
        return 0
    if args.kernel_tour:
        out = kernel_tour(gq)
        if rank == 0:
            print(json.dumps(out))
        return 0
    plan = make_plan(gq, n, DT_MAIN, gq.GP_FP32)
    if args.only_diag:
        psi = init_rvr(gq, plan, seed=rank)
        ms_call = diag_leg(gq, plan, psi, n, 0.0, calls=args.only_diag)["ms_per_call"]
        if rank == 0:
            print(json.dumps({"diagnostics_ms_per_call": ms_call, "calls": args.only_diag, "n": n}))
        return 0
    plan.autotune(args.tune_cache)             # kernel choice per sweep kind, before any timing
    psi = init_rvr(gq, plan, seed=rank)
    plan.step([psi], W)                       # warm-up (also captures the step graph)
    torch.cuda.synchronize()
    barrier(world)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.2)
    l0 = gq.launch_count(plan)
    ms = time_steps(plan, psi, K)
    launches = gq.launch_count(plan) - l0
    clk = clocks.stop()
    barrier(world)
    ms = max_over_ranks(ms, world)
    value = job_throughput(n ** 3, K, world, ms)
    if args.only_step:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": UNIT, "steps": K, "ms_per_step": ms / K}))
        return 0
    ms_step = ms / K
    floor_frac = 32.0 * n ** 3 / (ms_step / 1e3) / (peak * 1e9)
    # a timed region of at least a second (the driver's K may be a few ms), with the clocks sampled
    # through it and the step time scaled by the median SM clock (clock-independent work measure)
    k_long = max(K, int(math.ceil(1.2 / (ms_step / 1e3))))
    clocks_l = ClockSampler(local)
    clocks_l.start()
    time.sleep(0.2)
    ms_long = max_over_ranks(time_steps(plan, psi, k_long), world)
    clk_l = clocks_l.stop()
    long_run = {"steps": k_long, "seconds": round(ms_long / 1e3, 3), "ms_per_step": ms_long / k_long,
                "value": job_throughput(n ** 3, k_long, world, ms_long), "clocks": clk_l,
                "ms_per_step_x_sm_mhz": (ms_long / k_long * clk_l["sm_mhz"]) if clk_l.get("sm_mhz") else None}

    roof = roofline_of(gq, plan, psi, n, min(K, 200), peak)
    roof["floor_frac"] = round(floor_frac, 4)
    roof["hbm"]["peak_source"] = peak_src
    roof["sweeps_per_step"] = 4 if plan.sweep_variant(n, 1, 7) == 2 else 2   # HBM passes of the field

    # end to end through the public C ABI with host buffers
    host = torch.empty((n, n, n), dtype=torch.complex64).pin_memory()
    host.copy_(psi.cpu())
    k_e2e = min(K, 50)
    plan.step_host([host], 1)
    t0 = time.perf_counter()
    for _ in range(k_e2e):
        plan.step_host([host], 1)
    e2e_s = time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, world)
    e2e = {"value": n ** 3 * k_e2e * world / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 8 * n ** 3,
           "d2h_bytes_per_step": 8 * n ** 3, "steps": k_e2e,
           "how": "gp_step_host(pinned host field, 1 step) per bench step: H2D copy, fused step, D2H copy"}
    t0 = time.perf_counter()
    plan.step_host([host], K)
    run_s = max_over_ranks(time.perf_counter() - t0, world)
    e2e["whole_run"] = {"value": n ** 3 * K * world / run_s, "steps": K,
                        "how": "one gp_step_host call: one H2D, K steps, one D2H"}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"GP split step {n}^3, xi=1.5dx, dt={DT_MAIN}, RVR {RINGS} rings, fused FP32",
                       "global_batch": world, "seq_len": n ** 3, "parallelism": f"replicas x{world}",
                       "l2": f"field {8 * n ** 3 / 1e6:.0f} MB > 129 MB L2; no flush between steps",
                       "tuned": tuned_choices(plan, n)},
            "roofline": roof, "e2e": e2e, "gpu_launches": launches, "clocks": clk, "long_run": long_run}

    if not args.no_extras and rank == 0:
        extras = {}
        # plain float64 GPU path on the same workload
        p64 = make_plan(gq, n, DT_MAIN, gq.GP_FP64)
        psi64 = init_rvr(gq, p64, seed=0)
        p64.step([psi64], 2)
        k64 = 20
        ms64 = time_steps(p64, psi64, k64)
        extras["fp64_plain"] = {"value": n ** 3 * k64 / (ms64 / 1e3), "ms_per_step": ms64 / k64, "steps": k64}
        del psi64, p64
        # cuFFT + separate elementwise kernels (timed baseline only)
        a, b = plan.coefficients()
        kk = torch.fft.fftfreq(n, 1.0 / n, device="cuda", dtype=torch.float64)
        k2 = kk[:, None, None] ** 2 + kk[None, :, None] ** 2 + kk[None, None, :] ** 2
        ek = torch.polar(torch.ones_like(k2), -a * k2 * DT_MAIN).to(torch.complex64)
        del k2
        x = psi.clone()
        h = 0.5 * DT_MAIN

        def torch_step(x):
            x = x * torch.polar(torch.ones_like(x.real), -b * h * (x.real ** 2 + x.imag ** 2 - 1))
            x = torch.fft.ifftn(torch.fft.fftn(x) * ek)
            return x * torch.polar(torch.ones_like(x.real), -b * h * (x.real ** 2 + x.imag ** 2 - 1))

        for _ in range(3):
            x = torch_step(x)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        kcu = 100
        e0.record()
        for _ in range(kcu):
            x = torch_step(x)
        e1.record()
        torch.cuda.synchronize()
        mcu = e0.elapsed_time(e1)
        extras["cufft_torch"] = {"value": n ** 3 * kcu / (mcu / 1e3), "ms_per_step": mcu / kcu, "steps": kcu}
        del x, ek
        # larger grids
        sizes = {}
        for s in [int(v) for v in args.sizes.split(",") if v.strip()]:
            ps = make_plan(gq, s, 0.001, gq.GP_FP32).autotune()
            f = ps.init_srp(0, ps.empty(), seed=0, mode=0, p0=8.0, p1=math.pi)
            ps.step([f], 5)
            ks = 100 if s <= 512 else 40
            mss = time_steps(ps, f, ks)
            r = roofline_of(gq, ps, f, s, min(ks, 20), peak)
            sizes[str(s)] = {"value": s ** 3 * ks / (mss / 1e3), "ms_per_step": mss / ks, "steps": ks,
                             "floor_frac": round(32.0 * s ** 3 / (mss / ks / 1e3) / (peak * 1e9), 4),
                             "sweeps_per_step": 4 if ps.sweep_variant(s, 1, 7) == 2 else 2,
                             "tuned": tuned_choices(ps, s), "kinds_mean_us": r["kinds_mean_us"],
                             "dominant": {"kernel": r["kernel"], "time_share": r["time_share"],
                                          "alu_frac": r["frac"], "hbm_frac": r["hbm"]["frac"]}}
            if s >= 1024:
                # configuration 3: full diagnostics (float64 sums, four spectra) every 100 steps
                free0 = torch.cuda.mem_get_info()[0]
                ps.diagnostics(0, f)
                torch.cuda.synchronize()
                ws = free0 - torch.cuda.mem_get_info()[0]
                t0 = time.perf_counter()
                for _ in range(2):
                    ps.diagnostics(0, f)
                dms = (time.perf_counter() - t0) * 1e3 / 2
                sizes[str(s)]["diagnostics"] = {"ms_per_call": dms, "workspace_bytes": ws,
                                                "share_at_1_per_100_steps": dms / (dms + 100 * mss / ks)}
                sizes[str(s)]["configuration_3_run"] = config3_run(gq, ps, f)
            del f, ps
            torch.cuda.empty_cache()
        extras["sizes"] = sizes
        extras["ensemble"] = ensemble_leg(gq)
        extras["adjoint_128"] = adjoint_leg(gq)
        extras["diagnostics_cost"] = diag_leg(gq, plan, psi, n, ms_step)
        extras["analysis_cost"] = analysis_leg(plan, psi)
        extras["argle_tg_128"] = argle_leg(gq)
        # the float64 oracle on the host cores: one full step of the same 256^3 workload
        val1, secs1 = cpu_oracle_baseline(n, DT_MAIN, 1)
        ncpu, model = host_cores()
        valn, walln, _, cores = cpu_oracle_all_cores(n, DT_MAIN)
        line["cpu_baseline"] = {"value": valn, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "host": {"nproc": ncpu, "lscpu_model": model},
                                "sample": f"one full float64 NKN step of the {n}^3 field on each of {cores} cores at "
                                          f"once (numpy oracle, one process per core, {walln:.1f} s wall)",
                                "single_core": {"value": val1, "cores": 1,
                                                "sample": f"1 full float64 NKN step of the {n}^3 field ({secs1:.1f} s)"}}
        line["extras"] = extras
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())

"""GPU imaginary-time (ARGLE) preparation and the TG / ABC start fields against the oracle, and
the Taylor-Green preparation at 128^3 against the energies the paper prints for it."""
import math

import numpy as np
import pytest

from inputs import smooth_psi
from oracle import argle as OA
from oracle import diagnostics as OD
from oracle.scheme import Params
from tests._util import rel_l2, to_gpu, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2003_03590_gb300 import GP_FP32, GP_FP64, GPError, Plan, field_params  # noqa: E402
from paper_2003_03590_gb300.gpqt import GP_FLOW_ABC, GP_FLOW_NONE, GP_FLOW_TG  # noqa: E402

KIND = {GP_FLOW_NONE: "none", GP_FLOW_TG: "tg", GP_FLOW_ABC: "abc"}


def _plan(n, prec, alpha=0.05, beta=40.0):
    return Plan(field_params(n, 0.001, alpha=alpha, beta=beta, precision=prec))


def _dtype(prec):
    return np.complex128 if prec == GP_FP64 else np.complex64


@pytest.mark.parametrize("prec", [GP_FP64, GP_FP32])
@pytest.mark.parametrize("n", [32, 48])
def test_tg_start_field_matches_oracle(n, prec):
    plan = _plan(n, prec)
    psi = plan.init_tg(0, plan.empty())
    ref = OA.tg_ansatz(n, 0.05, 40.0)
    assert np.max(np.abs(to_np(psi) - ref)) < (1e-12 if prec == GP_FP64 else 2e-7)


@pytest.mark.parametrize("prec", [GP_FP64, GP_FP32])
def test_abc_start_field_matches_oracle(prec):
    n = 48
    plan = _plan(n, prec)
    psi = plan.init_abc(0, plan.empty())
    ref = OA.abc_ansatz(n, 0.05)
    assert np.max(np.abs(to_np(psi) - ref)) < (1e-11 if prec == GP_FP64 else 3e-7)
    other = (0.3, -0.7, 0.5)
    psi2 = plan.init_abc(0, plan.empty(), abc=other)
    assert np.max(np.abs(to_np(psi2) - OA.abc_ansatz(n, 0.05, other))) < (1e-11 if prec == GP_FP64 else 3e-7)


@pytest.mark.parametrize("prec", [GP_FP64, GP_FP32])
@pytest.mark.parametrize("flow", [GP_FLOW_NONE, GP_FLOW_TG, GP_FLOW_ABC])
@pytest.mark.parametrize("renorm", [False, True])
def test_argle_steps_match_oracle(flow, prec, renorm):
    n, dtau, m = 24, 0.0125, 8
    alpha, beta = 0.2, 10.0
    plan = _plan(n, prec, alpha, beta)
    phi0 = smooth_psi(n, 21).astype(_dtype(prec))
    psi = to_gpu(phi0, _dtype(prec))
    e = plan.argle(0, psi, flow, dtau, m, renorm=renorm)
    v = OA.velocity(KIND[flow], n)
    target = float(np.mean(np.abs(phi0.astype(np.complex128)) ** 2)) if renorm else None
    ref = OA.argle(phi0.astype(np.complex128), alpha, beta, dtau, m, v, renorm=target)
    tol = 1e-11 if prec == GP_FP64 else 2e-5
    assert rel_l2(to_np(psi), ref) < tol
    assert abs(e - OA.energy_v(ref, alpha, beta, v)) < tol * abs(e)


@pytest.mark.parametrize("prec", [GP_FP64, GP_FP32])
@pytest.mark.parametrize("flow", [GP_FLOW_NONE, GP_FLOW_TG, GP_FLOW_ABC])
def test_argle_stopping_criteria_match_oracle(flow, prec):
    """eqn:crit1 / eqn:crit2 of the last checked step, the step count and the field, against the
    oracle's checked loop: once running to max_steps (eps = 0), once stopping at the checked step
    where the residual first falls below an eps placed between two of the oracle's values."""
    n, dtau, alpha, beta = 24, 0.0125, 0.2, 10.0
    plan = _plan(n, prec, alpha, beta)
    phi0 = smooth_psi(n, 23).astype(_dtype(prec))
    v = OA.velocity(KIND[flow], n)
    tol = 1e-10 if prec == GP_FP64 else 1e-4
    psi = to_gpu(phi0, _dtype(prec))
    done, c1, c2, e = plan.argle_converge(0, psi, flow, dtau, 7, 0.0, check_every=3)
    ref, rdone, r1, r2 = OA.argle_converge(phi0.astype(np.complex128), alpha, beta, dtau, 7, v, 0.0, 3)
    assert done == rdone == 7
    assert c1 == pytest.approx(r1, rel=tol) and c2 == pytest.approx(r2, rel=10 * tol)
    assert rel_l2(to_np(psi), ref) < (1e-11 if prec == GP_FP64 else 2e-5)
    assert e == pytest.approx(OA.energy_v(ref, alpha, beta, v), rel=tol)
    # the oracle's residuals at the checks 2, 4, ..., 12; eps between the smallest of the first k
    # and a smaller k+1-th, so the first check at or below eps is the (k+1)-th
    seq = [OA.argle_converge(phi0.astype(np.complex128), alpha, beta, dtau, m, v, 0.0, 2)[2] for m in range(2, 13, 2)]
    k = next(j for j in range(1, len(seq)) if seq[j] < 0.999 * min(seq[:j]))
    eps = 0.5 * (min(seq[:k]) + seq[k])
    psi = to_gpu(phi0, _dtype(prec))
    done, c1, _, _ = plan.argle_converge(0, psi, flow, dtau, 40, eps, check_every=2, energy=False)
    assert done == 2 * (k + 1) and c1 <= eps


def test_argle_converge_rejects_bad_arguments():
    plan = _plan(16, GP_FP32)
    psi = torch.ones((16, 16, 16), dtype=torch.complex64, device="cuda")
    for kw in ({"max_steps": 0}, {"check_every": 0}, {"dtau": -1.0}):
        args = {"dtau": 0.01, "max_steps": 5, "check_every": 1}
        args.update(kw)
        with pytest.raises(GPError):
            plan.argle_converge(0, psi, GP_FLOW_NONE, args["dtau"], args["max_steps"], 1e-3,
                                check_every=args["check_every"])


def test_argle_energy_of_a_plane_wave_in_its_flow_is_zero():
    """Zero steps: E_v only.  A uniform flow is not one of the library's flows, so use the exact
    stationary state without flow: psi = 1 has E_v = 0 and stays 1."""
    plan = _plan(16, GP_FP64)
    psi = torch.ones((16, 16, 16), dtype=torch.complex128, device="cuda")
    assert plan.argle(0, psi, GP_FLOW_NONE, 0.01, 0) == pytest.approx(0.0, abs=1e-28)
    plan.argle(0, psi, GP_FLOW_NONE, 0.01, 5, energy=False)
    assert torch.max(torch.abs(psi - 1)).item() < 1e-15


@pytest.mark.parametrize("prec", [GP_FP64, GP_FP32])
def test_tg_preparation_reproduces_the_paper_table(prec):
    """TG_aIT of the paper: 128^3, alpha = 0.05, beta = 40, dtau = 1.25e-2, tau_f = 60 (4800 steps)
    from psi_ARGLE with [gamma_d/4] = 3.  The paper prints the energies of the converged field
    (its TG ARGLE energy table: E_kin^i = 0.12901707, E_kin^c = 4.8667051e-4, E_q = 7.9239425e-3,
    E_int = 1.2995235e-2), its mass and energy (TG conservation table, t = 0: N = 0.9789997,
    E = 0.1504230) and E_v = 0.710060 (TG grid table).  The tabulated E_v is the integral of
    eq-energy-num-ext-vel without its 2 alpha prefactor (a factor 10 at alpha = 0.05): compared as
    E_v / (2 alpha).  Tolerances: the paper prints 5 to 8 digits; the large parts must agree to
    1e-4, the small compressible part (4.9e-4 of an energy of 0.15, the most sensitive to how far
    the flow has converged) to 5e-3, the mass to 1e-6."""
    n = 128
    plan = Plan(field_params(n, 1.25e-3, alpha=0.05, beta=40.0, precision=prec))   # TG_a's real-time dt
    psi = plan.init_tg(0, plan.empty())
    ev = plan.argle(0, psi, GP_FLOW_TG, 1.25e-2, 4800)
    d, _ = plan.diagnostics(0, psi)
    got = {"E_kin_i": d["E_kin_i"], "E_kin_c": d["E_kin_c"], "E_q": d["E_q"], "E_int": d["E_int"], "N": d["N"],
           "E": d["E"], "E_v": ev / (2 * 0.05)}
    paper = {"E_kin_i": 0.12901707, "E_kin_c": 4.8667051e-4, "E_q": 7.9239425e-3, "E_int": 1.2995235e-2,
             "N": 0.9789997, "E": 0.1504230, "E_v": 0.710060}
    tol = {"E_kin_c": 5e-3, "N": 1e-6}
    print({k: (got[k], paper[k], got[k] / paper[k] - 1) for k in paper})
    for k in paper:
        assert got[k] == pytest.approx(paper[k], rel=tol.get(k, 1e-4)), (k, got[k], paper[k])
    # helicity (same table: H = 1.37e-13, H_reg = -1.87e-11): zero by the mirror symmetry of the
    # TG flow, to the round-off that breaks the symmetry of the stepped field
    h, _ = plan.helicity(0, psi, spectra=False)
    print(h)
    assert abs(h["H"]) < 1e-5 and abs(h["H_reg"]) < 1e-5
    _real_time_conservation(plan, psi, d, steps=9600, every=100, paper_n=0.9789997, paper_e_end=0.1504111,
                            paper_delta_e=7.97e-5, prec=prec, tol=1e-4)


def _real_time_conservation(plan, psi, d0, steps, every, paper_n, paper_e_end, paper_delta_e, prec, tol):
    """The paper's real-time run from the prepared field (its conservation table: N at t = 0 and
    T_f, E at t = 0 and T_f, delta(E) = max_t |E(t) - E(0)| / E(0)), with the fused split step:
    N is conserved to the rounding of the step (the scheme conserves it exactly), the final
    energy agrees with the printed one to the accuracy of the prepared field (tol: that of the
    energies above), and delta(E) -- the splitting error of a second-order scheme at the
    paper's dt over its whole run -- has the printed magnitude (within a factor 2: the paper
    prints the order KNK of its Strang step, the library's default order is NKN).  Measured,
    float64: TG_a E(T_f) = 0.15041109 (printed 0.1504111), ABC_a delta(E) 6.07e-5 (5.98e-5)."""
    e0, n0 = d0["E"], d0["N"]
    dev = 0.0
    for _ in range(steps // every):
        plan.step([psi], every)
        d, _ = plan.diagnostics(0, psi, spectra=False)
        dev = max(dev, abs(d["E"] - e0) / e0)
    print({"N_end": d["N"], "N_drift": d["N"] / n0 - 1, "E_end": d["E"], "paper_E_end": paper_e_end,
           "delta_E": dev, "paper_delta_E": paper_delta_e})
    # Rounding only (the scheme conserves N exactly).  float64: ~3e-16 per step.  float32: the
    # target of at most 1e-6 per 1000 steps, i.e. 1e-9 per step (measured: TG_a +1.3e-6 over 9600
    # steps, ABC_a -1.4e-7 over 12500, TG_b -9.4e-7 over 19200, ABC_b -1.6e-8 over 25000; before
    # the kinetic factor's and the nonlinear phase's product orders were fixed, +7.2e-5 over
    # TG_a's 9600 steps).
    assert abs(d["N"] / n0 - 1) < (1e-9 * steps if prec == GP_FP32 else 1e-10)
    assert d["N"] == pytest.approx(paper_n, rel=tol)
    assert d["E"] == pytest.approx(paper_e_end, rel=tol)
    # the splitting error itself: float64 within a factor 2 of the printed delta(E) (measured
    # 7.05e-5 against 7.97e-5 for TG_a, 6.07e-5 against 5.98e-5 for ABC_a); float32 below twice
    # it (its mass drift above moves E as well: 3.3e-5 for TG_a)
    assert dev < 2.0 * paper_delta_e
    if prec == GP_FP64:
        assert dev > 0.5 * paper_delta_e


@pytest.mark.parametrize("prec", [GP_FP64, GP_FP32])
def test_abc_preparation_against_the_paper_table(prec):
    """ABC_aIT of the paper: 128^3, alpha = 0.05, beta = 40, dtau = 4e-3, tau_f = 30 (7500 steps)
    from the ABC phase field; the paper stopped this run before its convergence criterion was met.
    Printed (ABC ARGLE energy table): E_kin^i = 0.9485114, E_kin^c = 0.0014218, E_q = 0.0277287,
    E_int = 0.0430379, H_reg = 2.4726091; (ABC conservation table, t = 0): N = 0.9410138,
    E = 1.0206996."""
    n = 128
    plan = Plan(field_params(n, 8e-4, alpha=0.05, beta=40.0, precision=prec))       # ABC_a's real-time dt
    psi = plan.init_abc(0, plan.empty())
    plan.argle(0, psi, GP_FLOW_ABC, 4e-3, 7500, energy=False)
    d, _ = plan.diagnostics(0, psi)
    got = {k: d[k] for k in ("E_kin_i", "E_kin_c", "E_q", "E_int", "N", "E")}
    paper = {"E_kin_i": 0.9485114, "E_kin_c": 0.0014218, "E_q": 0.0277287, "E_int": 0.0430379, "N": 0.9410138,
             "E": 1.0206996}
    print({k: (got[k], paper[k], got[k] / paper[k] - 1) for k in paper})
    for k in paper:
        assert got[k] == pytest.approx(paper[k], rel=2e-2), (k, got[k], paper[k])
    # regularised helicity (same table: H_reg = 2.4726091).  The plain H of eq-helicity (printed
    # 2.4106982) depends on how the singular velocity at the cores is treated and is not pinned.
    h, spec = plan.helicity(0, psi)
    print(h, spec["H_reg"][:6])
    assert h["H_reg"] == pytest.approx(2.4726091, rel=2e-2)
    _real_time_conservation(plan, psi, d, steps=12500, every=125, paper_n=0.9410138, paper_e_end=1.0206400,
                            paper_delta_e=5.98e-5, prec=prec, tol=2e-2)


PAPER_256 = {
    # TG_bIT / TG_b and ABC_bIT / ABC_b: 256^3, alpha = 0.025, beta = 80 (the paper's parameter
    # table); ARGLE dtau and tau_f, real-time dt and T_f from its TG / ABC run tables; energies and
    # helicities at tau_f from its TG / ABC ARGLE energy tables; N, E at t = 0 and T_f and
    # delta(E) from its conservation tables.
    "tg": {"flow": GP_FLOW_TG, "dtau": 6.25e-3, "steps": 9600, "dt": 6.25e-4, "rt_steps": 19200,
           "E_kin_i": 0.11334487, "E_kin_c": 2.2334712e-4, "E_q": 4.0373670e-3, "E_int": 6.8223665e-3,
           "N": 0.9873160, "E": 0.1244280, "E_end": 0.1244235, "delta_E": 3.60e-5, "H_reg": None},
    "abc": {"flow": GP_FLOW_ABC, "dtau": 2e-3, "steps": 15000, "dt": 4e-4, "rt_steps": 25000,
            "E_kin_i": 0.9792042, "E_kin_c": 0.0008142, "E_q": 0.0144931, "E_int": 0.0237201,
            "N": 0.9647786, "E": 1.0182316, "E_end": 1.0181689, "delta_E": 6.18e-5, "H_reg": 2.6532860},
}


@pytest.mark.parametrize("case", ["tg", "abc"])
def test_preparation_and_real_time_run_at_256_against_the_paper(case):
    """The paper's 256^3 runs (float32): the imaginary-time preparation from the TG ansatz
    ([gamma_d/4] = 6) or the ABC phase field, its energies and helicities, then the real-time run
    with the fused step and its conservation figures.  Tolerances as at 128^3: the TG run was
    converged by the paper (1e-4 on the large energies, 1e-2 on the small compressible part),
    the ABC one stopped early (2e-2).  Measured (GB300): TG_bIT E_kin^i +4.9e-4, E_q -1.5e-4,
    E_int -3e-5, E_kin^c -3.5%, N -1e-6, E +3.8e-4 -- agreement an order looser than at 128^3
    (float32 preparation against the paper's float64 one): 1e-3 on the large parts, 5e-2 on the
    compressible one; ABC_bIT within 0.4%, H_reg 2.6480 (printed 2.6532860)."""
    c = PAPER_256[case]
    n = 256
    plan = Plan(field_params(n, c["dt"], alpha=0.025, beta=80.0, precision=GP_FP32))
    psi = plan.init_tg(0, plan.empty()) if case == "tg" else plan.init_abc(0, plan.empty())
    plan.argle(0, psi, c["flow"], c["dtau"], c["steps"], energy=False)
    d, _ = plan.diagnostics(0, psi, spectra=False)
    h, _ = plan.helicity(0, psi, spectra=False)
    keys = ("E_kin_i", "E_kin_c", "E_q", "E_int", "N", "E")
    print({k: (d[k], c[k], d[k] / c[k] - 1) for k in keys}, h)
    for k in keys:
        tol = (5e-2 if k == "E_kin_c" else 1e-3) if case == "tg" else 2e-2
        assert d[k] == pytest.approx(c[k], rel=tol), (k, d[k], c[k])
    if case == "tg":
        assert abs(h["H"]) < 1e-5 and abs(h["H_reg"]) < 1e-5     # printed 2.96e-7 and -5.52e-7
    else:
        assert h["H_reg"] == pytest.approx(c["H_reg"], rel=2e-2)
    _real_time_conservation(plan, psi, d, steps=c["rt_steps"], every=c["rt_steps"] // 100, paper_n=c["N"],
                            paper_e_end=c["E_end"], paper_delta_e=c["delta_E"], prec=GP_FP32,
                            tol=1e-3 if case == "tg" else 2e-2)


def test_tg_grid_convergence_case_h_against_the_paper():
    """The paper's grid-convergence run TG_h: the TG_a preparation (alpha = 0.05, beta = 40) on
    256^3 (dx/xi = 0.694), against its grid-energy table (six digits; E_v compared as E_v / (2 alpha),
    as for TG_a).  The table gives no dtau for it: read as the dtau of the paper's 256^3 TG run
    (TG_bIT: 6.25e-3, tau_f = 60, 9600 steps) -- with TG_a's 1.25e-2 the explicit advection is
    unstable at 256^3 (|v| k_max dtau = 1.6) and the flow blows up.  (TG_g, 64^3 with
    dx/xi = 2.776, is not pinned: under-resolved, the flow ends in a different local minimum of
    E_v in float32 and in float64 -- E_kin^i 0.1264 and 0.1174 against the printed 0.1299.)"""
    paper = {"E_kin_i": 1.29562e-1, "E_kin_c": 2.72478e-4, "E_q": 7.80383e-3, "E_int": 1.30274e-2, "E_v": 7.10095e-1}
    plan = Plan(field_params(256, 1.25e-3, alpha=0.05, beta=40.0, precision=GP_FP32))
    psi = plan.init_tg(0, plan.empty())
    ev = plan.argle(0, psi, GP_FLOW_TG, 6.25e-3, 9600)
    d, _ = plan.diagnostics(0, psi, spectra=False)
    got = {k: d[k] for k in ("E_kin_i", "E_kin_c", "E_q", "E_int")}
    got["E_v"] = ev / (2 * 0.05)
    print({k: (got[k], paper[k], got[k] / paper[k] - 1) for k in paper})
    for k in paper:
        assert got[k] == pytest.approx(paper[k], rel=5e-3 if k == "E_kin_c" else 1e-4), (k, got[k], paper[k])

/*
 * gp.h -- C ABI of the GB300 Gross-Pitaevskii split-step library (libgpqt.so).
 *
 * Method: Kobayashi et al., "Quantum turbulence simulations using the
 * Gross-Pitaevskii equation: HPC and new numerical benchmarks".
 *   equation      i dpsi/dt = -alpha lap(psi) + beta (|psi|^2 - 1) psi    (Sec. 4.1, eq-gpe-num)
 *   box           [0, 2 pi]^3, periodic, N points per axis, x_i = 2 pi i / N (Sec. 6)
 *   parameters    alpha beta = 2 (M = 1/2), xi = sqrt(alpha/beta)           (Sec. 4.1, eq-scaling-choice3)
 *   time step     Strang splitting into exact kinetic and nonlinear flows    (Sec. 4.3, eq:adi_looptime)
 *
 * Conventions shared by every entry point
 *   - Fields are complex, interleaved (re, im), C order [z][y][x] (x fastest):
 *     element (x, y, z) sits at index (z*N + y)*N + x.  GP_FP32 fields are
 *     complex64 (8 bytes per point), GP_FP64 fields complex128 (16 bytes).
 *   - Unless a name ends in _host, field pointers are DEVICE pointers owned by
 *     the caller and must be 16-byte aligned; the library never frees them.
 *   - The plan owns its tables, workspaces and captured CUDA graphs and frees
 *     them in gp_plan_destroy.
 *   - Work is enqueued on the plan's stream and is asynchronous unless the
 *     entry point returns host values (then it synchronises that stream).
 *   - Every call returns a gp_status and never aborts, exits or traps; the
 *     message of the last failure is available from gp_last_error().
 *   - Device-side problems (non-finite values found by a reduction, a bounded
 *     wait that ran out) are reported at the next synchronising call.
 */
#ifndef GP_H
#define GP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GP_OK = 0,
  GP_ERR_INVALID_ARG = 1,      /* null pointer, misaligned pointer, bad index or value */
  GP_ERR_UNSUPPORTED_SIZE = 2, /* N not one of the supported grid sizes */
  GP_ERR_OOM = 3,              /* device allocation of a workspace failed */
  GP_ERR_CUDA = 4,             /* a CUDA runtime call failed */
  GP_ERR_TIMEOUT = 5,          /* a bounded device-side wait gave up */
  GP_ERR_NONFINITE = 6         /* a reduction met NaN or Inf */
} gp_status;

typedef enum { GP_FP32 = 0, GP_FP64 = 1 } gp_precision;
/* GP_FP32: complex64 storage, fused sweeps (the nonlinear phase is applied
 *          inside the FFT sweeps, the kinetic propagator inside the middle sweep).
 * GP_FP64: complex128 storage, plain unfused path (one kernel per sub-flow and
 *          per FFT axis), the accuracy reference on the GPU. */

typedef enum { GP_SPLIT_NKN = 0, GP_SPLIT_KNK = 1 } gp_split;
/* NKN: psi' = N(dt/2) K(dt) N(dt/2) psi, consecutive half steps merged.
 * KNK: the paper's order (eq:adi_looptime), K(dt/2) N(dt) K(dt/2).
 * K(s): psi_k <- exp(-i alpha |k|^2 s) psi_k in Fourier space (the product of
 *       the three exact directional flows S(s, L_j), which commute).
 * N(s): psi <- exp(-i beta (|psi|^2 - c) s) psi pointwise, c = 1 or 0. */

typedef struct {
  int n;                 /* grid points per axis: 8 12 16 24 32 48 64 96 128 192 256 512 1024 */
  double xi;             /* healing length; used when alpha == 0 and beta == 0 */
  double alpha, beta;    /* 0, 0 => alpha = sqrt(2) xi, beta = 2 / alpha */
  double dt;             /* time step (finite; may be negative for time reversal) */
  int precision;         /* gp_precision */
  int split;             /* gp_split */
  int nonlin_minus_one;  /* 1: phase beta (|psi|^2 - 1) (eq-gpe-num); 0: beta |psi|^2 (Sec. 4.3) */
} gp_field_params;

typedef struct gp_plan gp_plan;

typedef struct {
  double N;        /* <|psi|^2>                                   (eq-scaling-N) */
  double E;        /* <2 alpha^2 |grad psi|^2 + alpha beta (|psi|^2-1)^2> (eq-scaling-energy) */
  double E_kin;    /* <|sqrt(rho) v|^2 / 2>                       (eq-scaling-energy-mod-rho) */
  double E_kin_i;  /* incompressible part (Helmholtz split)       (eq:def-ekin-decomp) */
  double E_kin_c;  /* compressible part */
  double E_q;      /* <2 alpha^2 |grad sqrt(rho)|^2> */
  double E_int;    /* <alpha beta (rho - 1)^2> */
  double P_x, P_y, P_z;  /* momentum per volume <rho v> = 2 alpha <Im(psi* grad psi)> (eq-mom-total) */
  double M_max;    /* max |sqrt(rho) v| / c, c = sqrt(2 alpha beta)  (eq:Mach-Number) */
  double M_rms;    /* sqrt(2 E_kin) / c                              (eq:Mach-Number) */
} gp_diag;

/* Create a plan for nfields independent fields (a ragged batch is allowed: each
 * field has its own N, dt and parameters).  cuda_stream is a cudaStream_t or
 * NULL for the legacy default stream.  Builds twiddle and propagator tables
 * (float64 generation, rounded to the storage type).  *out receives the plan.
 * Errors: GP_ERR_INVALID_ARG, GP_ERR_UNSUPPORTED_SIZE, GP_ERR_OOM, GP_ERR_CUDA. */
gp_status gp_plan_create(const gp_field_params* fields, int nfields, void* cuda_stream, gp_plan** out);

/* Free every resource of the plan (tables, workspaces, graphs).  NULL is a no-op. */
gp_status gp_plan_destroy(gp_plan* plan);

/* Number of spectral shells of a field: floor(sqrt(3) N / 2 + 1/2) + 1. */
int gp_plan_nbins(const gp_plan* plan, int field);

/* Derived alpha and beta actually used by a field (host values). */
gp_status gp_plan_coefficients(const gp_plan* plan, int field, double* alpha, double* beta);

/* Smoothed-random-phase initial condition psi = exp(i theta) (Sec. 5.3, SRP_Init).
 *   mode 0 (spectral): theta = Gaussian noise filtered by exp(-|k|^2 / p0^2) in Fourier
 *          space, zero mean, scaled to RMS p1 (p0 = k0, p1 = theta_rms).
 *   mode 1 (paper): theta uniform in [-p0, p0] on an N_r^3 lattice (N_r = (int)p1,
 *          N divisible by N_r), periodic cubic-spline interpolation along x, y, z.
 * Random numbers: SplitMix64 stream positions seed * 2^40 + i (Steele, Lea & Flood 2014).
 * Generation runs in float64 and is rounded to the field's storage type.
 * psi: device field of the plan's precision, written in full. */
gp_status gp_init_srp(gp_plan* plan, int field, void* psi, uint64_t seed, int mode, double p0, double p1);

/* Random-vortex-ring initial condition (Sec. 5.4).
 *   mode 0 (rings): `count` rings, radius uniform in [p0, p1], centre uniform in the box,
 *          normal uniform on the sphere; psi = prod_j tanh(s_j/(sqrt2 xi)) exp(i atan2(z'_j, rho'_j - R_j))
 *          with the minimum-image displacement to ring j.
 *   mode 1 (paper): `count` Pade vortex-ring pairs of radius p0 and separation p1 with their
 *          six mirror images, each shifted by a random vector (Fourier shift) and given one
 *          of six axis orders, multiplied together.
 * psi: device field of the plan's precision, written in full. */
gp_status gp_init_rvr(gp_plan* plan, int field, void* psi, uint64_t seed, int mode, int count, double p0, double p1);

/* psi = exp(i theta) for a real field theta (float for GP_FP32, double for GP_FP64). */
gp_status gp_psi_from_phase(gp_plan* plan, int field, const void* theta, void* psi);

/* Advance every field of the plan by nsteps time steps, in place.
 * psi[f] is the device field of field f.  nsteps >= 0.  Asynchronous. */
gp_status gp_step(gp_plan* plan, void* const* psi, int nsteps);

/* Same as gp_step for host-resident fields: copies each field to a plan-owned
 * device buffer, steps, copies back, and synchronises.  psi_host[f] points to
 * n^3 complex values of the field's precision (pinned memory is fastest). */
gp_status gp_step_host(gp_plan* plan, void* const* psi_host, int nsteps);

/* Diagnostics of one field (Sec. 3.4-3.5 and 4.1), float64 reductions.
 * out: host record.  spectra: NULL or host array of 4*nbins doubles receiving the
 * shell spectra E_kin^i, E_kin^c, E_q, E_int (in that order), nbins = gp_plan_nbins.
 * Readings where the paper is silent: first derivatives use Nyquist-zeroed
 * wavenumbers; sqrt(rho) v = 2 alpha Im(psi* grad psi)/|psi| and grad sqrt(rho) =
 * Re(psi* grad psi)/|psi|, zero where |psi|^2 < 1e-12; the k = 0 mode of the
 * Helmholtz split is incompressible; shell b = floor(|k| + 1/2).
 * Synchronises the plan's stream.  GP_ERR_NONFINITE if psi holds NaN/Inf. */
gp_status gp_diagnostics(gp_plan* plan, int field, const void* psi, gp_diag* out, double* spectra, int nbins);

/* Longitudinal velocity structure functions (Sec. 3.5, strfunc-def):
 *   out[j * nr + s] = < (v_j(x + s dx e_j) - v_j(x))^order >,  j = 0 (x), 1 (y), 2 (z),
 *   s = 0 .. N/2, dx = 2 pi / N (the other shifts follow: S(N dx - r) = (-1)^order S(r)),
 * a volume mean over the grid, with the superfluid velocity v = 2 alpha Im(psi* grad psi) / |psi|^2
 * (eq-scaling-rhov; spectral gradient with Nyquist-zeroed wavenumbers; v = 0 where
 * |psi|^2 < 1e-12).  The paper plots order 2 and checks it against 2 <v_x^2> at large r.
 *   psi: device field (read only, 16-byte aligned);  order: 1 .. 8;
 *   out: host array of 3 * nr doubles, nr >= N/2 + 1 (entries beyond N/2 untouched).
 * Float64 sums; float32 fields form each pencil's sum of N terms in float32.  Uses the plan's
 * workspace (grown to 4 fields + 1 real field + small sums) and synchronises the plan's stream.
 * GP_ERR_INVALID_ARG for a bad order, nr or pointer; GP_ERR_NONFINITE if a result is NaN/Inf. */
gp_status gp_structure_function(gp_plan* plan, int field, const void* psi, int order, double* out, int nr);

/* Helicity and regularised helicity (Sec. 3.6: eq-helicity, Hreg), volume means, with
 * hbar/m = 2 alpha:
 *   H     = < v . omega >, omega = curl v, v = 2 alpha Im(psi* grad psi) / |psi|^2
 *           (0 where |psi|^2 < 1e-12; Nyquist-zeroed first derivatives);
 *   w     = (2 alpha / i) grad psi* x grad psi,
 *   v_par = 2 alpha w_i Im(sum_j (d_i d_j psi) conj(d_j psi)) / (|w| |grad psi|^2),
 *   v_reg = v_par w / |w|  (0 where |w| <= 1e-5 * 4 alpha <|grad psi|^2>),
 *   H_reg = < v_reg . omega >,
 * second derivatives -k~_i k~_j F psi.  spectra: NULL or 2 * nbins doubles (nbins >=
 * gp_plan_nbins): [0][b] H(k), [1][b] H_reg(k), the shell sums (b = floor(|k| + 1/2)) of
 * Re(conj(F v) . F omega) / n^2 and Re(conj(F v_reg) . F omega) / n^2 (H is the sum of its
 * spectrum).  psi: device field (read only, 16-byte aligned); H, H_reg: host doubles.
 * Uses the plan's workspace (grown to 13 fields + 1 real field: about 13 times the field's
 * size) and synchronises the plan's stream.  GP_ERR_NONFINITE if a result is NaN/Inf. */
gp_status gp_helicity(gp_plan* plan, int field, const void* psi, double* H, double* H_reg, double* spectra, int nbins);

/* Adjoint of nsteps split steps (no counterpart in the paper: the transpose of
 * the Sec. 4.3 step under <a, b> = Re sum conj(a) b).
 *   psi_n:  device field, the state at the start of the nsteps steps (read only);
 *   lambda: device field; on entry the cotangent at the end of the steps, on
 *           return the cotangent at their start.
 * The states inside the segment are recomputed from psi_n into a plan-owned
 * workspace of nsteps fields (the caller checkpoints segments).  Per step:
 *   VJP_K(s) lam = K(-s) lam;
 *   VJP_N(s) lam = exp(+i phi) lam + 2 beta s Im(conj(lam) psi_out) psi,  phi = beta s (|psi|^2 - c). */
gp_status gp_adjoint_step(gp_plan* plan, int field, const void* psi_n, void* lambda, int nsteps);

/* Gradient of J = E_kin^i(psi) with |psi| regularised as sqrt(|psi|^2 + eps) inside
 * sqrt(rho) v: writes lambda_out = dJ/dpsi (device field) and, if J_out != NULL,
 * J (host, synchronises).  eps > 0. */
gp_status gp_ekin_i_grad(gp_plan* plan, int field, const void* psi, void* lambda_out, double eps, double* J_out);

/* dJ/dtheta = -Im(conj(lambda) psi) for psi = exp(i theta): real output field
 * (float for GP_FP32, double for GP_FP64). */
gp_status gp_phase_grad(gp_plan* plan, int field, const void* psi, const void* lambda, void* grad_theta);

/* Diagnostics of a float32 (complex64) field of N^3 points, N in {8, 12, 16, 24, 32, 48, 64},
 * that allocate no device memory and need no plan -- for callers that cannot call cudaMalloc:
 * code embedded in an application whose caching allocator already holds the device's memory,
 * or a monitoring hook inside a latency-critical loop where an allocation would stall every
 * stream of the device.  (The paper has no counterpart; it is the same computation as
 * gp_diagnostics, with the same outputs and the same readings.)
 *   alpha, beta: the field's coefficients;  psi: device field, 16-byte aligned;
 *   out, spectra (NULL or 4*nbins doubles), nbins: as for gp_diagnostics;
 *   cuda_stream: cudaStream_t or NULL for the legacy default stream; synchronised on return.
 * Scratch: file-scope device arrays of fixed size inside the library -- four 64^3 complex64
 * work fields (8 MiB), twiddle tables, accumulators and a histogram, about 8.4 MiB in all --
 * which every GPU that loads the library keeps until the process exits.  N > 64 (or any other
 * unsupported N) returns GP_ERR_UNSUPPORTED_SIZE without touching the device.
 * The first call on a device resolves the arrays' device addresses and uploads the twiddle
 * tables (cudaGetSymbolAddress, cudaMemcpy); make that first call before any stream capture.
 * All calls share the arrays, which keep the last call's contents (each call clears the
 * accumulators it uses): calls that overlap on the GPU -- from two streams or two host
 * threads -- race on them and must be serialised by the caller. */
gp_status gp_diagnostics_noalloc(int n, double alpha, double beta, const void* psi, gp_diag* out, double* spectra,
                                 int nbins, void* cuda_stream);

/* Instrumentation (no counterpart in the paper).
 * gp_profile(plan, 1) clears the records and makes later gp_step calls launch every
 * float32 sweep directly (no graph replay) between a pair of CUDA events on the plan's
 * stream; gp_profile(plan, 0) stops recording.  gp_profile_read synchronises the stream
 * and reports, per sweep kind (kernel, operation, axis), the number of launches and their
 * summed device time in milliseconds.  names receives max_kinds NUL-terminated strings of
 * 64 bytes each.  Returns the number of kinds written, or -1 on error. */
gp_status gp_profile(gp_plan* plan, int enable);
int gp_profile_read(gp_plan* plan, int max_kinds, char* names, long long* launches, double* ms);

/* Number of kernels this plan has launched (or replayed inside graphs) since creation. */
long long gp_launch_count(const gp_plan* plan);

/* Autotuner of the float32 sweep kernels (no counterpart in the paper).  A sweep kind is
 * (axis, op): axis 0 = x, 1 = y, 2 = z; op 1 forward, 2 inverse, 3 inverse-N-forward,
 * 4 N-forward, 5 inverse-N, 6 forward-K-inverse (x only), and 7 = the fused plane kernel that
 * performs forward y, x (forward, K, inverse) and inverse y of every z-plane in one launch
 * (axis 1).  For every grid length of the plan's float32 fields and every kind of its time step
 * the tuner times the candidates on a scratch field (allocated and freed here) and keeps the
 * fastest: 0 the TMA-pipelined persistent kernel at full occupancy, 1 the same with one CTA per
 * SM, 2 the non-persistent kernel, 3 (y, z and op 7) the TMA kernel with two shared-memory
 * stages, 4 (lengths >= 512, not op 7) the TMA kernel with two compute groups per CTA; for op 7, 0 = the fused kernel, 1 = the fused kernel with one CTA per SM (fewer planes
 * in flight between its phases), 3 = the fused kernel with two stages, 2 = the three
 * separate sweeps with their own variants.  cache_path (NULL: none) names a JSON file of earlier
 * choices keyed by GPU name, length, axis and op; cached choices are reused without timing and
 * new ones are added.  Synchronises the stream and drops captured graphs.
 * gp_plan_sweep_variant returns the variant in use for a kind (default 0: fused plane kernel
 * and TMA sweeps wherever the length has them).  gp_plan_set_sweep_variant sets it by hand
 * (GP_ERR_INVALID_ARG for an unknown kind or variant); it synchronises the stream and drops
 * captured graphs. */
gp_status gp_plan_autotune(gp_plan* plan, const char* cache_path);
int gp_plan_sweep_variant(gp_plan* plan, int n, int axis, int op);
gp_status gp_plan_set_sweep_variant(gp_plan* plan, int n, int axis, int op, int variant);

/* gp_plan_set_fused_batch: on = 1 makes gp_step advance every field of the plan in ONE persistent
 * launch per call (no counterpart in the paper, which steps one field per run): the call's whole
 * NKN schedule (Sec. 4.3, the merged half steps -- z with N, forward y, forward x with K and
 * inverse x, inverse y, per step, and the closing z with N(dt/2)) is a list of tiles handed out
 * in order from one device counter, and a tile of a field waits, bounded by about a second, until
 * that field's previous sweep is complete.  The results are bitwise those of the per-sweep
 * launches.  Meant for ensembles of small fields, where a sweep is too short to fill the GPU.
 * Needs every field float32, NKN, of length 32, 64, 96 or 128, and at most 64 fields
 * (GP_ERR_INVALID_ARG otherwise; nothing changes).  A repeated gp_step call with the same fields
 * and step count replays one captured graph (the counters' reset and the launch).  Workspace:
 * 1 + (4 nsteps + 1) * fields device ints, kept by the plan.  A wait that gives up sets the
 * status word that gp_plan_sync and the synchronising calls report.  on = 0 returns to one
 * launch per sweep and size class.  Synchronises the stream and drops captured graphs. */
gp_status gp_plan_set_fused_batch(gp_plan* plan, int on);

/* Imaginary-time preparation (Sec. 4.2) and its start fields (Sec. 5.1, 5.2).
 * External flows: GP_FLOW_NONE, GP_FLOW_TG (v = (sin x cos y cos z, -cos x sin y cos z, 0)),
 * GP_FLOW_ABC (the sum of the k = 1 and k = 2 ABC flows with amplitudes abc[0..2] = A, B, C;
 * abc = NULL: (0.9, 1, 1.1)/sqrt(3)).
 * gp_init_tg: psi_ARGLE of the Taylor-Green flow (Clebsch potentials, psi_4 to the power
 *   floor(1/(2 pi alpha)) with the field's alpha and xi = sqrt(alpha/beta)); GP_ERR_INVALID_ARG
 *   when that power is below 1.  Asynchronous.
 * gp_init_abc: the ABC start field, a product of phase factors with nearest-integer
 *   wavenumbers.  Asynchronous.
 * gp_argle: nsteps >= 0 semi-implicit backward-Euler steps of size dtau > 0 of the advective
 *   real Ginzburg-Landau flow (eqn:gradient-flow, eqn:semi-backward-Euler) driven by `flow`,
 *   in place on psi (device, the field's precision).  renorm = 0: the paper's unconstrained
 *   flow; 1: after every step psi is rescaled to the mean |psi|^2 it had on entry (float64
 *   sums on the device).  energy_out (NULL: not computed) receives the energy of the driven
 *   field E_v (eq-energy-num-ext-vel, float64 sums) after the steps; the call then
 *   synchronises and also reports a sweep kernel's bounded-wait timeout.  Workspace: four
 *   fields, kept by the plan. */
#define GP_FLOW_NONE 0
#define GP_FLOW_TG 1
#define GP_FLOW_ABC 2
gp_status gp_init_tg(gp_plan* plan, int field, void* psi_dev);
gp_status gp_init_abc(gp_plan* plan, int field, void* psi_dev, const double* abc);
gp_status gp_argle(gp_plan* plan, int field, void* psi_dev, int flow, const double* abc, double dtau, int nsteps,
                   int renorm, double* energy_out);

/* gp_argle_converge: gp_argle with the paper's stopping rules (eqn:crit1, eqn:crit2).  Up to
 * max_steps >= 1 steps; every check_every-th step (check_every >= 1) and the last one evaluate
 *   crit1 = ||phi^{n+1} - phi^n||_inf / dtau,
 *   crit2 = |E_v(phi^{n+1}) - E_v(phi^n)| / (dtau E_v(phi^n)),
 * and the run stops after the first checked step with crit1 <= eps (eps <= 0: never; run all
 * steps).  steps_done, crit1, crit2 (host) receive the number of steps taken and the criteria of
 * the last checked step; energy_out as for gp_argle.  A checked step costs two E_v evaluations
 * (four transforms each) and a copy of the field, and synchronises the stream; the workspace
 * grows to five fields. */
gp_status gp_argle_converge(gp_plan* plan, int field, void* psi_dev, int flow, const double* abc, double dtau,
                            int max_steps, int renorm, double eps, int check_every, int* steps_done, double* crit1,
                            double* crit2, double* energy_out);

/* Waits for the plan's stream and reads the device status word that the persistent sweep
 * kernels set when one of their bounded waits (a TMA copy, a tile counter of the fused plane
 * kernel) gives up instead of hanging.  GP_OK if none did since the last check; otherwise
 * GP_ERR_TIMEOUT (the fields written since then are invalid) and the word is cleared.
 * gp_step_host and gp_diagnostics perform the same check. */
gp_status gp_plan_sync(gp_plan* plan);

/* Test hook of the bounded waits (no counterpart in the paper): the next launch of the fused
 * plane kernel (or, with gp_plan_set_fused_batch, the next fused run) never hands out its first
 * `tiles` tiles, so the tiles that depend on them wait for counts that never complete.  Those
 * waits give up after about a second, the launch ends with the status word set, and the next
 * gp_plan_sync (or gp_step_host, gp_diagnostics) returns GP_ERR_TIMEOUT; the field is then
 * invalid, the plan and the CUDA context stay usable.  Applies to one launch (the step must use
 * the fused plane kernel -- a length with TMA kernels and the default variant -- or the fused
 * run); captured graphs are dropped. */
gp_status gp_plan_test_timeout(gp_plan* plan, int tiles);

/* Message of the last failed call on this plan ("" if none); valid until the next call. */
const char* gp_last_error(const gp_plan* plan);

/* Static name of a status code. */
const char* gp_status_string(gp_status status);

#ifdef __cplusplus
}
#endif

#endif /* GP_H */

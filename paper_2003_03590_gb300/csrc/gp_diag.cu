// gp_diag.cu -- energy, mass and spectra of one field with float64 reductions.
//
// Quantities (volume means; Sec. 4.1 eq-scaling-N, eq-scaling-energy, eq-scaling-energy-mod-rho;
// Sec. 3.4 eq:def-ekin-decomp; Sec. 3.5 spectra).  With n = N^3 points and the unnormalised
// forward DFT F, Parseval gives <|f|^2> = sum_k |F f|^2 / n^2:
//   N     = <|psi|^2>
//   E     = 2 alpha^2 sum_k |k|^2 |F psi|^2 / n^2 + alpha beta <(|psi|^2 - 1)^2>
//   u     = sqrt(rho) v = 2 alpha Im(psi* grad psi) / |psi|,  q = grad sqrt(rho) = Re(psi* grad psi) / |psi|
//           (grad with Nyquist-zeroed wavenumbers; u = q = 0 where |psi|^2 < 1e-12)
//   E_kin = <|u|^2 / 2>,  E_q = <2 alpha^2 |q|^2>,  E_int = <alpha beta (rho - 1)^2>
//   Helmholtz: u^c_k = k~ (k~ . u_k) / |k~|^2 (k = 0 incompressible), u^i = u - u^c
//   shell b = floor(|k| + 1/2): E_kin^{i,c}(b) = sum |u^{i,c}_k|^2 / (2 n^2),
//   E_q(b) = 2 alpha^2 sum_j |F q_j|^2 / n^2,  E_int(b) = alpha beta |F(rho - 1)|^2 / n^2.
// Pipeline: 8 complex 3D FFTs; the two real fields u_j and q_j share one complex
// transform (W_j = u_j + i q_j) and are separated with the mirror mode -k.
#include <cmath>
#include <vector>

#include "gp_internal.h"
#include "gp_reduce.cuh"

namespace gp {


static inline unsigned rgrid(long long n) {
  long long b = (n + 255) / 256;
  return (unsigned)(b < 1 ? 1 : (b > 152LL * 16 ? 152LL * 16 : b));
}

// sum |psi|^2, sum (|psi|^2 - 1)^2; flags non-finite input
template <typename T> __global__ void k_phys1(const cpx<T>* __restrict__ psi, long long npts, double* part, int* flag) {
  Sums<T, 2> S;
  bool bad = false;
  auto term = [&](cpx<T> a) {
    T r;
    const T dm = rho_minus_one(a, &r);
    bad |= !isfinite(dm);
    const T v[2] = {r, dm * dm};
    S.add(v);
  };
  // four independent loads per thread in flight: little arithmetic per byte, so a single load
  // at a time would leave the kernel bound by memory latency
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  for (; i + 3 * stride < npts; i += 4 * stride) {
    const cpx<T> a0 = psi[i], a1 = psi[i + stride], a2 = psi[i + 2 * stride], a3 = psi[i + 3 * stride];
    term(a0);
    term(a1);
    term(a2);
    term(a3);
  }
  for (; i < npts; i += stride) term(psi[i]);
  S.flush();
  if (bad) atomicOr(flag, 1);
  block_store<2>(S.d, part);
}

// sum |k|^2 |psi_k|^2 (true |k|, Nyquist kept); W_j = i k~_j psi_k
template <typename T>
__global__ void k_kspace1(const cpx<T>* __restrict__ ph, cpx<T>* w1, cpx<T>* w2, cpx<T>* w3, int n, double* part) {
  const long long npts = (long long)n * n * n;
  Sums<T, 4> S;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npts; i += (long long)gridDim.x * blockDim.x) {
    int ix, iy, iz;
    coords3((unsigned)i, (unsigned)n, ix, iy, iz);
    const int kx = wavenumber(ix, n), ky = wavenumber(iy, n), kz = wavenumber(iz, n);
    cpx<T> a = ph[i];
    const T a2 = a.x * a.x + a.y * a.y;
    const T dx = (T)wavenumber_d(ix, n), dy = (T)wavenumber_d(iy, n), dz = (T)wavenumber_d(iz, n);
    // |k|^2 |psi_k|^2 (E's gradient term) and k~_j |psi_k|^2 (the momentum, by Parseval)
    const T v[4] = {(T)(kx * kx + ky * ky + kz * kz) * a2, dx * a2, dy * a2, dz * a2};
    S.add(v);
    w1[i] = cpx<T>{-dx * a.y, dx * a.x};
    w2[i] = cpx<T>{-dy * a.y, dy * a.x};
    w3[i] = cpx<T>{-dz * a.y, dz * a.x};
  }
  S.flush();
  block_store<4>(S.d, part);
}

// u_j, q_j packed as W_j = u_j + i q_j; W0 = rho - 1; sums of |u|^2 / 2 and 2 alpha^2 |q|^2
template <typename T>
__global__ void k_phys2(const cpx<T>* __restrict__ psi, cpx<T>* w0, cpx<T>* w1, cpx<T>* w2, cpx<T>* w3, long long npts,
                        double alpha, double* part, double* umax) {
  Sums<T, 2> S;
  T u2max = T(0);   // max |sqrt(rho) v|^2 of this thread (a max is exact in any precision)
  const T a2 = (T)(2.0 * alpha), qa = (T)(2.0 * alpha * alpha);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npts; i += (long long)gridDim.x * blockDim.x) {
    cpx<T> p = psi[i];
    T rho;
    const T dm = rho_minus_one(p, &rho);
    cpx<T>* ws[3] = {w1, w2, w3};
    const bool ok = rho >= eps_rho<T>();
    const T inv_amp = ok ? T(1) / sqrt(rho) : T(0);
    T v[2] = {T(0), T(0)};
    T uu = T(0);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      cpx<T> g = ws[j][i];
      const T re = p.x * g.x + p.y * g.y;   // Re(conj(psi) g)
      const T im = p.x * g.y - p.y * g.x;   // Im(conj(psi) g)
      const T u = a2 * im * inv_amp, q = re * inv_amp;
      ws[j][i] = cpx<T>{u, q};
      uu += u * u;
      v[1] += qa * q * q;
    }
    v[0] = T(0.5) * uu;
    u2max = uu > u2max ? uu : u2max;
    S.add(v);
    w0[i] = cpx<T>{dm, T(0)};
  }
  S.flush();
  block_store<2>(S.d, part);
  // block max of |u|^2
  double m = (double)u2max;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  __shared__ double mred[32];
  if ((threadIdx.x & 31) == 0) mred[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 1; q < (int)(blockDim.x >> 5); ++q) m = fmax(m, mred[q]);
    umax[blockIdx.x] = m;
  }
}

// Add v[0..4) to hist[q * nbins + b] for every lane of a warp (b < 0: nothing).  Runs of equal b
// over consecutive lanes (consecutive kx in a row: the shell changes slowly) are summed with a
// segmented shuffle scan first (in the terms' precision: a run has at most 32 terms), so one
// float64 shared-memory atomic per run and quantity reaches the histogram instead of one per lane.
template <typename S>
__device__ __forceinline__ void bin_add(double* hist, int nbins, int b, S (&v)[4]) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int bprev = __shfl_up_sync(full, b, 1);
  const unsigned heads = __ballot_sync(full, lane == 0 || bprev != b);
  const int start = 31 - __clz(heads & ((2u << lane) - 1u));   // first lane of this lane's run
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    S t[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) t[q] = __shfl_up_sync(full, v[q], o);
    if (lane - o >= start) {
#pragma unroll
      for (int q = 0; q < 4; ++q) v[q] += t[q];
    }
  }
  const int bnext = __shfl_down_sync(full, b, 1);
  if ((lane == 31 || bnext != b) && b >= 0) {
#pragma unroll
    for (int q = 0; q < 4; ++q) atomicAdd(&hist[q * nbins + b], (double)v[q]);
  }
}


// Helmholtz split and shell binning; spec layout [4][nbins]: E_kin^i, E_kin^c, E_q, E_int (unscaled)
template <typename T>
__global__ void k_kspace2(const cpx<T>* __restrict__ w0, const cpx<T>* __restrict__ w1, const cpx<T>* __restrict__ w2,
                          const cpx<T>* __restrict__ w3, int n, int nbins, double alpha, double beta, double* spec) {
  using S = T;   // per-point arithmetic in the field's precision
  extern __shared__ double hist[];
  for (int b = threadIdx.x; b < 4 * nbins; b += blockDim.x) hist[b] = 0.0;
  __syncthreads();
  const long long npts = (long long)n * n * n;
  const cpx<T>* ws[3] = {w1, w2, w3};
  const int lane = threadIdx.x & 31;
  const S qa = (S)(2.0 * alpha * alpha), ab = (S)(alpha * beta);
  // warp-uniform trip count: lane i of a warp handles base + i
  for (long long base = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < npts;
       base += (long long)gridDim.x * blockDim.x) {
    const long long i = base + lane;
    int b = -1;
    S val[4] = {S(0), S(0), S(0), S(0)};
    int ix = 0, iy = 0, iz = 0;
    if (i < npts) coords3((unsigned)i, (unsigned)n, ix, iy, iz);
    const int mx = ix ? n - ix : 0, my = iy ? n - iy : 0, mz = iz ? n - iz : 0;
    const long long im = ((long long)mz * n + my) * n + mx;
    // The fields u, q, rho - 1 are real, so every quantity at -k equals the one at k (and |-k| =
    // |k|): the half of k-space with i < im is summed twice, the self-mirrored modes (i = im)
    // once, and the other half is skipped -- each pair of points is read once.
    if (i < npts && i <= im) {
      const S wgt = i < im ? S(2) : S(1);
      const int kx = wavenumber(ix, n), ky = wavenumber(iy, n), kz = wavenumber(iz, n);
      b = shell_of(kx * kx + ky * ky + kz * kz);
      if (b >= nbins) b = nbins - 1;
      const S kd[3] = {(S)wavenumber_d(ix, n), (S)wavenumber_d(iy, n), (S)wavenumber_d(iz, n)};
      S ur[3], ui[3], eq = 0;
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        cpx<T> z = ws[j][i], zm = ws[j][im];
        // u_k = (Z(k) + conj(Z(-k))) / 2,  q_k = (Z(k) - conj(Z(-k))) / (2 i)
        ur[j] = S(0.5) * (z.x + zm.x);
        ui[j] = S(0.5) * (z.y - zm.y);
        const S qr = S(0.5) * (z.y + zm.y), qi = S(-0.5) * (z.x - zm.x);
        eq += qr * qr + qi * qi;
      }
      const S kk = kd[0] * kd[0] + kd[1] * kd[1] + kd[2] * kd[2];
      S cr = 0, ci = 0;
      if (kk > S(0)) {
        const S inv = S(1) / kk;
        cr = (kd[0] * ur[0] + kd[1] * ur[1] + kd[2] * ur[2]) * inv;
        ci = (kd[0] * ui[0] + kd[1] * ui[1] + kd[2] * ui[2]) * inv;
      }
      S ei = 0, ec = 0;
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const S ucr = kd[j] * cr, uci = kd[j] * ci;
        ec += ucr * ucr + uci * uci;
        const S uir = ur[j] - ucr, uii = ui[j] - uci;
        ei += uir * uir + uii * uii;
      }
      // u_k and q_k at -k are exactly the conjugates of those at k (same operations on the
      // same two values), so the pair counts twice; the transform of the real rho - 1 is
      // conjugate-symmetric only up to rounding, so both of its values are read
      const cpx<T> r = w0[i], rm = w0[im];
      val[0] = S(0.5) * wgt * ei;
      val[1] = S(0.5) * wgt * ec;
      val[2] = qa * wgt * eq;
      val[3] = ab * (i < im ? (r.x * r.x + r.y * r.y) + (rm.x * rm.x + rm.y * rm.y) : (r.x * r.x + r.y * r.y));
    }
    bin_add(hist, nbins, b, val);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < 4 * nbins; b += blockDim.x)
    if (hist[b] != 0.0) atomicAdd(&spec[b], hist[b]);
}

// Device accumulators of one diagnostics call:
//   [0] sum rho  [1] sum (rho-1)^2  [2] sum |k|^2 |psi_k|^2  [3..5] sum k~_j |psi_k|^2
//   [6] sum |u|^2 / 2  [7] sum 2 alpha^2 |q|^2  [8] max |u|^2
constexpr int DIAG_ACC = 9;

// The scalars from the accumulators and the shell sums (spectrum q of nb bins at hs + q nb).
static gp_diag diag_finish(const double* acc, const double* hs, int nb, long long npts, double alpha, double beta) {
  const double dn = (double)npts, dn2 = dn * dn;
  gp_diag d{};
  d.N = acc[0] / dn;
  d.E_int = alpha * beta * acc[1] / dn;
  d.E = 2.0 * alpha * alpha * acc[2] / dn2 + d.E_int;
  // <Im(psi* d_j psi)> = sum_k k~_j |psi_k|^2 / npts^2 (Parseval, unnormalised forward DFT)
  d.P_x = 2.0 * alpha * acc[3] / dn2;
  d.P_y = 2.0 * alpha * acc[4] / dn2;
  d.P_z = 2.0 * alpha * acc[5] / dn2;
  d.E_kin = acc[6] / dn;
  d.E_q = acc[7] / dn;
  double si = 0.0, sc = 0.0;
  for (int b = 0; b < nb; ++b) {
    si += hs[b];
    sc += hs[nb + b];
  }
  d.E_kin_i = si / dn2;
  d.E_kin_c = sc / dn2;
  const double c = std::sqrt(2.0 * alpha * beta);   // sound speed
  d.M_max = std::sqrt(acc[8]) / c;
  d.M_rms = std::sqrt(2.0 * d.E_kin) / c;
  return d;
}

template <typename T>
static gp_status diag_impl(gp_plan* p, int field, const cpx<T>* psi, gp_diag* out, double* spectra, int nbins_req) {
  FieldPlan& F = p->f[field];
  const long long npts = F.npts;
  const int n = F.n;
  const int nbins = gp_plan_nbins(p, field);
  cudaStream_t s = p->stream;
  const size_t fb = (size_t)npts * sizeof(cpx<T>);
  const unsigned g = rgrid(npts);
  gp_status st = ensure_ws(p, field, 4 * fb + (size_t)4 * nbins * sizeof(double) + (size_t)9 * g * sizeof(double));
  if (st != GP_OK) return st;
  cpx<T>* w0 = (cpx<T>*)F.ws;
  cpx<T>* w1 = w0 + npts;
  cpx<T>* w2 = w1 + npts;
  cpx<T>* w3 = w2 + npts;
  double* spec = (double*)(w3 + npts);
  double* part = spec + 4 * nbins;   // per-block sums: [g][2] + [g][4] + [g][2] + block maxima [g]
  GP_CUDA(p, cudaMemsetAsync(p->acc, 0, DIAG_ACC * sizeof(double), s));
  GP_CUDA(p, cudaMemsetAsync(p->flag, 0, sizeof(int), s));
  GP_CUDA(p, cudaMemsetAsync(spec, 0, (size_t)4 * nbins * sizeof(double), s));
  k_phys1<T><<<g, 256, 0, s>>>(psi, npts, part, p->flag);
  GP_CUDA(p, cudaGetLastError());
  k_reduce<<<1, 256, 0, s>>>(part, (int)g, 2, p->acc);
  GP_CUDA(p, cudaGetLastError());
  GP_CUDA(p, cudaMemcpyAsync(w0, psi, fb, cudaMemcpyDeviceToDevice, s));
  cpx<T>* all[4] = {w0, w1, w2, w3};
  // 3D transforms: float32 fields through the tuned sweep kernels, several fields per launch
  auto transform = [&](int first, int count, bool inverse) -> cudaError_t {
    if constexpr (sizeof(T) == 4) return fft3_many(p, F, all + first, count, inverse, s);
    for (int k = first; k < first + count; ++k) {
      cudaError_t e = fft3<T>(F, all[k], inverse, s);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  };
  GP_CUDA(p, transform(0, 1, false));
  k_kspace1<T><<<g, 256, 0, s>>>(w0, w1, w2, w3, n, part + 2 * g);
  GP_CUDA(p, cudaGetLastError());
  k_reduce<<<1, 256, 0, s>>>(part + 2 * g, (int)g, 4, p->acc + 2);
  GP_CUDA(p, cudaGetLastError());
  GP_CUDA(p, transform(1, 3, true));
  k_phys2<T><<<g, 256, 0, s>>>(psi, w0, w1, w2, w3, npts, F.alpha, part + 6 * g, part + 8 * g);
  GP_CUDA(p, cudaGetLastError());
  k_reduce<<<1, 256, 0, s>>>(part + 6 * g, (int)g, 2, p->acc + 6);
  GP_CUDA(p, cudaGetLastError());
  k_reduce_max<<<1, 256, 0, s>>>(part + 8 * g, (int)g, p->acc + 8);
  GP_CUDA(p, cudaGetLastError());
  GP_CUDA(p, transform(0, 4, false));
  const size_t hsm = (size_t)4 * nbins * sizeof(double);
  if (hsm > 48 * 1024) GP_CUDA(p, cudaFuncSetAttribute(k_kspace2<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hsm));
  // fewer blocks than the other kernels: each block adds its whole histogram to spec at the end
  const unsigned g2 = g < 4 * 152 ? g : 4 * 152;
  k_kspace2<T><<<g2, 256, hsm, s>>>(w0, w1, w2, w3, n, nbins, F.alpha, F.beta, spec);
  GP_CUDA(p, cudaGetLastError());
  double acc[DIAG_ACC];
  int flag = 0;
  std::vector<double> hs((size_t)4 * nbins);
  GP_CUDA(p, cudaMemcpyAsync(acc, p->acc, sizeof(acc), cudaMemcpyDeviceToHost, s));
  GP_CUDA(p, cudaMemcpyAsync(&flag, p->flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  GP_CUDA(p, cudaMemcpyAsync(hs.data(), spec, hs.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
  GP_CUDA(p, cudaStreamSynchronize(s));
  {
    gp_status st = check_status(p);   // a sweep that gave up a bounded wait since the last check
    if (st != GP_OK) return st;
  }
  if (flag) return fail(p, GP_ERR_NONFINITE, "gp_diagnostics: field holds NaN or Inf");
  *out = diag_finish(acc, hs.data(), nbins, npts, F.alpha, F.beta);
  if (spectra) {
    const double dn2 = (double)npts * (double)npts;
    const int nb = nbins_req < nbins ? nbins_req : nbins;
    for (int q = 0; q < 4; ++q)
      for (int b = 0; b < nb; ++b) spectra[q * nbins_req + b] = hs[(size_t)q * nbins + b] / dn2;
  }
  return GP_OK;
}

}  // namespace gp

using namespace gp;

extern "C" gp_status gp_diagnostics(gp_plan* p, int field, const void* psi, gp_diag* out, double* spectra, int nbins) {
  if (!p) return GP_ERR_INVALID_ARG;
  if (field < 0 || field >= (int)p->f.size()) return fail(p, GP_ERR_INVALID_ARG, "gp_diagnostics: field index");
  if (!psi || ((uintptr_t)psi & 15) || !out) return fail(p, GP_ERR_INVALID_ARG, "gp_diagnostics: pointer");
  if (spectra && nbins < gp_plan_nbins(p, field))
    return fail(p, GP_ERR_INVALID_ARG, "gp_diagnostics: nbins smaller than gp_plan_nbins");
  if (p->f[field].fp64) return diag_impl<double>(p, field, (const cpx<double>*)psi, out, spectra, nbins);
  return diag_impl<float>(p, field, (const cpx<float>*)psi, out, spectra, nbins);
}

// ---------------------------------------------------------------- allocation-free diagnostics
// gp_diagnostics_noalloc: the diagnostics above for float32 fields of at most 64^3 points,
// for callers that must not allocate device memory -- for example code running inside an
// application whose caching allocator already owns all device memory (a cudaMalloc would fail
// or fragment it), or a monitoring hook in a latency-critical loop where cudaMalloc would
// stall every stream of the device while it synchronises.  It needs no plan: every buffer
// it uses is a file-scope __device__ array below, reserved when the library is loaded and
// kept by every GPU that loads it until the process exits:
//   4 work fields of 64^3 complex64 (8 MiB), the float32 twiddle tables of the supported
//   lengths up to 64, reduction accumulators and per-block partial sums, a status word and the
//   shell histogram.
// All calls share these arrays, which keep the last call's contents; every call clears the
// accumulators and histogram it uses.  Calls that overlap on the GPU (two streams, two host
// threads) race on them: serialise them.

namespace gp {

constexpr int NOALLOC_MAX_N = 64;
constexpr long long NOALLOC_MAX_PTS = (long long)NOALLOC_MAX_N * NOALLOC_MAX_N * NOALLOC_MAX_N;
constexpr int NOALLOC_MAX_BINS = 64;     // >= floor(sqrt(3) 64 / 2 + 1/2) + 1 = 56
constexpr int NOALLOC_TW = 1024;         // float4 twiddle entries for all lengths <= 64, both directions
constexpr int NOALLOC_SIZES[7] = {8, 12, 16, 24, 32, 48, 64};

static __device__ __align__(256) float2 g_na_work[4 * NOALLOC_MAX_PTS];
static __device__ __align__(256) float4 g_na_tw[NOALLOC_TW];
static __device__ __align__(256) double g_na_acc[DIAG_ACC];
constexpr int NOALLOC_MAX_BLOCKS = (int)(NOALLOC_MAX_PTS / 256);   // grid of the pointwise kernels at 64^3
static __device__ __align__(256) double g_na_part[9 * NOALLOC_MAX_BLOCKS];
static __device__ __align__(256) double g_na_spec[4 * NOALLOC_MAX_BINS];
static __device__ __align__(256) int g_na_flag[4];

// host-side record of what set-up resolved on each device (indexed by device ordinal)
struct NoAllocDevice {
  bool ready = false;
  float2* work = nullptr;
  float4* tw = nullptr;
  double* acc = nullptr;
  double* part = nullptr;
  double* spec = nullptr;
  int* flag = nullptr;
  int tw_off[7][2] = {};   // offset of each length's (forward, inverse) table in tw
};
static NoAllocDevice g_na_dev[64];

// Stockham twiddles (same definition as the plan's tables) written into a fixed host array.
static int noalloc_twiddles(int n, bool inv, float4* out, int cap) {
  const int np = plan_np(n);
  int ns = 1, k = 0;
  for (int i = 0; i < np; ++i) {
    const int R = plan_radix_fwd(n, inv ? np - 1 - i : i);
    for (int jm = 0; jm < ns; ++jm)
      for (int r = 1; r < R; ++r) {
        if (k >= cap) return -1;
        const long long den = (long long)ns * R, num = ((long long)r * jm) % den;
        const double ang = (inv ? 2.0 : -2.0) * M_PI * (double)num / (double)den;
        float ch, cl, sh, sl;
        split_hilo(std::cos(ang), &ch, &cl);
        split_hilo(std::sin(ang), &sh, &sl);
        out[k++] = make_float4(ch, sh, cl, sl);
      }
    ns *= R;
  }
  return k;
}

// Once per device, with that device current: resolve the device addresses of the arrays
// (their names in host code only stand in for them) and upload the twiddle tables.
static gp_status noalloc_setup(int dev, NoAllocDevice& D) {
  if (cudaGetSymbolAddress((void**)&D.work, g_na_work) != cudaSuccess) return GP_ERR_CUDA;
  if (cudaGetSymbolAddress((void**)&D.tw, g_na_tw) != cudaSuccess) return GP_ERR_CUDA;
  if (cudaGetSymbolAddress((void**)&D.acc, g_na_acc) != cudaSuccess) return GP_ERR_CUDA;
  if (cudaGetSymbolAddress((void**)&D.part, g_na_part) != cudaSuccess) return GP_ERR_CUDA;
  if (cudaGetSymbolAddress((void**)&D.spec, g_na_spec) != cudaSuccess) return GP_ERR_CUDA;
  if (cudaGetSymbolAddress((void**)&D.flag, g_na_flag) != cudaSuccess) return GP_ERR_CUDA;
  float4 host[NOALLOC_TW];
  int used = 0;
  for (int q = 0; q < 7; ++q)
    for (int inv = 0; inv < 2; ++inv) {
      const int k = noalloc_twiddles(NOALLOC_SIZES[q], inv != 0, host + used, NOALLOC_TW - used);
      if (k < 0) return GP_ERR_CUDA;
      D.tw_off[q][inv] = used;
      used += k > 0 ? k : 1;   // keep distinct offsets even for single-pass lengths
    }
  if (cudaMemcpy(D.tw, host, sizeof(float4) * used, cudaMemcpyHostToDevice) != cudaSuccess) return GP_ERR_CUDA;
  (void)dev;
  D.ready = true;
  return GP_OK;
}

}  // namespace gp

extern "C" gp_status gp_diagnostics_noalloc(int n, double alpha, double beta, const void* psi, gp_diag* out,
                                            double* spectra, int nbins, void* cuda_stream) {
  using namespace gp;
  int q = -1;
  for (int i = 0; i < 7; ++i)
    if (NOALLOC_SIZES[i] == n) q = i;
  if (q < 0) return GP_ERR_UNSUPPORTED_SIZE;   // n > 64 or not a supported length
  if (!psi || ((uintptr_t)psi & 15) || !out || !std::isfinite(alpha) || !std::isfinite(beta))
    return GP_ERR_INVALID_ARG;
  const int nb = (int)std::floor(std::sqrt(3.0) * n / 2.0 + 0.5) + 1;
  if (spectra && nbins < nb) return GP_ERR_INVALID_ARG;
  // an error left pending by the caller's earlier work is reported, not consumed: the caller
  // still reads it with cudaGetLastError
  if (cudaPeekAtLastError() != cudaSuccess) return GP_ERR_CUDA;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return GP_ERR_CUDA;
  NoAllocDevice& D = g_na_dev[dev];
  if (!D.ready) {
    gp_status st = noalloc_setup(dev, D);
    if (st != GP_OK) return st;
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const long long npts = (long long)n * n * n;
  // a stack view of a plan field that points at the static tables (no allocation)
  FieldPlan F;
  F.n = n;
  F.npts = npts;
  F.alpha = alpha;
  F.beta = beta;
  F.t32.tw_fwd = D.tw + D.tw_off[q][0];
  F.t32.tw_inv = D.tw + D.tw_off[q][1];
  const cpx<float>* x = (const cpx<float>*)psi;
  cpx<float>* w0 = D.work;
  cpx<float>* w1 = w0 + npts;
  cpx<float>* w2 = w1 + npts;
  cpx<float>* w3 = w2 + npts;
  const unsigned g = rgrid(npts);
  if ((long long)g > NOALLOC_MAX_BLOCKS) return GP_ERR_UNSUPPORTED_SIZE;   // before any device work
  if (cudaMemsetAsync(D.acc, 0, DIAG_ACC * sizeof(double), s) != cudaSuccess) return GP_ERR_CUDA;
  if (cudaMemsetAsync(D.flag, 0, sizeof(int), s) != cudaSuccess) return GP_ERR_CUDA;
  if (cudaMemsetAsync(D.spec, 0, (size_t)4 * nb * sizeof(double), s) != cudaSuccess) return GP_ERR_CUDA;
  double* part = D.part;
  // every launch is checked at once (an error is then this call's own: a pending error of
  // earlier work was refused on entry)
  k_phys1<float><<<g, 256, 0, s>>>(x, npts, part, D.flag);
  if (cudaGetLastError() != cudaSuccess) return GP_ERR_CUDA;
  k_reduce<<<1, 256, 0, s>>>(part, (int)g, 2, D.acc);
  if (cudaGetLastError() != cudaSuccess) return GP_ERR_CUDA;
  if (cudaMemcpyAsync(w0, x, (size_t)npts * 8, cudaMemcpyDeviceToDevice, s) != cudaSuccess) return GP_ERR_CUDA;
  if (fft3<float>(F, w0, false, s) != cudaSuccess) return GP_ERR_CUDA;
  k_kspace1<float><<<g, 256, 0, s>>>(w0, w1, w2, w3, n, part + 2 * g);
  if (cudaGetLastError() != cudaSuccess) return GP_ERR_CUDA;
  k_reduce<<<1, 256, 0, s>>>(part + 2 * g, (int)g, 4, D.acc + 2);
  if (cudaGetLastError() != cudaSuccess) return GP_ERR_CUDA;
  if (fft3<float>(F, w1, true, s) != cudaSuccess || fft3<float>(F, w2, true, s) != cudaSuccess ||
      fft3<float>(F, w3, true, s) != cudaSuccess)
    return GP_ERR_CUDA;
  k_phys2<float><<<g, 256, 0, s>>>(x, w0, w1, w2, w3, npts, alpha, part + 6 * g, part + 8 * g);
  if (cudaGetLastError() != cudaSuccess) return GP_ERR_CUDA;
  k_reduce<<<1, 256, 0, s>>>(part + 6 * g, (int)g, 2, D.acc + 6);
  if (cudaGetLastError() != cudaSuccess) return GP_ERR_CUDA;
  k_reduce_max<<<1, 256, 0, s>>>(part + 8 * g, (int)g, D.acc + 8);
  if (cudaGetLastError() != cudaSuccess) return GP_ERR_CUDA;
  for (cpx<float>* w : {w0, w1, w2, w3})
    if (fft3<float>(F, w, false, s) != cudaSuccess) return GP_ERR_CUDA;
  k_kspace2<float><<<g, 256, (size_t)4 * nb * sizeof(double), s>>>(w0, w1, w2, w3, n, nb, alpha, beta, D.spec);
  if (cudaGetLastError() != cudaSuccess) return GP_ERR_CUDA;
  double acc[DIAG_ACC];
  double hs[4 * NOALLOC_MAX_BINS];
  int flag = 0;
  if (cudaMemcpyAsync(acc, D.acc, sizeof(acc), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(&flag, D.flag, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(hs, D.spec, (size_t)4 * nb * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return GP_ERR_CUDA;
  if (flag) return GP_ERR_NONFINITE;
  *out = diag_finish(acc, hs, nb, npts, alpha, beta);
  const double dn2 = (double)npts * (double)npts;
  if (spectra)
    for (int c = 0; c < 4; ++c)
      for (int b = 0; b < nb; ++b) spectra[c * nbins + b] = hs[(size_t)c * nb + b] / dn2;
  return GP_OK;
}

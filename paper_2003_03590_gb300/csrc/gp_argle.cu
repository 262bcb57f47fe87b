// gp_argle.cu -- imaginary-time (ARGLE) preparation and the Taylor-Green / ABC start fields.
//
// ARGLE (Sec. 4.2, eqn:gradient-flow): the gradient flow of the energy of a field driven by a
// divergence-free external velocity v (eq-energy-num-ext-vel), advanced by the semi-implicit
// backward-Euler step of eqn:semi-backward-Euler -- half of the Laplacian implicit, the rest
// explicit at the old level.  The implicit part is diagonal in Fourier space:
//   F phi' = [ (1 - a) F phi + dtau F(rest) ] / (1 + a),   a = dtau alpha |k|^2 / 2,
//   rest   = -i v . grad phi - |v|^2 / (4 alpha) phi + beta (1 - |phi|^2) phi.
// Per step: the field's spectrum F phi is kept from the previous step, so a step is three
// inverse transforms (grad phi, one launch per axis for the three components), one forward
// transform (rest) and one inverse (phi'), plus three pointwise kernels.  The velocity is
// evaluated from the grid coordinates inside the kernels (no velocity arrays).
// Optional L2 renormalisation (the normalised gradient flow): after each step phi and F phi
// are rescaled on the device to the mean |phi|^2 the field had on entry (float64 sums).
// E_v = < 2 alpha^2 |grad phi - i v phi / (2 alpha)|^2 + alpha beta (|phi|^2 - 1)^2 >.
//
// Start fields (generated in float64, rounded to the field's precision):
//   TG (Sec. 5.1): lambda = cos x sqrt(2|cos z|), mu = cos y sqrt(2|cos z|) sgn(cos z);
//     psi_e(l, m) = (l + i m) tanh(r / (sqrt2 xi)) / r; psi_4 = product of psi_e at
//     (lambda -+ 1/sqrt2, mu) and (lambda, mu -+ 1/sqrt2); psi = psi_4^m, m = floor(1/(2 pi alpha)).
//   ABC (Sec. 5.2): psi = prod over k = 1, 2 of exp(i [A sin kx/(2 alpha)] y + i [A cos kx/(2 alpha)] z)
//     and its two cyclic permutations (B: y, z, x; C: z, x, y), [.] the nearest integer.  The phase
//     is an integer combination of grid indices times 2 pi / N and is reduced modulo N exactly.
#include <cmath>

#include "gp_internal.h"
#include "gp_reduce.cuh"

namespace gp {

enum { FLOW_NONE = 0, FLOW_TG = 1, FLOW_ABC = 2 };

struct Flow {
  int kind;
  double A, B, C;
};

// Per-axis tables of the flows' trigonometric factors (x = 2 pi i / N), formed once per call in
// float64 with sincospi: [sin(2 pi i/N) | cos(2 pi i/N) | sin(4 pi i/N) |
// cos(4 pi i/N)], i = 0 .. N-1, in float64 (td) and rounded to float32 (tf).  The step kernels
// then read the velocity from them in the field's precision: GB300's float64 transcendentals
// made the per-point evaluation the largest part of an imaginary-time step.
__global__ void k_flow_tables(double* td, float* tf, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double inv = 2.0 / n;
  double s1, c1, s2, c2;
  sincospi(i * inv, &s1, &c1);
  sincospi((double)((2 * i) % n) * inv, &s2, &c2);
  const double v[4] = {s1, c1, s2, c2};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    td[q * n + i] = v[q];
    tf[q * n + i] = (float)v[q];
  }
}

// velocity at grid point (ix, iy, iz) from the tables, in the precision S of the tables
template <typename S>
__device__ __forceinline__ void flow_tab(const Flow& f, const S* __restrict__ tab, int ix, int iy, int iz, int n, S* v) {
  v[0] = v[1] = v[2] = S(0);
  if (f.kind == FLOW_NONE) return;
  const S* s1 = tab;
  const S* c1 = tab + n;
  if (f.kind == FLOW_TG) {
    const S cz = c1[iz];
    v[0] = s1[ix] * c1[iy] * cz;
    v[1] = -c1[ix] * s1[iy] * cz;
    return;
  }
  const S A = (S)f.A, B = (S)f.B, C = (S)f.C;
  S vx = S(0), vy = S(0), vz = S(0);
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const S* sk = tab + 2 * k * n;
    const S* ck = sk + n;
    vx += B * ck[iy] + C * sk[iz];
    vy += C * ck[iz] + A * sk[ix];
    vz += A * ck[ix] + B * sk[iy];
  }
  v[0] = vx;
  v[1] = vy;
  v[2] = vz;
}

__device__ __forceinline__ int kwave(int i, int n) { return i < (n + 1) / 2 ? i : i - n; }
__device__ __forceinline__ int kwave_d(int i, int n) { return (2 * i == n) ? 0 : kwave(i, n); }

// ---------------------------------------------------------------- start fields
__device__ __forceinline__ double2 psi_e(double l, double m, double xi) {
  const double r = sqrt(l * l + m * m);
  const double f = r > 0.0 ? tanh(r / (1.4142135623730951 * xi)) / r : 0.0;
  return double2{l * f, m * f};
}
__device__ __forceinline__ double2 zmul(double2 a, double2 b) { return double2{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }

template <typename T> __global__ void k_init_tg(cpx<T>* psi, int n, double xi, int m) {
  const long long npts = (long long)n * n * n;
  const double inv = 2.0 / n, h = 0.70710678118654752440;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npts; i += (long long)gridDim.x * blockDim.x) {
    const int ix = (int)(i % n), iy = (int)((i / n) % n), iz = (int)(i / ((long long)n * n));
    const double cz = cospi(iz * inv);
    const double s = sqrt(2.0 * fabs(cz));
    const double lam = cospi(ix * inv) * s;
    const double mu = cospi(iy * inv) * s * (cz > 0.0 ? 1.0 : (cz < 0.0 ? -1.0 : 0.0));
    const double2 p4 = zmul(zmul(psi_e(lam - h, mu, xi), psi_e(lam, mu - h, xi)),
                            zmul(psi_e(lam + h, mu, xi), psi_e(lam, mu + h, xi)));
    double2 r{1.0, 0.0};
    for (int q = 0; q < m; ++q) r = zmul(r, p4);
    psi[i] = cpx<T>{(T)r.x, (T)r.y};
  }
}

// nearest integer of a, halves away from zero; within 1e-9 of a half counts as the half (the
// default amplitudes hit exact halves on grids that contain 30 and 60 degrees)
__device__ __forceinline__ long long round_away(double a) {
  return (long long)(a < 0.0 ? -floor(-a + 0.5 + 1e-9) : floor(a + 0.5 + 1e-9));
}

template <typename T> __global__ void k_init_abc(cpx<T>* psi, int n, double alpha, double A, double B, double C) {
  const long long npts = (long long)n * n * n;
  const double inv = 2.0 / n, h = 1.0 / (2.0 * alpha);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npts; i += (long long)gridDim.x * blockDim.x) {
    const int ix = (int)(i % n), iy = (int)((i / n) % n), iz = (int)(i / ((long long)n * n));
    // phase = (2 pi / n) * M with the integer M = sum (integer coefficient) * (grid index)
    long long M = 0;
#pragma unroll
    for (int k = 1; k <= 2; ++k) {
      double sx, cx, sy, cy, sz, cz;
      sincospi((double)((k * ix) % n) * inv, &sx, &cx);
      sincospi((double)((k * iy) % n) * inv, &sy, &cy);
      sincospi((double)((k * iz) % n) * inv, &sz, &cz);
      M += round_away(A * sx * h) * iy + round_away(A * cx * h) * iz;   // psi_{A,k}^{x,y,z}
      M += round_away(B * sy * h) * iz + round_away(B * cy * h) * ix;   // psi_{B,k}^{y,z,x}
      M += round_away(C * sz * h) * ix + round_away(C * cz * h) * iy;   // psi_{C,k}^{z,x,y}
    }
    M %= n;
    if (M < 0) M += n;
    double s, c;
    sincospi((double)M * inv, &s, &c);
    psi[i] = cpx<T>{(T)c, (T)s};
  }
}

// ---------------------------------------------------------------- ARGLE step pieces
// w1..w3 = i k~_j * phi_hat (Nyquist-zeroed first-derivative wavenumbers)
template <typename T>
__global__ void k_grad_spec(const cpx<T>* ph, cpx<T>* w1, cpx<T>* w2, cpx<T>* w3, int n) {   // ph may be w1
  const long long npts = (long long)n * n * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npts; i += (long long)gridDim.x * blockDim.x) {
    const int ix = (int)(i % n), iy = (int)((i / n) % n), iz = (int)(i / ((long long)n * n));
    const cpx<T> a = ph[i];
    const T dx = (T)kwave_d(ix, n), dy = (T)kwave_d(iy, n), dz = (T)kwave_d(iz, n);
    w1[i] = cpx<T>{-dx * a.y, dx * a.x};
    w2[i] = cpx<T>{-dy * a.y, dy * a.x};
    w3[i] = cpx<T>{-dz * a.y, dz * a.x};
  }
}

// w1 = rest(phi, grad phi) in place of grad_x
template <typename T>
__global__ void k_argle_rest(const cpx<T>* __restrict__ phi, cpx<T>* w1, const cpx<T>* __restrict__ w2,
                             const cpx<T>* __restrict__ w3, int n, Flow f, const T* __restrict__ tab, double alpha,
                             double beta) {
  const long long npts = (long long)n * n * n;
  const T q = (T)(1.0 / (4.0 * alpha)), bt = (T)beta;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npts; i += (long long)gridDim.x * blockDim.x) {
    const int ix = (int)(i % n), iy = (int)((i / n) % n), iz = (int)(i / ((long long)n * n));
    T v[3];
    flow_tab<T>(f, tab, ix, iy, iz, n, v);
    const cpx<T> p = phi[i], gx = w1[i], gy = w2[i], gz = w3[i];
    // v . grad phi
    const T dr = v[0] * gx.x + v[1] * gy.x + v[2] * gz.x;
    const T di = v[0] * gx.y + v[1] * gy.y + v[2] * gz.y;
    const T c = bt * (T(1) - (p.x * p.x + p.y * p.y)) - q * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    // -i (dr + i di) + c p
    w1[i] = cpx<T>{di + c * p.x, -dr + c * p.y};
  }
}

// ph <- [(1 - a) ph + dtau * fr] / (1 + a), a = dtau alpha |k|^2 / 2; phi <- the same (for the inverse)
template <typename T>
__global__ void k_argle_combine(cpx<T>* ph, const cpx<T>* __restrict__ fr, cpx<T>* phi, int n, double dtau, double alpha) {
  const long long npts = (long long)n * n * n;
  const T hd = (T)(0.5 * dtau * alpha), dt = (T)dtau;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npts; i += (long long)gridDim.x * blockDim.x) {
    const int ix = (int)(i % n), iy = (int)((i / n) % n), iz = (int)(i / ((long long)n * n));
    const int kx = kwave(ix, n), ky = kwave(iy, n), kz = kwave(iz, n);
    // in the field's precision (float64 division per point is slow on GB300)
    const T a = hd * (T)(kx * kx + ky * ky + kz * kz);
    const T num = T(1) - a, den = T(1) / (T(1) + a);
    const cpx<T> x = ph[i], r = fr[i];
    const cpx<T> y{(num * x.x + dt * r.x) * den, (num * x.y + dt * r.y) * den};
    ph[i] = y;
    phi[i] = y;
  }
}

// per-block sums of |phi|^2
template <typename T> __global__ void k_mass(const cpx<T>* __restrict__ phi, long long npts, double* part) {
  Sums<T, 1> S;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npts; i += (long long)gridDim.x * blockDim.x) {
    const cpx<T> a = phi[i];
    const T v[1] = {a.x * a.x + a.y * a.y};
    S.add(v);
  }
  S.flush();
  block_store<1>(S.d, part);
}

// phi and ph *= sqrt(target / mass), mass = acc[0] / npts (on the device: no host round trip)
template <typename T>
__global__ void k_rescale(cpx<T>* phi, cpx<T>* ph, long long npts, const double* acc, const double* target) {
  const double m = acc[0] / (double)npts;
  const T s = (T)(m > 0.0 ? sqrt(*target / m) : 1.0);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npts; i += (long long)gridDim.x * blockDim.x) {
    const cpx<T> a = phi[i], b = ph[i];
    phi[i] = cpx<T>{a.x * s, a.y * s};
    ph[i] = cpx<T>{b.x * s, b.y * s};
  }
}

// per-block sums of |grad phi - i v phi / (2 alpha)|^2 and (|phi|^2 - 1)^2
template <typename T>
__global__ void k_energy_v(const cpx<T>* __restrict__ phi, const cpx<T>* __restrict__ w1, const cpx<T>* __restrict__ w2,
                           const cpx<T>* __restrict__ w3, int n, Flow f, const T* __restrict__ tab, double alpha,
                           double* part) {
  const long long npts = (long long)n * n * n;
  Sums<T, 2> S;
  const T h = (T)(1.0 / (2.0 * alpha));
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npts; i += (long long)gridDim.x * blockDim.x) {
    const int ix = (int)(i % n), iy = (int)((i / n) % n), iz = (int)(i / ((long long)n * n));
    T v[3];
    flow_tab<T>(f, tab, ix, iy, iz, n, v);
    const cpx<T> p = phi[i];
    const cpx<T> g[3] = {w1[i], w2[i], w3[i]};
    T t = 0;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      // g - i (v h) p
      const T re = g[j].x + v[j] * h * p.y, im = g[j].y - v[j] * h * p.x;
      t += re * re + im * im;
    }
    T rho;
    const T r = rho_minus_one(p, &rho);
    const T val[2] = {t, r * r};
    S.add(val);
  }
  S.flush();
  block_store<2>(S.d, part);
}

static inline unsigned agrid(long long n) {
  long long b = (n + 255) / 256;
  return (unsigned)(b < 1 ? 1 : (b > 152LL * 16 ? 152LL * 16 : b));
}

template <typename T> static cudaError_t transform(gp_plan* p, FieldPlan& F, cpx<T>** xs, int count, bool inverse,
                                                   cudaStream_t s) {
  if constexpr (sizeof(T) == 4) return fft3_many(p, F, xs, count, inverse, s);
  for (int k = 0; k < count; ++k) {
    cudaError_t e = fft3<T>(F, xs[k], inverse, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// per-block maxima of |phi - old|^2 (a maximum is exact in any precision)
template <typename T>
__global__ void k_maxdiff2(const cpx<T>* __restrict__ phi, const cpx<T>* __restrict__ old, long long npts, double* part) {
  T m = T(0);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npts; i += (long long)gridDim.x * blockDim.x) {
    const cpx<T> a = phi[i], b = old[i];
    const T dx = a.x - b.x, dy = a.y - b.y, d2 = dx * dx + dy * dy;
    m = d2 > m ? d2 : m;
  }
  double md = (double)m;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) md = fmax(md, __shfl_xor_sync(0xffffffffu, md, o));
  __shared__ double red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = md;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 1; q < (int)(blockDim.x >> 5); ++q) md = fmax(md, red[q]);
    part[blockIdx.x] = md;
  }
}

// Convergence checks of a run (eqn:crit1, eqn:crit2): every `every`-th step and the last one
// evaluate ||phi^{n+1} - phi^n||_inf / dtau and |E_v(phi^{n+1}) - E_v(phi^n)| / (dtau E_v(phi^n));
// the run stops after the first checked step with crit1 <= eps (eps <= 0: never).
struct ArgleCheck {
  int every = 0;   // 0: no checks
  double eps = 0.0;
  int* steps_done = nullptr;
  double* crit1 = nullptr;
  double* crit2 = nullptr;
};

template <typename T>
static gp_status argle_impl(gp_plan* p, int field, cpx<T>* phi, Flow flow, double dtau, int nsteps, int renorm,
                            double* energy_out, const ArgleCheck& chk = ArgleCheck()) {
  FieldPlan& F = p->f[field];
  const int n = F.n;
  const long long npts = F.npts;
  const size_t fb = (size_t)npts * sizeof(cpx<T>);
  const unsigned g = agrid(npts);
  const int nf = chk.every > 0 ? 5 : 4;
  gp_status st = ensure_ws(p, field, nf * fb + (size_t)(2 * g + 16 + 4 * n) * sizeof(double) + (size_t)4 * n * sizeof(float));
  if (st != GP_OK) return st;
  cpx<T>* ph = (cpx<T>*)F.ws;
  cpx<T>* w1 = ph + npts;
  cpx<T>* w2 = w1 + npts;
  cpx<T>* w3 = w2 + npts;
  cpx<T>* old = w3 + npts;                       // the field before a checked step
  double* part = (double*)(ph + (size_t)nf * npts);
  // red: [0] mass sum, [1] target mean |phi|^2, [2..3] energy sums, [4..5] E_v sums before and
  // [6..7] after a checked step, [8] max |phi^{n+1} - phi^n|^2
  double* red = part + 2 * g;
  double* tab_d = red + 16;                      // flow tables, float64 and float32
  float* tab_f = (float*)(tab_d + 4 * n);
  const T* tab = (const T*)(sizeof(T) == 8 ? (const void*)tab_d : (const void*)tab_f);
  cudaStream_t s = p->stream;
  k_flow_tables<<<(n + 127) / 128, 128, 0, s>>>(tab_d, tab_f, n);
  GP_CUDA(p, cudaGetLastError());
  const double alpha = F.alpha, beta = F.beta, dn = (double)npts;
  cpx<T>* grads[3] = {w1, w2, w3};
  // E_v sums of the current phi into dst[0..1] (enqueued only; uses w1..w3)
  auto energy_sums = [&](double* dst) -> gp_status {
    GP_CUDA(p, cudaMemcpyAsync(w1, phi, fb, cudaMemcpyDeviceToDevice, s));
    GP_CUDA(p, transform<T>(p, F, &w1, 1, false, s));
    k_grad_spec<T><<<g, 256, 0, s>>>(w1, w1, w2, w3, n);   // in place: w1 is read before it is written
    GP_CUDA(p, cudaGetLastError());
    GP_CUDA(p, transform<T>(p, F, grads, 3, true, s));
    k_energy_v<T><<<g, 256, 0, s>>>(phi, w1, w2, w3, n, flow, tab, alpha, part);
    k_reduce<<<1, 256, 0, s>>>(part, (int)g, 2, dst);
    GP_CUDA(p, cudaGetLastError());
    return GP_OK;
  };
  auto energy_of = [&](const double* e) { return 2.0 * alpha * alpha * e[0] / dn + alpha * beta * e[1] / dn; };
  if (chk.every > 0) {
    *chk.steps_done = 0;
    *chk.crit1 = *chk.crit2 = std::nan("");
  }
  if (nsteps > 0) {
    if (renorm) {
      k_mass<T><<<g, 256, 0, s>>>(phi, npts, part);
      k_reduce<<<1, 256, 0, s>>>(part, (int)g, 1, red);
      k_scale_to_mean<<<1, 1, 0, s>>>(red, red + 1, (double)npts);
      GP_CUDA(p, cudaGetLastError());
    }
    GP_CUDA(p, cudaMemcpyAsync(ph, phi, fb, cudaMemcpyDeviceToDevice, s));
    GP_CUDA(p, transform<T>(p, F, &ph, 1, false, s));
    for (int it = 0; it < nsteps; ++it) {
      const bool check = chk.every > 0 && ((it + 1) % chk.every == 0 || it + 1 == nsteps);
      if (check) {
        GP_CUDA(p, cudaMemcpyAsync(old, phi, fb, cudaMemcpyDeviceToDevice, s));
        st = energy_sums(red + 4);
        if (st != GP_OK) return st;
      }
      k_grad_spec<T><<<g, 256, 0, s>>>(ph, w1, w2, w3, n);
      GP_CUDA(p, cudaGetLastError());
      GP_CUDA(p, transform<T>(p, F, grads, 3, true, s));
      k_argle_rest<T><<<g, 256, 0, s>>>(phi, w1, w2, w3, n, flow, tab, alpha, beta);
      GP_CUDA(p, cudaGetLastError());
      GP_CUDA(p, transform<T>(p, F, &w1, 1, false, s));
      k_argle_combine<T><<<g, 256, 0, s>>>(ph, w1, phi, n, dtau, alpha);
      GP_CUDA(p, cudaGetLastError());
      GP_CUDA(p, transform<T>(p, F, &phi, 1, true, s));
      if (renorm) {
        k_mass<T><<<g, 256, 0, s>>>(phi, npts, part);
        k_reduce<<<1, 256, 0, s>>>(part, (int)g, 1, red);
        k_rescale<T><<<g, 256, 0, s>>>(phi, ph, npts, red, red + 1);
        GP_CUDA(p, cudaGetLastError());
      }
      if (check) {
        k_maxdiff2<T><<<g, 256, 0, s>>>(phi, old, npts, part + g);
        k_reduce_max<<<1, 256, 0, s>>>(part + g, (int)g, red + 8);
        GP_CUDA(p, cudaGetLastError());
        st = energy_sums(red + 6);
        if (st != GP_OK) return st;
        double h[5];
        GP_CUDA(p, cudaMemcpyAsync(h, red + 4, sizeof(h), cudaMemcpyDeviceToHost, s));
        GP_CUDA(p, cudaStreamSynchronize(s));
        st = check_status(p);
        if (st != GP_OK) return st;
        const double e_old = energy_of(h), e_new = energy_of(h + 2);
        *chk.steps_done = it + 1;
        *chk.crit1 = std::sqrt(h[4]) / dtau;
        *chk.crit2 = std::fabs(e_new - e_old) / (dtau * e_old);
        if (!std::isfinite(*chk.crit1) || !std::isfinite(e_new))
          return fail(p, GP_ERR_NONFINITE, "gp_argle_converge: the field is not finite");
        if (chk.eps > 0.0 && *chk.crit1 <= chk.eps) break;
      }
    }
  }
  if (!energy_out) return GP_OK;
  st = energy_sums(red + 2);
  if (st != GP_OK) return st;
  double e[2];
  GP_CUDA(p, cudaMemcpyAsync(e, red + 2, sizeof(e), cudaMemcpyDeviceToHost, s));
  GP_CUDA(p, cudaStreamSynchronize(s));
  {
    gp_status cs = check_status(p);
    if (cs != GP_OK) return cs;
  }
  *energy_out = energy_of(e);
  if (!std::isfinite(*energy_out)) return fail(p, GP_ERR_NONFINITE, "gp_argle: energy is not finite");
  return GP_OK;
}

static bool flow_of(int kind, const double* abc, Flow* f) {
  if (kind < FLOW_NONE || kind > FLOW_ABC) return false;
  f->kind = kind;
  f->A = abc ? abc[0] : 0.9 / std::sqrt(3.0);
  f->B = abc ? abc[1] : 1.0 / std::sqrt(3.0);
  f->C = abc ? abc[2] : 1.1 / std::sqrt(3.0);
  return std::isfinite(f->A) && std::isfinite(f->B) && std::isfinite(f->C);
}

}  // namespace gp

using namespace gp;

extern "C" {

gp_status gp_init_tg(gp_plan* p, int field, void* psi) {
  if (!p) return GP_ERR_INVALID_ARG;
  if (field < 0 || field >= (int)p->f.size()) return fail(p, GP_ERR_INVALID_ARG, "gp_init_tg: field index");
  if (!psi || ((uintptr_t)psi & 15)) return fail(p, GP_ERR_INVALID_ARG, "gp_init_tg: pointer");
  FieldPlan& F = p->f[field];
  const int m = (int)std::floor(1.0 / (2.0 * M_PI * F.alpha));
  if (m < 1 || m > 4096) return fail(p, GP_ERR_INVALID_ARG, "gp_init_tg: [1/(2 pi alpha)] must be between 1 and 4096");
  const double xi = std::sqrt(F.alpha / F.beta);
  if (F.fp64) k_init_tg<double><<<agrid(F.npts), 256, 0, p->stream>>>((cpx<double>*)psi, F.n, xi, m);
  else k_init_tg<float><<<agrid(F.npts), 256, 0, p->stream>>>((cpx<float>*)psi, F.n, xi, m);
  GP_CUDA(p, cudaGetLastError());
  return GP_OK;
}

gp_status gp_init_abc(gp_plan* p, int field, void* psi, const double* abc) {
  if (!p) return GP_ERR_INVALID_ARG;
  if (field < 0 || field >= (int)p->f.size()) return fail(p, GP_ERR_INVALID_ARG, "gp_init_abc: field index");
  if (!psi || ((uintptr_t)psi & 15)) return fail(p, GP_ERR_INVALID_ARG, "gp_init_abc: pointer");
  Flow f;
  if (!flow_of(FLOW_ABC, abc, &f)) return fail(p, GP_ERR_INVALID_ARG, "gp_init_abc: amplitudes");
  FieldPlan& F = p->f[field];
  if (F.fp64) k_init_abc<double><<<agrid(F.npts), 256, 0, p->stream>>>((cpx<double>*)psi, F.n, F.alpha, f.A, f.B, f.C);
  else k_init_abc<float><<<agrid(F.npts), 256, 0, p->stream>>>((cpx<float>*)psi, F.n, F.alpha, f.A, f.B, f.C);
  GP_CUDA(p, cudaGetLastError());
  return GP_OK;
}

gp_status gp_argle(gp_plan* p, int field, void* psi, int flow, const double* abc, double dtau, int nsteps, int renorm,
                   double* energy_out) {
  if (!p) return GP_ERR_INVALID_ARG;
  if (field < 0 || field >= (int)p->f.size()) return fail(p, GP_ERR_INVALID_ARG, "gp_argle: field index");
  if (!psi || ((uintptr_t)psi & 15)) return fail(p, GP_ERR_INVALID_ARG, "gp_argle: pointer");
  if (nsteps < 0 || !(dtau > 0.0) || !std::isfinite(dtau) || (renorm != 0 && renorm != 1))
    return fail(p, GP_ERR_INVALID_ARG, "gp_argle: nsteps >= 0, dtau > 0, renorm 0 or 1");
  Flow f;
  if (!flow_of(flow, abc, &f)) return fail(p, GP_ERR_INVALID_ARG, "gp_argle: flow must be 0 (none), 1 (TG) or 2 (ABC)");
  FieldPlan& F = p->f[field];
  if (F.fp64) return argle_impl<double>(p, field, (cpx<double>*)psi, f, dtau, nsteps, renorm, energy_out);
  return argle_impl<float>(p, field, (cpx<float>*)psi, f, dtau, nsteps, renorm, energy_out);
}

gp_status gp_argle_converge(gp_plan* p, int field, void* psi, int flow, const double* abc, double dtau, int max_steps,
                            int renorm, double eps, int check_every, int* steps_done, double* crit1, double* crit2,
                            double* energy_out) {
  if (!p) return GP_ERR_INVALID_ARG;
  if (field < 0 || field >= (int)p->f.size()) return fail(p, GP_ERR_INVALID_ARG, "gp_argle_converge: field index");
  if (!psi || ((uintptr_t)psi & 15) || !steps_done || !crit1 || !crit2)
    return fail(p, GP_ERR_INVALID_ARG, "gp_argle_converge: pointer");
  if (max_steps < 1 || check_every < 1 || !(dtau > 0.0) || !std::isfinite(dtau) || !std::isfinite(eps) ||
      (renorm != 0 && renorm != 1))
    return fail(p, GP_ERR_INVALID_ARG, "gp_argle_converge: max_steps >= 1, check_every >= 1, dtau > 0, renorm 0 or 1");
  Flow f;
  if (!flow_of(flow, abc, &f))
    return fail(p, GP_ERR_INVALID_ARG, "gp_argle_converge: flow must be 0 (none), 1 (TG) or 2 (ABC)");
  ArgleCheck chk;
  chk.every = check_every;
  chk.eps = eps;
  chk.steps_done = steps_done;
  chk.crit1 = crit1;
  chk.crit2 = crit2;
  FieldPlan& F = p->f[field];
  if (F.fp64) return argle_impl<double>(p, field, (cpx<double>*)psi, f, dtau, max_steps, renorm, energy_out, chk);
  return argle_impl<float>(p, field, (cpx<float>*)psi, f, dtau, max_steps, renorm, energy_out, chk);
}

}  // extern "C"

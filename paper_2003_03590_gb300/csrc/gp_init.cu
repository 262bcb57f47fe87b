// gp_init.cu -- initial conditions of Sec. 5.3 (smoothed random phase) and Sec. 5.4 (random
// vortex rings), generated in float64 and rounded to the field's storage type.
//
// Random numbers: SplitMix64 (Steele, Lea & Flood 2014) used as a counter-based stream:
// position c outputs mix((c + 1) * 0x9E3779B97F4A7C15), mix = the SplitMix64 finaliser;
// a run with seed s reads positions s * 2^40 + i.  Uniforms u = (v >> 11) 2^-53 in [0, 1),
// u1 = ((v >> 11) + 1) 2^-53 in (0, 1]; normals by Box-Muller.
//   SRP spectral  point i: positions 2i, 2i+1 -> sqrt(-2 ln u1) cos(2 pi u)
//   SRP spline    lattice (i, j, k): position (k N_r + j) N_r + i -> K (2u - 1)
//   RVR rings     ring j: positions 8j..8j+7 -> R, centre x/y/z, normal from two Box-Muller pairs
//   RVR pairs     pair p: positions 4p..4p+3 -> shift X, Y, Z (2 pi u) and axis order floor(6u)
#include <cmath>
#include <cstring>
#include <vector>

#include "gp_internal.h"

namespace gp {

__host__ __device__ __forceinline__ uint64_t splitmix_at(uint64_t c) {
  uint64_t z = (c + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__host__ __device__ __forceinline__ double u01(uint64_t v) { return (double)(v >> 11) * 0x1.0p-53; }
__host__ __device__ __forceinline__ double u01_open0(uint64_t v) { return ((double)(v >> 11) + 1.0) * 0x1.0p-53; }
static inline uint64_t stream_pos(uint64_t seed, uint64_t i) { return seed * (1ull << 40) + i; }

__device__ __forceinline__ int kwave(int i, int n) { return i < (n + 1) / 2 ? i : i - n; }
__device__ __forceinline__ int kwave_d(int i, int n) { return (2 * i == n) ? 0 : kwave(i, n); }

static inline unsigned igrid(long long n) {
  long long b = (n + 255) / 256;
  return (unsigned)(b < 1 ? 1 : (b > 152LL * 32 ? 152LL * 32 : b));
}

// ---------------------------------------------------------------- SRP, spectral
__global__ void k_noise(double2* w, long long npts, uint64_t base) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npts; i += (long long)gridDim.x * blockDim.x) {
    const uint64_t a = splitmix_at(base + 2ull * (uint64_t)i), b = splitmix_at(base + 2ull * (uint64_t)i + 1ull);
    const double r = sqrt(-2.0 * log(u01_open0(a)));
    w[i] = make_double2(r * cospi(2.0 * u01(b)), 0.0);
  }
}

__global__ void k_srp_filter(double2* w, int n, double inv_k02) {
  const long long npts = (long long)n * n * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npts; i += (long long)gridDim.x * blockDim.x) {
    const int ix = (int)(i % n), iy = (int)((i / n) % n), iz = (int)(i / ((long long)n * n));
    const double kx = kwave(ix, n), ky = kwave(iy, n), kz = kwave(iz, n);
    const double f = (i == 0) ? 0.0 : exp(-(kx * kx + ky * ky + kz * kz) * inv_k02);
    w[i] = make_double2(w[i].x * f, w[i].y * f);
  }
}

// Sum of Re(w)^2 as SUM_BLOCKS partial sums, each formed in a fixed order (a thread's strided
// elements in turn, a warp's tree, the block's warps in turn); the host adds the partials in
// order.  The total does not depend on scheduling, so a seed always gives the same field.
constexpr int SUM_BLOCKS = 64, SUM_THREADS = 1024;
__global__ void __launch_bounds__(SUM_THREADS) k_sum_re2(const double2* w, long long npts, double* part) {
  __shared__ double wsum[SUM_THREADS / 32];
  double v = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npts; i += (long long)gridDim.x * blockDim.x)
    v = fma(w[i].x, w[i].x, v);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < SUM_THREADS / 32; ++q) t += wsum[q];
    part[blockIdx.x] = t;
  }
}

template <typename T> __global__ void k_phase_out(const double2* w, cpx<T>* psi, long long npts, double scale) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npts; i += (long long)gridDim.x * blockDim.x) {
    double sn, cs;
    sincos(w[i].x * scale, &sn, &cs);
    psi[i] = cpx<T>{(T)cs, (T)sn};
  }
}

template <typename T> __global__ void k_copy_out(const double2* w, cpx<T>* psi, long long npts) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npts; i += (long long)gridDim.x * blockDim.x)
    psi[i] = cpx<T>{(T)w[i].x, (T)w[i].y};
}

// ---------------------------------------------------------------- SRP, spline
// theta(x, y, z) = sum_{k,j,i} S[z][k] S[y][j] S[x][i] lat[k][j][i] with S the N x N_r matrix of
// the periodic cubic spline (the paper's sequential x, y, z interpolation is this tensor product).
// The interpolation is separable: theta(ix, iy, iz) = sum_k S[iz][k] sum_j S[iy][j] sum_q S[ix][q]
// lat[k][j][q].  The two inner sums are formed once on their own grids (nr^2 x N, then nr x N^2
// values) and every point only does the outer one; each sum runs over the same terms in the same
// order as written, so the values are those of the direct triple sum.
__global__ void k_spline_x(const double* __restrict__ S, const double* __restrict__ lat, int n, int nr, double* T1) {
  const long long total = (long long)nr * nr * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const int ix = (int)(i % n);
    const long long kj = i / n;                     // k nr + j
    double tx = 0.0;
    for (int q = 0; q < nr; ++q) tx += S[(long long)ix * nr + q] * lat[kj * nr + q];
    T1[i] = tx;                                     // [k][j][ix]
  }
}
__global__ void k_spline_y(const double* __restrict__ S, const double* __restrict__ T1, int n, int nr, double* T2) {
  const long long total = (long long)nr * n * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const int ix = (int)(i % n);
    const int iy = (int)((i / n) % n);
    const int k = (int)(i / ((long long)n * n));
    double ty = 0.0;
    for (int j = 0; j < nr; ++j) ty += S[(long long)iy * nr + j] * T1[((long long)k * nr + j) * n + ix];
    T2[i] = ty;                                     // [k][iy][ix]
  }
}
template <typename T>
__global__ void k_spline(const double* __restrict__ S, const double* __restrict__ T2, int n, int nr, cpx<T>* psi) {
  const long long npts = (long long)n * n * n, nn = (long long)n * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npts; i += (long long)gridDim.x * blockDim.x) {
    const long long iyx = i % nn;
    const int iz = (int)(i / nn);
    double th = 0.0;
    for (int k = 0; k < nr; ++k) th += S[(long long)iz * nr + k] * T2[(long long)k * nn + iyx];
    double sn, cs;
    sincos(th, &sn, &cs);
    psi[i] = cpx<T>{(T)cs, (T)sn};
  }
}

// periodic uniform cubic spline through nr nodes spaced ns apart: fine sample x = ns r + s is
// A y_r + B y_{r+1} + C M_r + D M_{r+1}, A = (ns - s)/ns, B = s/ns, C = (A^3 - A) ns^2 / 6,
// D = (B^3 - B) ns^2 / 6, with M solving M_{r-1} + 4 M_r + M_{r+1} = 6 (y_{r-1} - 2 y_r + y_{r+1}) / ns^2.
// Returns the n x nr matrix of that linear map.
static std::vector<double> spline_matrix(int n, int nr) {
  const int ns = n / nr;
  // inverse of the cyclic matrix tridiag(1, 4, 1) by Gauss-Jordan elimination
  std::vector<double> A((size_t)nr * nr, 0.0), Inv((size_t)nr * nr, 0.0);
  for (int r = 0; r < nr; ++r) {
    A[(size_t)r * nr + r] += 4.0;
    A[(size_t)r * nr + (r + nr - 1) % nr] += 1.0;
    A[(size_t)r * nr + (r + 1) % nr] += 1.0;
    Inv[(size_t)r * nr + r] = 1.0;
  }
  for (int c = 0; c < nr; ++c) {
    int piv = c;
    for (int r = c + 1; r < nr; ++r)
      if (std::fabs(A[(size_t)r * nr + c]) > std::fabs(A[(size_t)piv * nr + c])) piv = r;
    for (int q = 0; q < nr; ++q) {
      std::swap(A[(size_t)c * nr + q], A[(size_t)piv * nr + q]);
      std::swap(Inv[(size_t)c * nr + q], Inv[(size_t)piv * nr + q]);
    }
    const double d = A[(size_t)c * nr + c];
    for (int q = 0; q < nr; ++q) {
      A[(size_t)c * nr + q] /= d;
      Inv[(size_t)c * nr + q] /= d;
    }
    for (int r = 0; r < nr; ++r)
      if (r != c) {
        const double f = A[(size_t)r * nr + c];
        if (f == 0.0) continue;
        for (int q = 0; q < nr; ++q) {
          A[(size_t)r * nr + q] -= f * A[(size_t)c * nr + q];
          Inv[(size_t)r * nr + q] -= f * Inv[(size_t)c * nr + q];
        }
      }
  }
  // G = Inv * D2 with (D2 y)_r = 6 (y_{r-1} - 2 y_r + y_{r+1}) / ns^2 maps node values to M
  std::vector<double> G((size_t)nr * nr, 0.0);
  const double c6 = 6.0 / ((double)ns * ns);
  for (int r = 0; r < nr; ++r)
    for (int q = 0; q < nr; ++q) {
      double g = 0.0;
      for (int t = 0; t < nr; ++t) {
        double d2 = 0.0;
        if (q == (t + nr - 1) % nr) d2 += c6;
        if (q == t) d2 -= 2.0 * c6;
        if (q == (t + 1) % nr) d2 += c6;
        g += Inv[(size_t)r * nr + t] * d2;
      }
      G[(size_t)r * nr + q] = g;
    }
  std::vector<double> S((size_t)n * nr, 0.0);
  for (int r = 0; r < nr; ++r)
    for (int s = 0; s < ns; ++s) {
      const double a = (double)(ns - s) / ns, b = (double)s / ns;
      const double cc = (a * a * a - a) * ns * ns / 6.0, dd = (b * b * b - b) * ns * ns / 6.0;
      const int x = ns * r + s, r1 = (r + 1) % nr;
      double* row = &S[(size_t)x * nr];
      row[r] += a;
      row[r1] += b;
      for (int q = 0; q < nr; ++q) row[q] += cc * G[(size_t)r * nr + q] + dd * G[(size_t)r1 * nr + q];
    }
  return S;
}

// ---------------------------------------------------------------- RVR, rings
struct Ring {
  double R, cx, cy, cz, nx, ny, nz;
};

template <typename T>
__global__ void k_rings(const Ring* __restrict__ rings, int count, int n, double xi, cpx<T>* psi) {
  const long long npts = (long long)n * n * n;
  const double dx = 2.0 * M_PI / n, two_pi = 2.0 * M_PI, inv = 1.0 / (sqrt(2.0) * xi);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npts; i += (long long)gridDim.x * blockDim.x) {
    const int ix = (int)(i % n), iy = (int)((i / n) % n), iz = (int)(i / ((long long)n * n));
    const double x = ix * dx, y = iy * dx, z = iz * dx;
    double re = 1.0, im = 0.0;
    for (int j = 0; j < count; ++j) {
      const Ring g = rings[j];
      double d0 = x - g.cx, d1 = y - g.cy, d2 = z - g.cz;
      d0 -= two_pi * floor((d0 + M_PI) / two_pi);
      d1 -= two_pi * floor((d1 + M_PI) / two_pi);
      d2 -= two_pi * floor((d2 + M_PI) / two_pi);
      const double zp = d0 * g.nx + d1 * g.ny + d2 * g.nz;
      const double p0 = d0 - zp * g.nx, p1 = d1 - zp * g.ny, p2 = d2 - zp * g.nz;
      const double rp = sqrt(p0 * p0 + p1 * p1 + p2 * p2);
      const double s = sqrt((rp - g.R) * (rp - g.R) + zp * zp);
      // tanh(s / (sqrt 2 xi)) exp(i atan2(z', rho' - R)) = tanh(.) (rho' - R + i z') / s: the
      // phase factor is the unit vector of the core offset (no float64 atan2 and sincos, which
      // are slow on GB300); at s = 0 the amplitude is 0
      // (beyond 22 core widths tanh is 1 to far below an ulp: skip the float64 tanh there)
      const double sa = s * inv;
      const double f = s > 0.0 ? (sa < 22.0 ? tanh(sa) : 1.0) / s : 0.0;
      const double fr = f * (rp - g.R), fi = f * zp;
      const double nr = re * fr - im * fi, ni = re * fi + im * fr;
      re = nr;
      im = ni;
    }
    psi[i] = cpx<T>{(T)re, (T)im};
  }
}

// ---------------------------------------------------------------- RVR, Pade pairs
__device__ __forceinline__ double2 vring(double x, double y, double z, double R, double xi) {
  const double a1 = (73.0 + 3.0 * sqrt(201.0)) / 352.0, a2 = (6.0 + sqrt(201.0)) / 528.0,
               b1 = (21.0 + sqrt(201.0)) / 96.0;
  const double xt = x - M_PI, yt = y - M_PI, zt = z - M_PI;
  const double r = sqrt(xt * xt + yt * yt);
  const double d = sqrt((r - R) * (r - R) + zt * zt);
  const double e2 = (d / xi) * (d / xi);
  const double f = sqrt((a1 * e2 + a2 * e2 * e2) / (1.0 + b1 * e2 + a2 * e2 * e2));
  // f exp(i atan2(z~, r - R)) = f (r - R + i z~) / d (the amplitude vanishes at d = 0)
  const double q = d > 0.0 ? f / d : 0.0;
  return make_double2(q * (r - R), q * zt);
}
__device__ __forceinline__ double2 dmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 dconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 vpair(double x, double y, double z, double R, double d, double xi) {
  return dmul(vring(x, y, z - 0.5 * d, R, xi), dconj(vring(x, y, z + 0.5 * d, R, xi)));
}

__global__ void k_pair_base(double2* w, int n, double R, double d, double xi) {
  const long long npts = (long long)n * n * n;
  const double dx = 2.0 * M_PI / n, L = 2.0 * M_PI;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npts; i += (long long)gridDim.x * blockDim.x) {
    const int ix = (int)(i % n), iy = (int)((i / n) % n), iz = (int)(i / ((long long)n * n));
    const double x = ix * dx, y = iy * dx, z = iz * dx;
    double2 v = vpair(x, y, z, R, d, xi);
    v = dmul(v, dconj(vpair(2 * L - x, y, z, R, d, xi)));
    v = dmul(v, dconj(vpair(-x, y, z, R, d, xi)));
    v = dmul(v, dconj(vpair(x, 2 * L - y, z, R, d, xi)));
    v = dmul(v, dconj(vpair(x, -y, z, R, d, xi)));
    v = dmul(v, dconj(vpair(x, y, 2 * L - z, R, d, xi)));
    v = dmul(v, dconj(vpair(x, y, -z, R, d, xi)));
    w[i] = v;
  }
}

// T_k = W_k exp(i k~ . X): after the inverse transform T(x) = W(x + X)
__global__ void k_shift(const double2* __restrict__ w, double2* t, int n, double X, double Y, double Z) {
  const long long npts = (long long)n * n * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npts; i += (long long)gridDim.x * blockDim.x) {
    const int ix = (int)(i % n), iy = (int)((i / n) % n), iz = (int)(i / ((long long)n * n));
    const double ph = kwave_d(ix, n) * X + kwave_d(iy, n) * Y + kwave_d(iz, n) * Z;
    double sn, cs;
    sincos(ph, &sn, &cs);
    t[i] = dmul(w[i], make_double2(cs, sn));
  }
}

// A(x, y, z) *= T(a0, a1, a2) with (a0, a1, a2) the (x, y, z) indices in the chosen axis order
__global__ void k_accum_perm(double2* acc, const double2* __restrict__ t, int n, int o0, int o1, int o2) {
  const long long npts = (long long)n * n * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npts; i += (long long)gridDim.x * blockDim.x) {
    const int c[3] = {(int)(i % n), (int)((i / n) % n), (int)(i / ((long long)n * n))};
    const long long src = ((long long)c[o2] * n + c[o1]) * n + c[o0];
    acc[i] = dmul(acc[i], t[src]);
  }
}

__global__ void k_fill_one(double2* a, long long npts) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npts; i += (long long)gridDim.x * blockDim.x)
    a[i] = make_double2(1.0, 0.0);
}

template <typename T> static gp_status srp_spectral(gp_plan* p, int field, cpx<T>* psi, uint64_t seed, double k0, double trms) {
  FieldPlan& F = p->f[field];
  const long long npts = F.npts;
  cudaStream_t s = p->stream;
  gp_status st = ensure_ws(p, field, (size_t)npts * sizeof(double2));
  if (st != GP_OK) return st;
  double2* w = (double2*)F.ws;
  k_noise<<<igrid(npts), 256, 0, s>>>(w, npts, stream_pos(seed, 0));
  GP_CUDA(p, cudaGetLastError());
  GP_CUDA(p, fft3<double>(F, w, false, s));
  k_srp_filter<<<igrid(npts), 256, 0, s>>>(w, F.n, 1.0 / (k0 * k0));
  GP_CUDA(p, cudaGetLastError());
  GP_CUDA(p, fft3<double>(F, w, true, s));
  static_assert(SUM_BLOCKS <= 64, "partial sums fit the plan's accumulators");
  k_sum_re2<<<SUM_BLOCKS, SUM_THREADS, 0, s>>>(w, npts, p->acc);
  GP_CUDA(p, cudaGetLastError());
  double part[SUM_BLOCKS];
  GP_CUDA(p, cudaMemcpyAsync(part, p->acc, sizeof(part), cudaMemcpyDeviceToHost, s));
  GP_CUDA(p, cudaStreamSynchronize(s));
  double sum = 0.0;
  for (int b = 0; b < SUM_BLOCKS; ++b) sum += part[b];
  if (!(sum > 0.0)) return fail(p, GP_ERR_NONFINITE, "gp_init_srp: filtered noise has zero or non-finite RMS");
  const double scale = trms / std::sqrt(sum / (double)npts);
  k_phase_out<T><<<igrid(npts), 256, 0, s>>>(w, psi, npts, scale);
  GP_CUDA(p, cudaGetLastError());
  return GP_OK;
}

template <typename T> static gp_status srp_spline(gp_plan* p, int field, cpx<T>* psi, uint64_t seed, double K, int nr) {
  FieldPlan& F = p->f[field];
  const int n = F.n;
  std::vector<double> S = spline_matrix(n, nr);
  std::vector<double> lat((size_t)nr * nr * nr);
  for (size_t i = 0; i < lat.size(); ++i) lat[i] = K * (2.0 * u01(splitmix_at(stream_pos(seed, i))) - 1.0);
  const size_t t1 = (size_t)nr * nr * n, t2 = (size_t)nr * n * n;
  gp_status st = ensure_ws(p, field, (S.size() + lat.size() + t1 + t2) * sizeof(double));
  if (st != GP_OK) return st;
  double* dS = (double*)F.ws;
  double* dL = dS + S.size();
  double* dT1 = dL + lat.size();
  double* dT2 = dT1 + t1;
  cudaStream_t s = p->stream;
  GP_CUDA(p, cudaMemcpyAsync(dS, S.data(), S.size() * sizeof(double), cudaMemcpyHostToDevice, s));
  GP_CUDA(p, cudaMemcpyAsync(dL, lat.data(), lat.size() * sizeof(double), cudaMemcpyHostToDevice, s));
  k_spline_x<<<igrid((long long)t1), 256, 0, s>>>(dS, dL, n, nr, dT1);
  k_spline_y<<<igrid((long long)t2), 256, 0, s>>>(dS, dT1, n, nr, dT2);
  k_spline<T><<<igrid(F.npts), 256, 0, s>>>(dS, dT2, n, nr, psi);
  GP_CUDA(p, cudaGetLastError());
  GP_CUDA(p, cudaStreamSynchronize(s));  // host vectors go out of scope
  return GP_OK;
}

static void box_muller(uint64_t va, uint64_t vb, double* g0, double* g1) {
  const double r = std::sqrt(-2.0 * std::log(u01_open0(va)));
  const double t = 2.0 * M_PI * u01(vb);
  *g0 = r * std::cos(t);
  *g1 = r * std::sin(t);
}

template <typename T>
static gp_status rvr_rings(gp_plan* p, int field, cpx<T>* psi, uint64_t seed, int count, double rmin, double rmax) {
  FieldPlan& F = p->f[field];
  std::vector<Ring> rings(count > 0 ? count : 1);
  for (int j = 0; j < count; ++j) {
    auto U = [&](int c) { return u01(splitmix_at(stream_pos(seed, 8ull * j + c))); };
    Ring g;
    g.R = rmin + (rmax - rmin) * U(0);
    g.cx = 2.0 * M_PI * U(1);
    g.cy = 2.0 * M_PI * U(2);
    g.cz = 2.0 * M_PI * U(3);
    double n0, n1, n2, unused;
    box_muller(splitmix_at(stream_pos(seed, 8ull * j + 4)), splitmix_at(stream_pos(seed, 8ull * j + 5)), &n0, &n1);
    box_muller(splitmix_at(stream_pos(seed, 8ull * j + 6)), splitmix_at(stream_pos(seed, 8ull * j + 7)), &n2, &unused);
    const double nn = std::sqrt(n0 * n0 + n1 * n1 + n2 * n2);
    g.nx = n0 / nn;
    g.ny = n1 / nn;
    g.nz = n2 / nn;
    rings[j] = g;
  }
  gp_status st = ensure_ws(p, field, rings.size() * sizeof(Ring));
  if (st != GP_OK) return st;
  cudaStream_t s = p->stream;
  GP_CUDA(p, cudaMemcpyAsync(F.ws, rings.data(), rings.size() * sizeof(Ring), cudaMemcpyHostToDevice, s));
  const double xi = std::sqrt(F.alpha / F.beta);
  k_rings<T><<<igrid(F.npts), 256, 0, s>>>((const Ring*)F.ws, count, F.n, xi, psi);
  GP_CUDA(p, cudaGetLastError());
  GP_CUDA(p, cudaStreamSynchronize(s));
  return GP_OK;
}

template <typename T>
static gp_status rvr_pairs(gp_plan* p, int field, cpx<T>* psi, uint64_t seed, int npairs, double R, double d) {
  FieldPlan& F = p->f[field];
  const long long npts = F.npts;
  gp_status st = ensure_ws(p, field, 3 * (size_t)npts * sizeof(double2));
  if (st != GP_OK) return st;
  double2* w = (double2*)F.ws;
  double2* t = w + npts;
  double2* a = t + npts;
  cudaStream_t s = p->stream;
  const double xi = std::sqrt(F.alpha / F.beta);
  k_pair_base<<<igrid(npts), 256, 0, s>>>(w, F.n, R, d, xi);
  GP_CUDA(p, cudaGetLastError());
  GP_CUDA(p, fft3<double>(F, w, false, s));
  k_fill_one<<<igrid(npts), 256, 0, s>>>(a, npts);
  static const int orders[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  for (int q = 0; q < npairs; ++q) {
    auto U = [&](int c) { return u01(splitmix_at(stream_pos(seed, 4ull * q + c))); };
    const double X = 2.0 * M_PI * U(0), Y = 2.0 * M_PI * U(1), Z = 2.0 * M_PI * U(2);
    int o = (int)(6.0 * U(3));
    if (o > 5) o = 5;
    k_shift<<<igrid(npts), 256, 0, s>>>(w, t, F.n, X, Y, Z);
    GP_CUDA(p, cudaGetLastError());
    GP_CUDA(p, fft3<double>(F, t, true, s));
    k_accum_perm<<<igrid(npts), 256, 0, s>>>(a, t, F.n, orders[o][0], orders[o][1], orders[o][2]);
    GP_CUDA(p, cudaGetLastError());
  }
  k_copy_out<T><<<igrid(npts), 256, 0, s>>>(a, psi, npts);
  GP_CUDA(p, cudaGetLastError());
  return GP_OK;
}

}  // namespace gp

using namespace gp;

extern "C" {

gp_status gp_init_srp(gp_plan* p, int field, void* psi, uint64_t seed, int mode, double p0, double p1) {
  if (!p) return GP_ERR_INVALID_ARG;
  if (field < 0 || field >= (int)p->f.size()) return fail(p, GP_ERR_INVALID_ARG, "gp_init_srp: field index");
  if (!psi || ((uintptr_t)psi & 15)) return fail(p, GP_ERR_INVALID_ARG, "gp_init_srp: pointer");
  if (seed >= (1ull << 23)) return fail(p, GP_ERR_INVALID_ARG, "gp_init_srp: seed must be below 2^23");
  FieldPlan& F = p->f[field];
  if (mode == 0) {
    if (!(p0 > 0.0) || !std::isfinite(p0) || !std::isfinite(p1)) return fail(p, GP_ERR_INVALID_ARG, "gp_init_srp: k0 and theta_rms");
    return F.fp64 ? srp_spectral<double>(p, field, (cpx<double>*)psi, seed, p0, p1)
                  : srp_spectral<float>(p, field, (cpx<float>*)psi, seed, p0, p1);
  }
  if (mode == 1) {
    const int nr = (int)p1;
    if (nr < 3 || nr > 16 || F.n % nr || !std::isfinite(p0)) return fail(p, GP_ERR_INVALID_ARG, "gp_init_srp: need 3 <= N_r <= 16 dividing N");
    return F.fp64 ? srp_spline<double>(p, field, (cpx<double>*)psi, seed, p0, nr)
                  : srp_spline<float>(p, field, (cpx<float>*)psi, seed, p0, nr);
  }
  return fail(p, GP_ERR_INVALID_ARG, "gp_init_srp: mode must be 0 or 1");
}

gp_status gp_init_rvr(gp_plan* p, int field, void* psi, uint64_t seed, int mode, int count, double p0, double p1) {
  if (!p) return GP_ERR_INVALID_ARG;
  if (field < 0 || field >= (int)p->f.size()) return fail(p, GP_ERR_INVALID_ARG, "gp_init_rvr: field index");
  if (!psi || ((uintptr_t)psi & 15)) return fail(p, GP_ERR_INVALID_ARG, "gp_init_rvr: pointer");
  if (count < 0 || count > 4096 || !std::isfinite(p0) || !std::isfinite(p1))
    return fail(p, GP_ERR_INVALID_ARG, "gp_init_rvr: count or radius");
  if (seed >= (1ull << 23)) return fail(p, GP_ERR_INVALID_ARG, "gp_init_rvr: seed must be below 2^23");
  FieldPlan& F = p->f[field];
  if (mode == 0)
    return F.fp64 ? rvr_rings<double>(p, field, (cpx<double>*)psi, seed, count, p0, p1)
                  : rvr_rings<float>(p, field, (cpx<float>*)psi, seed, count, p0, p1);
  if (mode == 1)
    return F.fp64 ? rvr_pairs<double>(p, field, (cpx<double>*)psi, seed, count, p0, p1)
                  : rvr_pairs<float>(p, field, (cpx<float>*)psi, seed, count, p0, p1);
  return fail(p, GP_ERR_INVALID_ARG, "gp_init_rvr: mode must be 0 or 1");
}

}  // extern "C"

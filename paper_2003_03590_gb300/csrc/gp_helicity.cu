// gp_helicity.cu -- helicity and regularised helicity of one field (Sec. 3.6).
//
// Volume means, hbar/m = 2 alpha in the dimensionless units (v = 2 alpha grad theta):
//   H     = < v . omega >,  omega = curl v                                      (eq-helicity)
//   w     = (2 alpha / i) grad psi* x grad psi = 4 alpha grad Re(psi) x grad Im(psi)
//   v_par = 2 alpha w . Im(X) / (|w| |grad psi|^2),  X_i = sum_j (d_i d_j psi) conj(d_j psi)
//           (the paper's [(d_i d_j psi) d_j psi* - c.c.] / (2 i) is Im(X_i))
//   v_reg = v_par w / |w|,   H_reg = < v_reg . omega >                                  (Hreg)
// with v = 2 alpha Im(psi* grad psi) / |psi|^2 (0 where |psi|^2 < 1e-12), spectral first
// derivatives with Nyquist-zeroed wavenumbers k~, second derivatives -k~_i k~_j F psi, and
// v_reg = 0 where |w| <= 1e-5 * 4 alpha <|grad psi|^2> (v_par has no limit where grad psi
// vanishes; |w| <= 2 alpha |grad psi|^2, so the one cut covers both).
// Spectra: shell sums (b = floor(|k| + 1/2)) of Re(conj(F v) . F omega) / n^2 and
// Re(conj(F v_reg) . F omega) / n^2; H is the sum of its spectrum (Parseval), H_reg a
// pointwise mean.
//
// Pipeline (16 complex 3D FFTs, 19 with the spectra): F psi; the gradient (3 inverse); the
// velocity (3 forward); the curl in k-space with the H shell sums, omega (3 inverse); the six
// second derivatives in two batches of three (6 inverse), each followed by a pointwise kernel
// that accumulates w . Im(X); the pointwise v_reg and H_reg; with spectra, F v_reg (3 forward)
// and its shell sums against the curl of F v recomputed from the kept velocity spectrum.
#include <cmath>
#include <vector>

#include "gp_internal.h"
#include "gp_reduce.cuh"

namespace gp {
namespace {

constexpr double W_CUT = 1e-5;

inline unsigned hgrid(long long npts) {
  long long b = (npts + 255) / 256;
  return (unsigned)(b < 1 ? 1 : (b > 152LL * 16 ? 152LL * 16 : b));
}

#define HEL_LOOP(i, npts) \
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (npts); i += (long long)gridDim.x * blockDim.x)

// g_j = i k~_j psi_k, and the block sums of |k~|^2 |psi_k|^2 (= n^2 <|grad psi|^2> in total)
template <typename T>
__global__ void k_hel_grad(const cpx<T>* __restrict__ ph, cpx<T>* g1, cpx<T>* g2, cpx<T>* g3, int n, double* part) {
  const long long npts = (long long)n * n * n;
  Sums<T, 1> S;
  HEL_LOOP(i, npts) {
    int ix, iy, iz;
    coords3((unsigned)i, (unsigned)n, ix, iy, iz);
    const T dx = (T)wavenumber_d(ix, n), dy = (T)wavenumber_d(iy, n), dz = (T)wavenumber_d(iz, n);
    const cpx<T> a = ph[i];
    const T v[1] = {(dx * dx + dy * dy + dz * dz) * (a.x * a.x + a.y * a.y)};
    S.add(v);
    g1[i] = cpx<T>{-dx * a.y, dx * a.x};
    g2[i] = cpx<T>{-dy * a.y, dy * a.x};
    g3[i] = cpx<T>{-dz * a.y, dz * a.x};
  }
  S.flush();
  block_store<1>(S.d, part);
}

// v_j = 2 alpha Im(conj(psi) g_j) / |psi|^2 as complex fields (v_j, 0)
template <typename T>
__global__ void k_hel_velocity(const cpx<T>* __restrict__ psi, const cpx<T>* __restrict__ g1, const cpx<T>* __restrict__ g2,
                               const cpx<T>* __restrict__ g3, cpx<T>* v1, cpx<T>* v2, cpx<T>* v3, long long npts,
                               double alpha) {
  const T a2 = (T)(2.0 * alpha);
  HEL_LOOP(i, npts) {
    const cpx<T> p = psi[i];
    const T rho = p.x * p.x + p.y * p.y;
    const T f = rho >= eps_rho<T>() ? a2 / rho : T(0);
    const cpx<T> a = g1[i], b = g2[i], c = g3[i];
    v1[i] = cpx<T>{f * (p.x * a.y - p.y * a.x), T(0)};
    v2[i] = cpx<T>{f * (p.x * b.y - p.y * b.x), T(0)};
    v3[i] = cpx<T>{f * (p.x * c.y - p.y * c.x), T(0)};
  }
}

// i k~ x F v at mode i (grid coordinates ix, iy, iz)
template <typename T>
__device__ __forceinline__ void curl_mode(const cpx<T> (&vh)[3], int ix, int iy, int iz, int n, cpx<T> (&om)[3]) {
  const T k0 = (T)wavenumber_d(ix, n), k1 = (T)wavenumber_d(iy, n), k2 = (T)wavenumber_d(iz, n);
  // c = k~ x vh;  i c = (-c.y, c.x)
  const cpx<T> c0 = {k1 * vh[2].x - k2 * vh[1].x, k1 * vh[2].y - k2 * vh[1].y};
  const cpx<T> c1 = {k2 * vh[0].x - k0 * vh[2].x, k2 * vh[0].y - k0 * vh[2].y};
  const cpx<T> c2 = {k0 * vh[1].x - k1 * vh[0].x, k0 * vh[1].y - k1 * vh[0].y};
  om[0] = cpx<T>{-c0.y, c0.x};
  om[1] = cpx<T>{-c1.y, c1.x};
  om[2] = cpx<T>{-c2.y, c2.x};
}

// Re(conj(a) . b) summed over the three components
template <typename T> __device__ __forceinline__ T re_dot(const cpx<T> (&a)[3], const cpx<T> (&b)[3]) {
  return a[0].x * b[0].x + a[0].y * b[0].y + a[1].x * b[1].x + a[1].y * b[1].y + a[2].x * b[2].x + a[2].y * b[2].y;
}

// Shell sums of Re(conj(a_k) . (i k~ x vh_k)) into spec[0 .. nbins); optionally om_k = i k~ x vh_k.
// a = vh for H(k); a = F v_reg (with om = nullptr) for H_reg(k).
template <typename T>
__global__ void k_hel_shells(const cpx<T>* __restrict__ a1, const cpx<T>* __restrict__ a2, const cpx<T>* __restrict__ a3,
                             const cpx<T>* __restrict__ vh1, const cpx<T>* __restrict__ vh2, const cpx<T>* __restrict__ vh3,
                             cpx<T>* om1, cpx<T>* om2, cpx<T>* om3, int n, int nbins, double* spec) {
  extern __shared__ double hist[];
  for (int b = threadIdx.x; b < nbins; b += blockDim.x) hist[b] = 0.0;
  __syncthreads();
  const long long npts = (long long)n * n * n;
  HEL_LOOP(i, npts) {
    int ix, iy, iz;
    coords3((unsigned)i, (unsigned)n, ix, iy, iz);
    const cpx<T> vh[3] = {vh1[i], vh2[i], vh3[i]};
    cpx<T> om[3];
    curl_mode<T>(vh, ix, iy, iz, n, om);
    if (om1) {
      om1[i] = om[0];
      om2[i] = om[1];
      om3[i] = om[2];
    }
    const cpx<T> a[3] = {a1[i], a2[i], a3[i]};
    const T d = re_dot<T>(a, om);
    const int kx = wavenumber(ix, n), ky = wavenumber(iy, n), kz = wavenumber(iz, n);
    int b = shell_of(kx * kx + ky * ky + kz * kz);
    if (b >= nbins) b = nbins - 1;
    if (d != T(0)) atomicAdd(&hist[b], (double)d);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < nbins; b += blockDim.x)
    if (hist[b] != 0.0) atomicAdd(&spec[b], hist[b]);
}

// The three second derivatives of one batch: batch 0 = (xx, xy, xz), batch 1 = (yy, yz, zz).
template <typename T>
__global__ void k_hel_hess(const cpx<T>* __restrict__ ph, cpx<T>* t0, cpx<T>* t1, cpx<T>* t2, int n, int batch) {
  const long long npts = (long long)n * n * n;
  HEL_LOOP(i, npts) {
    int ix, iy, iz;
    coords3((unsigned)i, (unsigned)n, ix, iy, iz);
    const T k[3] = {(T)wavenumber_d(ix, n), (T)wavenumber_d(iy, n), (T)wavenumber_d(iz, n)};
    const cpx<T> a = ph[i];
    T m0, m1, m2;
    if (batch == 0) {
      m0 = -k[0] * k[0]; m1 = -k[0] * k[1]; m2 = -k[0] * k[2];
    } else {
      m0 = -k[1] * k[1]; m1 = -k[1] * k[2]; m2 = -k[2] * k[2];
    }
    t0[i] = cpx<T>{m0 * a.x, m0 * a.y};
    t1[i] = cpx<T>{m1 * a.x, m1 * a.y};
    t2[i] = cpx<T>{m2 * a.x, m2 * a.y};
  }
}

template <typename T> struct WG {
  T w[3];    // w = 4 alpha grad Re psi x grad Im psi
  T g2;      // |grad psi|^2
};

template <typename T>
__device__ __forceinline__ WG<T> w_of(const cpx<T> (&g)[3], T a4) {
  WG<T> r;
  r.w[0] = a4 * (g[1].x * g[2].y - g[2].x * g[1].y);
  r.w[1] = a4 * (g[2].x * g[0].y - g[0].x * g[2].y);
  r.w[2] = a4 * (g[0].x * g[1].y - g[1].x * g[0].y);
  r.g2 = g[0].x * g[0].x + g[0].y * g[0].y + g[1].x * g[1].x + g[1].y * g[1].y + g[2].x * g[2].x + g[2].y * g[2].y;
  return r;
}

// Im(h conj(g))
template <typename T> __device__ __forceinline__ T im_hcg(cpx<T> h, cpx<T> g) { return h.y * g.x - h.x * g.y; }

// num += sum over the batch's pairs (i <= j) of w_i Im(H_ij conj g_j) + [i != j] w_j Im(H_ij conj g_i)
template <typename T>
__global__ void k_hel_accum(const cpx<T>* __restrict__ g1, const cpx<T>* __restrict__ g2, const cpx<T>* __restrict__ g3,
                            const cpx<T>* __restrict__ t0, const cpx<T>* __restrict__ t1, const cpx<T>* __restrict__ t2,
                            T* num, long long npts, double alpha, int batch) {
  const T a4 = (T)(4.0 * alpha);
  HEL_LOOP(i, npts) {
    const cpx<T> g[3] = {g1[i], g2[i], g3[i]};
    const WG<T> q = w_of<T>(g, a4);
    const cpx<T> h0 = t0[i], h1 = t1[i], h2 = t2[i];
    T s;
    if (batch == 0) {   // (0,0), (0,1), (0,2)
      s = q.w[0] * im_hcg<T>(h0, g[0]) + (q.w[0] * im_hcg<T>(h1, g[1]) + q.w[1] * im_hcg<T>(h1, g[0])) +
          (q.w[0] * im_hcg<T>(h2, g[2]) + q.w[2] * im_hcg<T>(h2, g[0]));
      num[i] = s;
    } else {            // (1,1), (1,2), (2,2)
      s = q.w[1] * im_hcg<T>(h0, g[1]) + (q.w[1] * im_hcg<T>(h1, g[2]) + q.w[2] * im_hcg<T>(h1, g[1])) +
          q.w[2] * im_hcg<T>(h2, g[2]);
      num[i] += s;
    }
  }
}

// v_reg and the block sums of v_reg . omega; with write_vreg, g_j <- (v_reg_j, 0).
template <typename T>
__global__ void k_hel_final(cpx<T>* g1, cpx<T>* g2, cpx<T>* g3, const cpx<T>* __restrict__ om1,
                            const cpx<T>* __restrict__ om2, const cpx<T>* __restrict__ om3, const T* __restrict__ num,
                            long long npts, double alpha, const double* __restrict__ gsum, int write_vreg, double* part) {
  const T a4 = (T)(4.0 * alpha), a2 = (T)(2.0 * alpha);
  const double dn = (double)npts;
  const T cut = (T)(W_CUT * 4.0 * alpha * (gsum[0] / (dn * dn)));
  Sums<T, 1> S;
  HEL_LOOP(i, npts) {
    const cpx<T> g[3] = {g1[i], g2[i], g3[i]};
    const WG<T> q = w_of<T>(g, a4);
    const T wn = sqrt(q.w[0] * q.w[0] + q.w[1] * q.w[1] + q.w[2] * q.w[2]);
    T vr[3] = {T(0), T(0), T(0)};
    if (wn > cut && q.g2 > T(0)) {
      const T vpar = a2 * num[i] / (wn * q.g2);
      const T f = vpar / wn;
      vr[0] = f * q.w[0];
      vr[1] = f * q.w[1];
      vr[2] = f * q.w[2];
    }
    const T v[1] = {vr[0] * om1[i].x + vr[1] * om2[i].x + vr[2] * om3[i].x};
    S.add(v);
    if (write_vreg) {
      g1[i] = cpx<T>{vr[0], T(0)};
      g2[i] = cpx<T>{vr[1], T(0)};
      g3[i] = cpx<T>{vr[2], T(0)};
    }
  }
  S.flush();
  block_store<1>(S.d, part);
}

#undef HEL_LOOP

template <typename T>
gp_status helicity_impl(gp_plan* p, int field, const cpx<T>* psi, double* H, double* H_reg, double* spectra, int nbins_req) {
  FieldPlan& F = p->f[field];
  const long long npts = F.npts;
  const int n = F.n;
  const int nbins = gp_plan_nbins(p, field);
  cudaStream_t s = p->stream;
  const size_t fb = (size_t)npts * sizeof(cpx<T>);
  const unsigned g = hgrid(npts);
  const size_t numb = ((size_t)npts * sizeof(T) + 255) / 256 * 256;
  gp_status st = ensure_ws(p, field, 13 * fb + numb + ((size_t)2 * g + 2 * nbins) * sizeof(double));
  if (st != GP_OK) return st;
  cpx<T>* w[13];
  w[0] = (cpx<T>*)F.ws;
  for (int k = 1; k < 13; ++k) w[k] = w[k - 1] + npts;
  // w0 F psi | w1..3 grad psi (then v_reg) | w4..6 F v | w7..9 omega | w10..12 second derivatives
  T* num = (T*)(w[12] + npts);
  double* part = (double*)((unsigned char*)num + numb);   // [g] gradient sums, [g] H_reg sums
  double* spec = part + 2 * g;                              // [2][nbins] H(k), H_reg(k)
  GP_CUDA(p, cudaMemsetAsync(p->acc, 0, 2 * sizeof(double), s));
  GP_CUDA(p, cudaMemsetAsync(spec, 0, (size_t)2 * nbins * sizeof(double), s));
  auto transform = [&](int first, int count, bool inverse) -> cudaError_t {
    if constexpr (sizeof(T) == 4) return fft3_many(p, F, w + first, count, inverse, s);
    for (int k = first; k < first + count; ++k) {
      cudaError_t e = fft3<T>(F, w[k], inverse, s);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  };
  GP_CUDA(p, cudaMemcpyAsync(w[0], psi, fb, cudaMemcpyDeviceToDevice, s));
  GP_CUDA(p, transform(0, 1, false));
  k_hel_grad<T><<<g, 256, 0, s>>>(w[0], w[1], w[2], w[3], n, part);
  GP_CUDA(p, cudaGetLastError());
  k_reduce<<<1, 256, 0, s>>>(part, (int)g, 1, p->acc);
  GP_CUDA(p, cudaGetLastError());
  GP_CUDA(p, transform(1, 3, true));
  k_hel_velocity<T><<<g, 256, 0, s>>>(psi, w[1], w[2], w[3], w[4], w[5], w[6], npts, F.alpha);
  GP_CUDA(p, cudaGetLastError());
  GP_CUDA(p, transform(4, 3, false));
  const size_t hsm = (size_t)nbins * sizeof(double);
  const unsigned g2 = g < 4 * 152 ? g : 4 * 152;
  k_hel_shells<T><<<g2, 256, hsm, s>>>(w[4], w[5], w[6], w[4], w[5], w[6], w[7], w[8], w[9], n, nbins, spec);
  GP_CUDA(p, cudaGetLastError());
  GP_CUDA(p, transform(7, 3, true));
  for (int batch = 0; batch < 2; ++batch) {
    k_hel_hess<T><<<g, 256, 0, s>>>(w[0], w[10], w[11], w[12], n, batch);
    GP_CUDA(p, cudaGetLastError());
    GP_CUDA(p, transform(10, 3, true));
    k_hel_accum<T><<<g, 256, 0, s>>>(w[1], w[2], w[3], w[10], w[11], w[12], num, npts, F.alpha, batch);
    GP_CUDA(p, cudaGetLastError());
  }
  k_hel_final<T><<<g, 256, 0, s>>>(w[1], w[2], w[3], w[7], w[8], w[9], num, npts, F.alpha, p->acc, spectra ? 1 : 0,
                                   part + g);
  GP_CUDA(p, cudaGetLastError());
  k_reduce<<<1, 256, 0, s>>>(part + g, (int)g, 1, p->acc + 1);
  GP_CUDA(p, cudaGetLastError());
  if (spectra) {
    GP_CUDA(p, transform(1, 3, false));
    k_hel_shells<T><<<g2, 256, hsm, s>>>(w[1], w[2], w[3], w[4], w[5], w[6], nullptr, nullptr, nullptr, n, nbins,
                                         spec + nbins);
    GP_CUDA(p, cudaGetLastError());
  }
  double acc[2];
  std::vector<double> hs((size_t)2 * nbins);
  GP_CUDA(p, cudaMemcpyAsync(acc, p->acc, sizeof(acc), cudaMemcpyDeviceToHost, s));
  GP_CUDA(p, cudaMemcpyAsync(hs.data(), spec, hs.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
  GP_CUDA(p, cudaStreamSynchronize(s));
  st = check_status(p);
  if (st != GP_OK) return st;
  const double dn = (double)npts, dn2 = dn * dn;
  double h = 0.0;
  for (int b = 0; b < nbins; ++b) h += hs[b];
  *H = h / dn2;
  *H_reg = acc[1] / dn;
  if (!std::isfinite(*H) || !std::isfinite(*H_reg))
    return fail(p, GP_ERR_NONFINITE, "gp_helicity: non-finite result (field holds NaN or Inf)");
  if (spectra)
    for (int q = 0; q < 2; ++q)
      for (int b = 0; b < nbins; ++b) spectra[q * nbins_req + b] = hs[(size_t)q * nbins + b] / dn2;
  return GP_OK;
}

}  // namespace
}  // namespace gp

using namespace gp;

extern "C" gp_status gp_helicity(gp_plan* p, int field, const void* psi, double* H, double* H_reg, double* spectra,
                                 int nbins) {
  if (!p) return GP_ERR_INVALID_ARG;
  if (field < 0 || field >= (int)p->f.size()) return fail(p, GP_ERR_INVALID_ARG, "gp_helicity: field index");
  if (!psi || ((uintptr_t)psi & 15) || !H || !H_reg) return fail(p, GP_ERR_INVALID_ARG, "gp_helicity: pointer");
  if (spectra && nbins < gp_plan_nbins(p, field))
    return fail(p, GP_ERR_INVALID_ARG, "gp_helicity: nbins smaller than gp_plan_nbins");
  if (p->f[field].fp64) return helicity_impl<double>(p, field, (const cpx<double>*)psi, H, H_reg, spectra, nbins);
  return helicity_impl<float>(p, field, (const cpx<float>*)psi, H, H_reg, spectra, nbins);
}

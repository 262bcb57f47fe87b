// gp_adjoint.cu -- transpose of the split step (no counterpart in the paper) and the gradient
// of the incompressible kinetic energy of Sec. 3.4 (eq:def-ekin-decomp).
//
// Inner product <a, b> = Re sum_x conj(a_x) b_x.  Sub-flow VJPs:
//   K(s) = F^-1 exp(-i alpha |k|^2 s) F is unitary:  VJP_K(s) lam = K(-s) lam
//   N(s): psi_out = exp(-i phi) psi, phi = beta s (|psi|^2 - c):
//         VJP_N(s) lam = exp(+i phi) lam + 2 beta s Im(conj(lam) psi_out) psi
// A step's VJP applies these in reverse order at the step's intermediate states.
//
// J(psi) = E_kin^i with u = 2 alpha Im(psi* grad psi) / |psi|_e, |psi|_e = sqrt(|psi|^2 + eps):
//   lam = dJ/dpsi = (2 alpha / n) sum_j [ -i w_j d_j psi - d_j(i w_j psi) - w_j Im(psi* d_j psi) psi / |psi|_e^2 ],
//   w_j = u^i_j / |psi|_e, d_j the Nyquist-zeroed spectral derivative (d_j^T = -d_j).
#include <cmath>
#include <vector>

#include "gp_internal.h"
#include "gp_reduce.cuh"

namespace gp {

__device__ __forceinline__ int kw(int i, int n) { return i < (n + 1) / 2 ? i : i - n; }
__device__ __forceinline__ int kwd(int i, int n) { return (2 * i == n) ? 0 : kw(i, n); }

static inline unsigned agrid(long long n) {
  long long b = (n + 255) / 256;
  return (unsigned)(b < 1 ? 1 : (b > 152LL * 32 ? 152LL * 32 : b));
}

// W_j = i k~_j psi_k
template <typename T> __global__ void k_grad_spec(const cpx<T>* ph, cpx<T>* w1, cpx<T>* w2, cpx<T>* w3, int n) {
  const long long npts = (long long)n * n * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npts; i += (long long)gridDim.x * blockDim.x) {
    const int ix = (int)(i % n), iy = (int)((i / n) % n), iz = (int)(i / ((long long)n * n));
    cpx<T> a = ph[i];
    const T dx = (T)kwd(ix, n), dy = (T)kwd(iy, n), dz = (T)kwd(iz, n);
    w1[i] = cpx<T>{-dx * a.y, dx * a.x};
    w2[i] = cpx<T>{-dy * a.y, dy * a.x};
    w3[i] = cpx<T>{-dz * a.y, dz * a.x};
  }
}

// u_j = 2 alpha Im(conj(psi) g_j) / |psi|_e, packed as (u_x + i u_y) and (u_z + 0 i)
template <typename T>
__global__ void k_u_reg(const cpx<T>* psi, const cpx<T>* g1, const cpx<T>* g2, const cpx<T>* g3, cpx<T>* uxy, cpx<T>* uz,
                        long long npts, T alpha2, T eps) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npts; i += (long long)gridDim.x * blockDim.x) {
    cpx<T> p = psi[i];
    const T inv = T(1) / sqrt(p.x * p.x + p.y * p.y + eps);
    cpx<T> a = g1[i], b = g2[i], c = g3[i];
    const T ux = alpha2 * (p.x * a.y - p.y * a.x) * inv;
    const T uy = alpha2 * (p.x * b.y - p.y * b.x) * inv;
    const T uzv = alpha2 * (p.x * c.y - p.y * c.x) * inv;
    uxy[i] = cpx<T>{ux, uy};
    uz[i] = cpx<T>{uzv, T(0)};
  }
}

// incompressible projection of the packed spectra; per-block sums of |u^i|^2 / 2 into part.
// Per-point arithmetic in the field's precision (float64 per point is slow on GB300), sums in
// float64 (Sums: float32 partials of at most 32 terms), added up over blocks in a fixed order.
template <typename T>
__global__ void k_proj_i(const cpx<T>* __restrict__ uxy, const cpx<T>* __restrict__ uz, cpx<T>* oxy, cpx<T>* oz, int n,
                         double* part) {
  const long long npts = (long long)n * n * n;
  Sums<T, 1> S;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npts; i += (long long)gridDim.x * blockDim.x) {
    const int ix = (int)(i % n), iy = (int)((i / n) % n), iz = (int)(i / ((long long)n * n));
    const long long im = ((long long)((n - iz) % n) * n + (n - iy) % n) * n + (n - ix) % n;
    const cpx<T> z = uxy[i], zm = uxy[im];
    // X_k = (Z(k) + conj Z(-k)) / 2, Y_k = (Z(k) - conj Z(-k)) / (2i)
    T xr = T(0.5) * (z.x + zm.x), xi = T(0.5) * (z.y - zm.y);
    T yr = T(0.5) * (z.y + zm.y), yi = T(-0.5) * (z.x - zm.x);
    const cpx<T> w = uz[i];
    T zr = w.x, zi = w.y;
    const T k0 = (T)kwd(ix, n), k1 = (T)kwd(iy, n), k2 = (T)kwd(iz, n);
    const T kk = k0 * k0 + k1 * k1 + k2 * k2;
    if (kk > T(0)) {
      const T inv = T(1) / kk;
      const T cr = (k0 * xr + k1 * yr + k2 * zr) * inv, ci = (k0 * xi + k1 * yi + k2 * zi) * inv;
      xr -= k0 * cr; xi -= k0 * ci;
      yr -= k1 * cr; yi -= k1 * ci;
      zr -= k2 * cr; zi -= k2 * ci;
    }
    const T v[1] = {T(0.5) * (xr * xr + xi * xi + yr * yr + yi * yi + zr * zr + zi * zi)};
    S.add(v);
    // spectrum of u^i_x + i u^i_y is X + i Y
    oxy[i] = cpx<T>{xr - yi, xi + yr};
    oz[i] = cpx<T>{zr, zi};
  }
  S.flush();
  block_store<1>(S.d, part);
}

// pointwise part of lam and the fields V_j = i w_j psi whose derivatives are needed
template <typename T>
__global__ void k_lam_local(const cpx<T>* psi, cpx<T>* g1, cpx<T>* g2, cpx<T>* g3, const cpx<T>* uixy, const cpx<T>* uiz,
                            cpx<T>* lam, long long npts, T eps) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npts; i += (long long)gridDim.x * blockDim.x) {
    cpx<T> p = psi[i];
    const T a2 = p.x * p.x + p.y * p.y + eps;
    const T inv = T(1) / sqrt(a2);
    cpx<T> uxy = uixy[i];
    const T w[3] = {uxy.x * inv, uxy.y * inv, uiz[i].x * inv};
    cpx<T>* gs[3] = {g1, g2, g3};
    T lr = 0, li = 0;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      cpx<T> g = gs[j][i];
      const T im = p.x * g.y - p.y * g.x;  // Im(conj(psi) g)
      // -i w g
      lr += w[j] * g.y;
      li += -w[j] * g.x;
      // - w Im(conj(psi) g) psi / |psi|_e^2
      const T c = w[j] * im / a2;
      lr -= c * p.x;
      li -= c * p.y;
      gs[j][i] = cpx<T>{-w[j] * p.y, w[j] * p.x};  // V_j = i w_j psi
    }
    lam[i] = cpx<T>{lr, li};
  }
}

// D_k = sum_j i k~_j V_j,k
template <typename T> __global__ void k_div_spec(const cpx<T>* v1, const cpx<T>* v2, const cpx<T>* v3, cpx<T>* d, int n) {
  const long long npts = (long long)n * n * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npts; i += (long long)gridDim.x * blockDim.x) {
    const int ix = (int)(i % n), iy = (int)((i / n) % n), iz = (int)(i / ((long long)n * n));
    const T kx = (T)kwd(ix, n), ky = (T)kwd(iy, n), kz = (T)kwd(iz, n);
    cpx<T> a = v1[i], b = v2[i], c = v3[i];
    const T sr = kx * a.x + ky * b.x + kz * c.x, si = kx * a.y + ky * b.y + kz * c.y;
    d[i] = cpx<T>{-si, sr};
  }
}

// lam = scale (lam - D)
template <typename T> __global__ void k_lam_final(cpx<T>* lam, const cpx<T>* d, long long npts, T scale) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npts; i += (long long)gridDim.x * blockDim.x) {
    cpx<T> l = lam[i], q = d[i];
    lam[i] = cpx<T>{scale * (l.x - q.x), scale * (l.y - q.y)};
  }
}

template <typename T> static gp_status ekin_grad_impl(gp_plan* p, int field, const cpx<T>* psi, cpx<T>* lam, double eps,
                                                     double* J_out) {
  FieldPlan& F = p->f[field];
  const long long npts = F.npts;
  const int n = F.n;
  cudaStream_t s = p->stream;
  const size_t fb = (size_t)npts * sizeof(cpx<T>);
  const unsigned g = agrid(npts);
  gp_status st = ensure_ws(p, field, 7 * fb + (size_t)g * sizeof(double));
  if (st != GP_OK) return st;
  cpx<T>* w[7];
  for (int i = 0; i < 7; ++i) w[i] = (cpx<T>*)F.ws + (size_t)i * npts;
  double* part = (double*)(w[6] + npts);
  GP_CUDA(p, cudaMemcpyAsync(w[0], psi, fb, cudaMemcpyDeviceToDevice, s));
  GP_CUDA(p, fft3<T>(F, w[0], false, s));
  k_grad_spec<T><<<agrid(npts), 256, 0, s>>>(w[0], w[1], w[2], w[3], n);
  for (int j = 1; j <= 3; ++j) GP_CUDA(p, fft3<T>(F, w[j], true, s));
  k_u_reg<T><<<agrid(npts), 256, 0, s>>>(psi, w[1], w[2], w[3], w[0], w[4], npts, (T)(2.0 * F.alpha), (T)eps);
  GP_CUDA(p, fft3<T>(F, w[0], false, s));
  GP_CUDA(p, fft3<T>(F, w[4], false, s));
  k_proj_i<T><<<g, 256, 0, s>>>(w[0], w[4], w[5], w[6], n, part);
  k_reduce<<<1, 256, 0, s>>>(part, (int)g, 1, p->acc);
  GP_CUDA(p, fft3<T>(F, w[5], true, s));
  GP_CUDA(p, fft3<T>(F, w[6], true, s));
  k_lam_local<T><<<agrid(npts), 256, 0, s>>>(psi, w[1], w[2], w[3], w[5], w[6], lam, npts, (T)eps);
  for (int j = 1; j <= 3; ++j) GP_CUDA(p, fft3<T>(F, w[j], false, s));
  k_div_spec<T><<<agrid(npts), 256, 0, s>>>(w[1], w[2], w[3], w[0], n);
  GP_CUDA(p, fft3<T>(F, w[0], true, s));
  k_lam_final<T><<<agrid(npts), 256, 0, s>>>(lam, w[0], npts, (T)(2.0 * F.alpha / (double)npts));
  GP_CUDA(p, cudaGetLastError());
  if (J_out) {
    double acc = 0.0;
    GP_CUDA(p, cudaMemcpyAsync(&acc, p->acc, sizeof(double), cudaMemcpyDeviceToHost, s));
    GP_CUDA(p, cudaStreamSynchronize(s));
    *J_out = acc / ((double)npts * (double)npts);
  }
  return GP_OK;
}

template <typename T> static gp_status adjoint_impl(gp_plan* p, int field, const cpx<T>* psi_n, cpx<T>* lam, int nsteps) {
  FieldPlan& F = p->f[field];
  const long long npts = F.npts;
  cudaStream_t s = p->stream;
  const size_t fb = (size_t)npts * sizeof(cpx<T>);
  const size_t need = (size_t)(nsteps + 1) * fb;
  if (p->adj_bytes < need) {
    if (p->adj_ws) cudaFree(p->adj_ws);
    p->adj_ws = nullptr;
    p->adj_bytes = 0;
    GP_CUDA(p, cudaMalloc(&p->adj_ws, need));
    p->adj_bytes = need;
  }
  cpx<T>* S = (cpx<T>*)p->adj_ws;
  cpx<T>* tmp = S + (size_t)nsteps * npts;
  const double dt = F.prm.dt, h = 0.5 * dt, shift = F.prm.nonlin_minus_one ? 1.0 : 0.0;
  const bool f64 = sizeof(T) == 8;
  const cpx<T>* kd = (const cpx<T>*)ktable(p, field, dt, f64);
  const cpx<T>* kmd = (const cpx<T>*)ktable(p, field, -dt, f64);
  const cpx<T>* kh = (const cpx<T>*)ktable(p, field, h, f64);
  const cpx<T>* kmh = (const cpx<T>*)ktable(p, field, -h, f64);
  if (!kd || !kmd || !kh || !kmh) return fail(p, GP_ERR_OOM, "kinetic table allocation");
  // recompute the states at the start of every step of the segment
  GP_CUDA(p, cudaMemcpyAsync(S, psi_n, fb, cudaMemcpyDeviceToDevice, s));
  for (int m = 1; m < nsteps; ++m) {
    GP_CUDA(p, cudaMemcpyAsync(S + (size_t)m * npts, S + (size_t)(m - 1) * npts, fb, cudaMemcpyDeviceToDevice, s));
    gp_status st = step_field(p, field, S + (size_t)m * npts, 1);
    if (st != GP_OK) return st;
  }
  for (int m = nsteps - 1; m >= 0; --m) {
    const cpx<T>* Sm = S + (size_t)m * npts;
    GP_CUDA(p, cudaMemcpyAsync(tmp, Sm, fb, cudaMemcpyDeviceToDevice, s));
    if (F.prm.split == GP_SPLIT_NKN) {
      GP_CUDA(p, launch_nonlinear<T>(tmp, npts, F.beta * h, shift, s));          // a = N(h) S_m
      GP_CUDA(p, kinetic3<T>(F, tmp, kd, s));                                    // b = K(dt) a
      GP_CUDA(p, launch_vjp_nonlinear<T>(tmp, lam, npts, F.beta * h, shift, s)); // through N(h) at b
      GP_CUDA(p, kinetic3<T>(F, lam, kmd, s));                                   // through K(dt)
      GP_CUDA(p, launch_vjp_nonlinear<T>(Sm, lam, npts, F.beta * h, shift, s));  // through N(h) at S_m
    } else {
      GP_CUDA(p, kinetic3<T>(F, tmp, kh, s));                                    // a = K(h) S_m
      GP_CUDA(p, kinetic3<T>(F, lam, kmh, s));                                   // through the last K(h)
      GP_CUDA(p, launch_vjp_nonlinear<T>(tmp, lam, npts, F.beta * dt, shift, s));// through N(dt) at a
      GP_CUDA(p, kinetic3<T>(F, lam, kmh, s));                                   // through the first K(h)
    }
  }
  return GP_OK;
}

}  // namespace gp

using namespace gp;

extern "C" {

gp_status gp_adjoint_step(gp_plan* p, int field, const void* psi_n, void* lambda, int nsteps) {
  if (!p) return GP_ERR_INVALID_ARG;
  if (field < 0 || field >= (int)p->f.size()) return fail(p, GP_ERR_INVALID_ARG, "gp_adjoint_step: field index");
  if (!psi_n || !lambda || ((uintptr_t)psi_n & 15) || ((uintptr_t)lambda & 15))
    return fail(p, GP_ERR_INVALID_ARG, "gp_adjoint_step: pointer");
  if (nsteps < 0) return fail(p, GP_ERR_INVALID_ARG, "gp_adjoint_step: negative nsteps");
  if (nsteps == 0) return GP_OK;
  if (p->f[field].fp64) return adjoint_impl<double>(p, field, (const cpx<double>*)psi_n, (cpx<double>*)lambda, nsteps);
  return adjoint_impl<float>(p, field, (const cpx<float>*)psi_n, (cpx<float>*)lambda, nsteps);
}

gp_status gp_ekin_i_grad(gp_plan* p, int field, const void* psi, void* lambda_out, double eps, double* J_out) {
  if (!p) return GP_ERR_INVALID_ARG;
  if (field < 0 || field >= (int)p->f.size()) return fail(p, GP_ERR_INVALID_ARG, "gp_ekin_i_grad: field index");
  if (!psi || !lambda_out || ((uintptr_t)psi & 15) || ((uintptr_t)lambda_out & 15))
    return fail(p, GP_ERR_INVALID_ARG, "gp_ekin_i_grad: pointer");
  if (!(eps > 0.0) || !std::isfinite(eps)) return fail(p, GP_ERR_INVALID_ARG, "gp_ekin_i_grad: eps must be positive");
  if (p->f[field].fp64)
    return ekin_grad_impl<double>(p, field, (const cpx<double>*)psi, (cpx<double>*)lambda_out, eps, J_out);
  return ekin_grad_impl<float>(p, field, (const cpx<float>*)psi, (cpx<float>*)lambda_out, eps, J_out);
}

}  // extern "C"

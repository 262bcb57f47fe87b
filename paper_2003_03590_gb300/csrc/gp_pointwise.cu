// gp_pointwise.cu -- pointwise kernels of the plain (unfused) path and of the adjoint.
#include "gp_internal.h"

namespace gp {

static inline unsigned grid_for(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  return (unsigned)(b < 1 ? 1 : (b > 152LL * 64 ? 152LL * 64 : b));
}

// N(s): psi <- exp(-i coef (|psi|^2 - shift)) psi   (Sec. 4.3, exact nonlinear flow)
template <typename T> __global__ void k_nonlinear(cpx<T>* psi, long long npts, T coef, T shift) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npts; i += (long long)gridDim.x * blockDim.x)
    psi[i] = nonlinear(psi[i], coef, shift);
}

// K in Fourier space: psi_k *= E[kx] E[ky] E[kz]
template <typename T> __global__ void k_kinetic_mul(cpx<T>* psi, int n, const cpx<T>* __restrict__ ek) {
  const long long npts = (long long)n * n * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npts; i += (long long)gridDim.x * blockDim.x) {
    int ix = (int)(i % n), iy = (int)((i / n) % n), iz = (int)(i / ((long long)n * n));
    cpx<T> f = cmul(cmul(__ldg(ek + ix), __ldg(ek + iy)), __ldg(ek + iz));
    psi[i] = cmul(psi[i], f);
  }
}

// VJP of N(s) at input psi_in: lam <- exp(+i phi) lam + 2 coef Im(conj(lam) psi_out) psi_in,
// phi = coef (|psi_in|^2 - shift), psi_out = exp(-i phi) psi_in, coef = beta s.
template <typename T>
__global__ void k_vjp_nonlinear(const cpx<T>* __restrict__ psi_in, cpx<T>* lam, long long npts, T coef, T shift) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npts; i += (long long)gridDim.x * blockDim.x) {
    cpx<T> p = psi_in[i], l = lam[i];
    T ph = coef * (p.x * p.x + p.y * p.y - shift);
    T sn, cs;
    if constexpr (sizeof(T) == 4) sincosf(ph, &sn, &cs);
    else sincos(ph, &sn, &cs);
    cpx<T> po{p.x * cs + p.y * sn, p.y * cs - p.x * sn};          // exp(-i ph) p
    T im = l.x * po.y - l.y * po.x;                                 // Im(conj(l) po)
    T g = T(2) * coef * im;
    lam[i] = cpx<T>{l.x * cs - l.y * sn + g * p.x, l.y * cs + l.x * sn + g * p.y};
  }
}

template <typename T> __global__ void k_psi_from_phase(const T* __restrict__ th, cpx<T>* psi, long long npts) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npts; i += (long long)gridDim.x * blockDim.x) {
    T sn, cs;
    if constexpr (sizeof(T) == 4) sincosf(th[i], &sn, &cs);
    else sincos(th[i], &sn, &cs);
    psi[i] = cpx<T>{cs, sn};
  }
}

// dJ/dtheta = -Im(conj(lam) psi) for psi = exp(i theta)
template <typename T>
__global__ void k_phase_grad(const cpx<T>* __restrict__ psi, const cpx<T>* __restrict__ lam, T* g, long long npts) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npts; i += (long long)gridDim.x * blockDim.x) {
    cpx<T> p = psi[i], l = lam[i];
    g[i] = -(l.x * p.y - l.y * p.x);
  }
}

template <typename T> cudaError_t launch_nonlinear(cpx<T>* psi, long long npts, double coef, double shift, cudaStream_t s) {
  k_nonlinear<T><<<grid_for(npts, 256), 256, 0, s>>>(psi, npts, (T)coef, (T)shift);
  return cudaGetLastError();
}
template <typename T> cudaError_t launch_kinetic_mul(cpx<T>* psi, int n, const cpx<T>* ek, cudaStream_t s) {
  k_kinetic_mul<T><<<grid_for((long long)n * n * n, 256), 256, 0, s>>>(psi, n, ek);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_vjp_nonlinear(const cpx<T>* psi_in, cpx<T>* lam, long long npts, double coef, double shift, cudaStream_t s) {
  k_vjp_nonlinear<T><<<grid_for(npts, 256), 256, 0, s>>>(psi_in, lam, npts, (T)coef, (T)shift);
  return cudaGetLastError();
}
template cudaError_t launch_nonlinear<float>(cpx<float>*, long long, double, double, cudaStream_t);
template cudaError_t launch_nonlinear<double>(cpx<double>*, long long, double, double, cudaStream_t);
template cudaError_t launch_kinetic_mul<float>(cpx<float>*, int, const cpx<float>*, cudaStream_t);
template cudaError_t launch_kinetic_mul<double>(cpx<double>*, int, const cpx<double>*, cudaStream_t);
template cudaError_t launch_vjp_nonlinear<float>(const cpx<float>*, cpx<float>*, long long, double, double, cudaStream_t);
template cudaError_t launch_vjp_nonlinear<double>(const cpx<double>*, cpx<double>*, long long, double, double, cudaStream_t);

}  // namespace gp

using namespace gp;

static bool bad_ptr(const void* q) { return q == nullptr || ((uintptr_t)q & 15) != 0; }

extern "C" {

gp_status gp_psi_from_phase(gp_plan* p, int field, const void* theta, void* psi) {
  if (!p) return GP_ERR_INVALID_ARG;
  if (field < 0 || field >= (int)p->f.size()) return fail(p, GP_ERR_INVALID_ARG, "gp_psi_from_phase: field index");
  if (theta == nullptr || ((uintptr_t)theta & 7) || bad_ptr(psi)) return fail(p, GP_ERR_INVALID_ARG, "gp_psi_from_phase: pointer");
  FieldPlan& F = p->f[field];
  if (F.fp64)
    k_psi_from_phase<double><<<grid_for(F.npts, 256), 256, 0, p->stream>>>((const double*)theta, (cpx<double>*)psi, F.npts);
  else
    k_psi_from_phase<float><<<grid_for(F.npts, 256), 256, 0, p->stream>>>((const float*)theta, (cpx<float>*)psi, F.npts);
  GP_CUDA(p, cudaGetLastError());
  return GP_OK;
}

gp_status gp_phase_grad(gp_plan* p, int field, const void* psi, const void* lam, void* g) {
  if (!p) return GP_ERR_INVALID_ARG;
  if (field < 0 || field >= (int)p->f.size()) return fail(p, GP_ERR_INVALID_ARG, "gp_phase_grad: field index");
  if (bad_ptr(psi) || bad_ptr(lam) || g == nullptr || ((uintptr_t)g & 7)) return fail(p, GP_ERR_INVALID_ARG, "gp_phase_grad: pointer");
  FieldPlan& F = p->f[field];
  if (F.fp64)
    k_phase_grad<double><<<grid_for(F.npts, 256), 256, 0, p->stream>>>((const cpx<double>*)psi, (const cpx<double>*)lam,
                                                                        (double*)g, F.npts);
  else
    k_phase_grad<float><<<grid_for(F.npts, 256), 256, 0, p->stream>>>((const cpx<float>*)psi, (const cpx<float>*)lam,
                                                                      (float*)g, F.npts);
  GP_CUDA(p, cudaGetLastError());
  return GP_OK;
}

}  // extern "C"

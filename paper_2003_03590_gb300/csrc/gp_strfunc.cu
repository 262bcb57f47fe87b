// gp_strfunc.cu -- longitudinal velocity structure functions (Sec. 3.5, strfunc-def).
//
//   S^p_j(s dx) = < (v_j(x + s dx e_j) - v_j(x))^p >,   j = x, y, z,  s = 0 .. N/2,
// with the superfluid velocity v = 2 alpha Im(psi* grad psi) / |psi|^2 (eq-scaling-rhov; the
// spectral gradient of the diagnostics, Nyquist-zeroed wavenumbers; v = 0 where |psi|^2 < 1e-12).
//
// Pipeline: one forward 3D FFT, the three gradient spectra, three inverse FFTs, a pointwise
// kernel that writes the three real velocity components, then per direction one kernel over
// "pencils" (the N points of a line along e_j).  A block stages W pencils in shared memory, each
// row followed by a wrapped copy of its start so that the periodic shift needs no modulo, and
// every thread sums R consecutive separations of one pencil at a time: a register window of 2R
// shifted values slides along the pencil, so each shared-memory load serves R differences.
// The per-pencil sums (N terms) are formed in the field's precision and added in float64; the
// per-block sums are added up over blocks in a fixed order (no atomics: the result is the same
// on every call).
#include <cmath>
#include <vector>

#include "gp_internal.h"
#include "gp_reduce.cuh"

namespace gp {
namespace {

constexpr int SF_R = 8;          // separations per thread
constexpr int SF_THREADS = 256;
constexpr int SF_MAX_ORDER = 8;

// W_j = i k~_j psi_k
template <typename T>
__global__ void k_sf_grad(const cpx<T>* __restrict__ ph, cpx<T>* w1, cpx<T>* w2, cpx<T>* w3, int n) {
  const long long npts = (long long)n * n * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npts; i += (long long)gridDim.x * blockDim.x) {
    int ix, iy, iz;
    coords3((unsigned)i, (unsigned)n, ix, iy, iz);
    const T dx = (T)wavenumber_d(ix, n), dy = (T)wavenumber_d(iy, n), dz = (T)wavenumber_d(iz, n);
    const cpx<T> a = ph[i];
    w1[i] = cpx<T>{-dx * a.y, dx * a.x};
    w2[i] = cpx<T>{-dy * a.y, dy * a.x};
    w3[i] = cpx<T>{-dz * a.y, dz * a.x};
  }
}

// v_j = 2 alpha Im(conj(psi) g_j) / |psi|^2, 0 where |psi|^2 < eps_rho
template <typename T>
__global__ void k_sf_velocity(const cpx<T>* __restrict__ psi, const cpx<T>* __restrict__ g1, const cpx<T>* __restrict__ g2,
                              const cpx<T>* __restrict__ g3, T* vx, T* vy, T* vz, long long npts, double alpha) {
  const T a2 = (T)(2.0 * alpha);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npts; i += (long long)gridDim.x * blockDim.x) {
    const cpx<T> p = psi[i];
    const T rho = p.x * p.x + p.y * p.y;
    const T f = rho >= eps_rho<T>() ? a2 / rho : T(0);
    const cpx<T> a = g1[i], b = g2[i], c = g3[i];
    vx[i] = f * (p.x * a.y - p.y * a.x);
    vy[i] = f * (p.x * b.y - p.y * b.x);
    vz[i] = f * (p.x * c.y - p.y * c.x);
  }
}

template <typename T, int P> __device__ __forceinline__ T ipow(T d) {
  T t = d;
#pragma unroll
  for (int k = 1; k < P; ++k) t *= d;
  return t;
}

// Per block: part[blockIdx.x * ns + s] = sum over the block's pencils of sum_i (v[i + s] - v[i])^P.
//   v: one real velocity component [z][y][x];  axis: the direction of the pencils;
//   W pencils per tile (a power of two dividing n);  ntiles = n^2 / W;
//   row stride PL = n + ns + 3R (the wrapped copy covers every index the window reads).
template <typename T, int P>
__global__ void __launch_bounds__(SF_THREADS) k_strfunc(const T* __restrict__ v, int n, int axis, int W, int ntiles,
                                                         double* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char sf_smem[];
  T* rows = (T*)sf_smem;
  const int ns = n / 2 + 1, PL = n + ns + 3 * SF_R;
  const int G = (ns + SF_R - 1) / SF_R;           // separation groups
  const int TPG = SF_THREADS / G;                 // threads per group (G <= 256 for n <= 4094)
  const int g = threadIdx.x % G, lw = threadIdx.x / G;
  const bool active = lw < TPG;
  const int s0 = g * SF_R;
  double acc[SF_R];
#pragma unroll
  for (int r = 0; r < SF_R; ++r) acc[r] = 0.0;
  const long long nn = (long long)n * n;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    __syncthreads();   // the previous tile's rows are no longer read
    // stage W pencils: rows[w * PL + i] = v(pencil w, point i)
    if (axis == 0) {
      const T* src = v + (long long)tile * W * n;     // W consecutive rows along x
      for (int e = threadIdx.x; e < W * n; e += SF_THREADS) rows[(e / n) * PL + e % n] = src[e];
    } else {
      // tile -> (outer, x0): outer = z (axis y) or y (axis z), x0 = first of W consecutive x
      const int per = n / W, outer = tile / per, x0 = (tile - outer * per) * W;
      for (int e = threadIdx.x; e < W * n; e += SF_THREADS) {
        const int w = e % W, i = e / W;
        const long long idx = axis == 1 ? ((long long)outer * n + i) * n + x0 + w : (long long)i * nn + (long long)outer * n + x0 + w;
        rows[w * PL + i] = v[idx];
      }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < W * (PL - n); e += SF_THREADS) {
      const int w = e / (PL - n), t = e - w * (PL - n);
      rows[w * PL + n + t] = rows[w * PL + t % n];
    }
    __syncthreads();
    if (active) {
      for (int w = lw; w < W; w += TPG) {
        const T* rw = rows + w * PL;
        T win[2 * SF_R];
#pragma unroll
        for (int q = 0; q < 2 * SF_R; ++q) win[q] = rw[s0 + q];
        T sum[SF_R];
#pragma unroll
        for (int r = 0; r < SF_R; ++r) sum[r] = T(0);
        for (int i0 = 0; i0 < n; i0 += SF_R) {
#pragma unroll
          for (int ii = 0; ii < SF_R; ++ii) {
            if (i0 + ii < n) {
              const T a = rw[i0 + ii];
#pragma unroll
              for (int r = 0; r < SF_R; ++r) sum[r] += ipow<T, P>(win[ii + r] - a);
            }
          }
#pragma unroll
          for (int q = 0; q < SF_R; ++q) {
            win[q] = win[q + SF_R];
            win[q + SF_R] = rw[i0 + s0 + 2 * SF_R + q];
          }
        }
#pragma unroll
        for (int r = 0; r < SF_R; ++r) acc[r] += (double)sum[r];
      }
    }
  }
  __syncthreads();
  double* red = (double*)sf_smem;   // [SF_THREADS][SF_R]
#pragma unroll
  for (int r = 0; r < SF_R; ++r) red[threadIdx.x * SF_R + r] = active ? acc[r] : 0.0;
  __syncthreads();
  for (int s = threadIdx.x; s < ns; s += SF_THREADS) {
    const int gs = s / SF_R, r = s - gs * SF_R;
    double t = 0.0;
    for (int l = 0; l < TPG; ++l) t += red[(l * G + gs) * SF_R + r];
    part[(long long)blockIdx.x * ns + s] = t;
  }
}

// out[s] = sum over blocks b (in order) of part[b * ns + s]
__global__ void k_sf_sum_blocks(const double* __restrict__ part, int nblocks, int ns, double* out) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < ns; s += gridDim.x * blockDim.x) {
    double t = 0.0;
    for (int b = 0; b < nblocks; ++b) t += part[(long long)b * ns + s];
    out[s] = t;
  }
}

inline unsigned sf_grid(long long npts) {
  long long b = (npts + 255) / 256;
  return (unsigned)(b < 1 ? 1 : (b > 152LL * 16 ? 152LL * 16 : b));
}

// pencils per tile: a power of two dividing n, at most 32, rows within the shared-memory budget
inline int sf_tile_width(int n, size_t elem) {
  const int ns = n / 2 + 1, PL = n + ns + 3 * SF_R;
  int w = 1;
  while (w < 32 && n % (2 * w) == 0 && (size_t)(2 * w) * PL * elem <= 96 * 1024) w *= 2;
  return w;
}

template <typename T, int P>
cudaError_t launch_strfunc(const T* v, int n, int axis, double* part, int nblocks, cudaStream_t s) {
  const int W = sf_tile_width(n, sizeof(T));
  const int ns = n / 2 + 1, PL = n + ns + 3 * SF_R;
  size_t smem = (size_t)W * PL * sizeof(T);
  const size_t red = (size_t)SF_THREADS * SF_R * sizeof(double);
  if (smem < red) smem = red;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_strfunc<T, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_strfunc<T, P><<<nblocks, SF_THREADS, smem, s>>>(v, n, axis, W, n * n / W, part);
  return cudaGetLastError();
}

template <typename T>
cudaError_t strfunc_order(int order, const T* v, int n, int axis, double* part, int nblocks, cudaStream_t s) {
  switch (order) {
    case 1: return launch_strfunc<T, 1>(v, n, axis, part, nblocks, s);
    case 2: return launch_strfunc<T, 2>(v, n, axis, part, nblocks, s);
    case 3: return launch_strfunc<T, 3>(v, n, axis, part, nblocks, s);
    case 4: return launch_strfunc<T, 4>(v, n, axis, part, nblocks, s);
    case 5: return launch_strfunc<T, 5>(v, n, axis, part, nblocks, s);
    case 6: return launch_strfunc<T, 6>(v, n, axis, part, nblocks, s);
    case 7: return launch_strfunc<T, 7>(v, n, axis, part, nblocks, s);
    default: return launch_strfunc<T, 8>(v, n, axis, part, nblocks, s);
  }
}

template <typename T>
gp_status strfunc_impl(gp_plan* p, int field, const cpx<T>* psi, int order, double* out, int nr) {
  FieldPlan& F = p->f[field];
  const long long npts = F.npts;
  const int n = F.n, ns = n / 2 + 1;
  cudaStream_t s = p->stream;
  const size_t fb = (size_t)npts * sizeof(cpx<T>);
  const int W = sf_tile_width(n, sizeof(T));
  const int ntiles = n * n / W;
  const int nblocks = ntiles < 2 * 152 ? ntiles : 2 * 152;
  const size_t vz_bytes = ((size_t)npts * sizeof(T) + 255) / 256 * 256;
  gp_status st = ensure_ws(p, field, 4 * fb + vz_bytes + ((size_t)nblocks * ns + 3 * ns) * sizeof(double));
  if (st != GP_OK) return st;
  cpx<T>* w0 = (cpx<T>*)F.ws;
  cpx<T>* w1 = w0 + npts;
  cpx<T>* w2 = w1 + npts;
  cpx<T>* w3 = w2 + npts;
  T* vx = (T*)w0;                 // the spectrum in w0 is not needed once the gradients exist
  T* vy = vx + npts;
  T* vz = (T*)(w3 + npts);
  double* part = (double*)((unsigned char*)vz + vz_bytes);
  double* sums = part + (size_t)nblocks * ns;
  GP_CUDA(p, cudaMemcpyAsync(w0, psi, fb, cudaMemcpyDeviceToDevice, s));
  cpx<T>* all[4] = {w0, w1, w2, w3};
  auto transform = [&](int first, int count, bool inverse) -> cudaError_t {
    if constexpr (sizeof(T) == 4) return fft3_many(p, F, all + first, count, inverse, s);
    for (int k = first; k < first + count; ++k) {
      cudaError_t e = fft3<T>(F, all[k], inverse, s);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  };
  GP_CUDA(p, transform(0, 1, false));
  const unsigned g = sf_grid(npts);
  k_sf_grad<T><<<g, 256, 0, s>>>(w0, w1, w2, w3, n);
  GP_CUDA(p, cudaGetLastError());
  GP_CUDA(p, transform(1, 3, true));
  k_sf_velocity<T><<<g, 256, 0, s>>>(psi, w1, w2, w3, vx, vy, vz, npts, F.alpha);
  GP_CUDA(p, cudaGetLastError());
  const T* comp[3] = {vx, vy, vz};
  for (int j = 0; j < 3; ++j) {
    GP_CUDA(p, strfunc_order<T>(order, comp[j], n, j, part, nblocks, s));
    k_sf_sum_blocks<<<(ns + 127) / 128, 128, 0, s>>>(part, nblocks, ns, sums + (size_t)j * ns);
    GP_CUDA(p, cudaGetLastError());
  }
  std::vector<double> h((size_t)3 * ns);
  GP_CUDA(p, cudaMemcpyAsync(h.data(), sums, h.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
  GP_CUDA(p, cudaStreamSynchronize(s));
  st = check_status(p);
  if (st != GP_OK) return st;
  const double dn = (double)npts;
  for (int j = 0; j < 3; ++j)
    for (int q = 0; q < ns; ++q) {
      const double val = h[(size_t)j * ns + q] / dn;
      if (!std::isfinite(val)) return fail(p, GP_ERR_NONFINITE, "gp_structure_function: non-finite velocity");
      out[(size_t)j * nr + q] = val;
    }
  return GP_OK;
}

}  // namespace
}  // namespace gp

using namespace gp;

extern "C" gp_status gp_structure_function(gp_plan* p, int field, const void* psi, int order, double* out, int nr) {
  if (!p) return GP_ERR_INVALID_ARG;
  if (field < 0 || field >= (int)p->f.size()) return fail(p, GP_ERR_INVALID_ARG, "gp_structure_function: field index");
  if (!psi || ((uintptr_t)psi & 15) || !out) return fail(p, GP_ERR_INVALID_ARG, "gp_structure_function: pointer");
  if (order < 1 || order > SF_MAX_ORDER) return fail(p, GP_ERR_INVALID_ARG, "gp_structure_function: order not in 1..8");
  if (nr < p->f[field].n / 2 + 1) return fail(p, GP_ERR_INVALID_ARG, "gp_structure_function: nr < N/2 + 1");
  if (p->f[field].fp64) return strfunc_impl<double>(p, field, (const cpx<double>*)psi, order, out, nr);
  return strfunc_impl<float>(p, field, (const cpx<float>*)psi, order, out, nr);
}

// gp_reduce.cuh -- float64 sums of per-point terms, shared by the diagnostics and the
// imaginary-time preparation.
#pragma once
#include "gp_fft.cuh"

namespace gp {

constexpr double EPS_RHO = 1e-12;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// block-reduce NA partial sums; the block's sums go to part[blockIdx.x * NA + a].  The
// per-block sums are added up by k_reduce in a fixed order: no float64 atomics on one
// address (they serialise), and the totals are the same on every call.
template <int NA> __device__ __forceinline__ void block_store(double (&v)[NA], double* part) {
  __shared__ double red[NA][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int a = 0; a < NA; ++a) {
    double s = warp_sum(v[a]);
    if (lane == 0) red[a][w] = s;
  }
  __syncthreads();
  if (w == 0) {
    const int nw = blockDim.x >> 5;
#pragma unroll
    for (int a = 0; a < NA; ++a) {
      double s = lane < nw ? red[a][lane] : 0.0;
      s = warp_sum(s);
      if (lane == 0) part[blockIdx.x * NA + a] = s;
    }
  }
}

// acc[a] = sum over blocks b of part[b * na + a]; one block of 256 threads
static __global__ void k_reduce(const double* __restrict__ part, int nblocks, int na, double* acc) {
  __shared__ double red[8][8];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int a = 0; a < na; ++a) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) s += part[b * na + a];
    s = warp_sum(s);
    if (lane == 0) red[a][w] = s;
  }
  __syncthreads();
  if (threadIdx.x < na) {
    double s = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += red[threadIdx.x][q];
    acc[threadIdx.x] = s;
  }
}


// acc[0] = max over blocks b of part[b] (non-negative values)
static __global__ void k_reduce_max(const double* __restrict__ part, int nblocks, double* acc) {
  __shared__ double red[32];
  double m = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) m = fmax(m, part[b]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 1; q < (int)(blockDim.x >> 5); ++q) m = fmax(m, red[q]);
    *acc = m;
  }
}

// target = sum / npts (the mean that a renormalisation keeps)
static __global__ void k_scale_to_mean(const double* sum, double* target, double npts) { *target = *sum / npts; }

// Sums of NA per-point terms.  float fields: each term is formed in float32 and added to a
// float32 partial that is moved into a float64 sum every 32 points (a partial of at most 32
// terms carries a relative rounding of at most 32 * 2^-24, and nearly all of the float64 rate,
// which this GPU has little of, is avoided); float64 fields: float64 throughout.
template <typename T, int NA> struct Sums {
  double d[NA] = {};
  T f[NA] = {};
  int k = 0;
  __device__ __forceinline__ void add(const T (&v)[NA]) {
    if constexpr (sizeof(T) == 8) {
#pragma unroll
      for (int a = 0; a < NA; ++a) d[a] += v[a];
    } else {
#pragma unroll
      for (int a = 0; a < NA; ++a) f[a] += v[a];
      if (++k == 32) flush();
    }
  }
  __device__ __forceinline__ void flush() {
#pragma unroll
    for (int a = 0; a < NA; ++a) {
      d[a] += (double)f[a];
      f[a] = T(0);
    }
    k = 0;
  }
};

// rho - 1 = a.x^2 + a.y^2 - 1 to about one rounding of the result, in the field's precision:
// rounding rho first would leave an absolute error of one ulp of 1 in rho - 1, a large relative
// one for a nearly uniform density.  float: the two squares split into value + exact error
// (fma), their sum by Knuth's two-sum, then 1 subtracted from the sum (exact for rho in
// [1/2, 2], Sterbenz) and the three error terms added.  (float64 arithmetic would do the same
// but runs at a small fraction of the float32 rate on this GPU.)
template <typename T> __device__ __forceinline__ T rho_minus_one(cpx<T> a, T* rho) {
  if constexpr (sizeof(T) == 8) {
    *rho = a.x * a.x + a.y * a.y;
    return *rho - 1.0;
  } else {
    const float px = a.x * a.x, ex = fmaf(a.x, a.x, -px);
    const float py = a.y * a.y, ey = fmaf(a.y, a.y, -py);
    const float s = px + py, bp = s - px, es = (px - (s - bp)) + (py - bp);
    *rho = s;
    return (s - 1.0f) + (es + (ex + ey));
  }
}

// |psi|^2 below this is treated as zero (1e-12; for float the smallest float not below 1e-12,
// so that the float comparison agrees with the float64 one)
template <typename T> __device__ __forceinline__ T eps_rho() {
  if constexpr (sizeof(T) == 8) return EPS_RHO;
  else return __int_as_float(0x2b8cbccd);
}

// signed wavenumber of grid index i; the derivative's, with the Nyquist mode set to 0
__device__ __forceinline__ int wavenumber(int i, int n) { return i < (n + 1) / 2 ? i : i - n; }
__device__ __forceinline__ int wavenumber_d(int i, int n) { return (2 * i == n) ? 0 : wavenumber(i, n); }

// grid coordinates of linear index i (fits in 32 bits: N <= 1024)
__device__ __forceinline__ void coords3(unsigned i, unsigned n, int& ix, int& iy, int& iz) {
  const unsigned r = i / n;
  ix = (int)(i - r * n);
  iz = (int)(r / n);
  iy = (int)(r - (unsigned)iz * n);
}

// shell index floor(|k| + 1/2) of the integer |k|^2 = K, exactly: the b with (2b-1)^2 <= 4K < (2b+1)^2
__device__ __forceinline__ int shell_of(int K) {
  int b = (int)(sqrtf((float)K) + 0.5f);
  while ((2 * b + 1) * (2 * b + 1) <= 4 * K) ++b;
  while (b > 0 && (2 * b - 1) * (2 * b - 1) > 4 * K) --b;
  return b;
}

}  // namespace gp

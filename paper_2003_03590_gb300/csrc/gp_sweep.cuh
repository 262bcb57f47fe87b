// gp_sweep.cuh -- one HBM sweep over an N^3 field: 1D transforms along one axis with the
// pointwise sub-flows of the split step (Sec. 4.3) fused into the same pass.
//
// Ops (applied to every pencil of the chosen axis, in place):
//   OP_FWD        forward DFT
//   OP_INV        inverse DFT (with 1/N)
//   OP_INV_N_FWD  inverse DFT, nonlinear flow N(s), forward DFT
//   OP_N_FWD      N(s), forward DFT
//   OP_INV_N      inverse DFT, N(s)
//   OP_FWD_K_INV  forward DFT, kinetic flow K(s) (needs every other axis already in
//                 Fourier space), inverse DFT
// N(s):  psi <- exp(-i (beta s) (|psi|^2 - c)) psi                 (exact nonlinear flow)
// K(s):  psi_k <- exp(-i alpha s (kx^2 + ky^2 + kz^2)) psi_k          (exact kinetic flows)
// The kinetic factor is applied with an exact magnitude (unit_rotate) and the 1/N^3
// of the inverse transform is folded into the same multiplication (the inverse
// sweeps that follow it in a step then do not scale).
#pragma once
#include "gp_fft.cuh"

namespace gp {

enum SweepOp : int { OP_FWD = 1, OP_INV = 2, OP_INV_N_FWD = 3, OP_N_FWD = 4, OP_INV_N = 5, OP_FWD_K_INV = 6,
                     OP_PLANE = 7 };   // OP_PLANE: forward y, OP_FWD_K_INV along x, inverse y (gp_plane.cuh)

constexpr int GP_MAXB = 32;  // fields of one shape handled by one launch (blockIdx.y)

template <typename T> struct SweepArgs {
  cpx<T>* psi[GP_MAXB];     // device fields, N^3 each, [z][y][x]; field blockIdx.y
  int count;                // number of fields in psi[]
  const tw_t<T>* tw_fwd;    // forward Stockham twiddles for length N
  const tw_t<T>* tw_inv;    // inverse Stockham twiddles for length N
  const cpx<T>* ek;         // float64: exp(-i alpha s k^2) by grid index, length N (OP_FWD_K_INV)
  const float4* ekx;        // float32: the same as hi/lo pairs, length N
  const float4* ek2;        // float32: E[i1] E[i2] / N^3 as hi/lo pairs, index i2 * N + i1
  KConst k_norm;            // float64: factor applied with K, 1/N^3
  T nl_coef;                // beta * s of N(s)
  T nl_shift;               // c of N(s): 1 (eq-gpe-num) or 0
  int op;
  int axis;                 // 0: x (contiguous rows), 1: y, 2: z (strided pencils)
  int scale_inv;            // 1: inverse ops multiply by 1/N; 0: normalisation done with K
};

// K factor of one element (float64): E[kx] (E[ky] E[kz]) from the table of exp(-i alpha s k^2), then 1/N^3.
__device__ __forceinline__ double2 kinetic_apply(double2 x, double2 e_other, double2 e_pos, KConst norm) {
  const double2 y = cmul(x, cmul(e_pos, e_other));
  return double2{y.x * norm.v, y.y * norm.v};
}

template <typename V> __device__ __forceinline__ V kscale(V x, KConst k) { return V{kmul(x.x, k), kmul(x.y, k)}; }

// pencils per CTA (16: rows of 128 bytes, the fewest rows per byte read of a z-pencil tile, whose
// rows lie one z-plane apart; float64 at 1024: 8, for the registers)
template <typename T, int L> __host__ __device__ constexpr int strided_batch() {
  return (L % 16 == 0) ? ((sizeof(T) == 8 && L >= 1024) ? 8 : 16) : (L % 8 == 0 ? 8 : 4);
}
// float32 kernels whose threads hold 32 elements each (L >= 512) run with register caps for
// several CTAs per SM (see rcap_blocks); their x-row CTAs have 128 threads, four per SM
template <typename T, int L> __host__ __device__ constexpr bool rcapped() { return sizeof(T) == 4 && Plan<L>::E >= 32; }
template <typename T, int L> __host__ __device__ constexpr int contig_batch() {
  int b = (rcapped<T, L>() ? 128 : 256) / (L / Plan<L>::E);
  b = b > 64 ? 64 : (b < 1 ? 1 : b);
  while ((L * L) % b) b /= 2;
  return b;
}
template <int L> __host__ __device__ constexpr int contig_pitch() { return L + (L >= 16 ? L / 16 : 1); }
// CTAs per SM the registers of the capped one-tile-per-CTA kernels must allow (y/z: 256 threads,
// two per SM, or at 1024 512 threads, one; x: 128 threads, four per SM).  Without a cap the compiler keeps all of a thread's 32
// loads in flight at once and uses so many registers (~175) that one 8-warp CTA fills the SM
// (measured at 512^3: z N-forward 752 us uncapped, 452 us capped).  Kernels of shorter lengths keep
// the compiler's own choice (naming a minimum of one CTA per SM lifts its default limit and made
// the 256-point kernels twice as slow).
template <typename T, int L> __host__ __device__ constexpr int rcap_blocks(bool contig) {
  return contig ? 4 : (strided_batch<T, L>() * (L / Plan<L>::E) >= 512 ? 1 : 2);
}

struct LayStrided {  // [pos][pencil]
  int B;
  __device__ __forceinline__ int operator()(int p, int pos) const { return pos * B + p; }
};
template <int L> struct LayContig {  // [pencil][pos] with one pad element every 16
  __device__ __forceinline__ int operator()(int p, int pos) const {
    return p * contig_pitch<L>() + pos + (L >= 16 ? (pos >> 4) : 0);
  }
};

// cos(x) - 1 and sin(x) for |x| <= 1/2 by their Taylor series (terms to x^10 and x^9; the first
// omitted term is below 2e-11).  cos(x) - 1 keeps full relative precision for small x: rounding
// cos(x) itself to float would give exactly 1 for |x| < 2.4e-4 and |w|^2 = 1 + x^2, a bias.
__device__ __forceinline__ void sincos_m1_small(float x, float* s, float* cm1) {
  const float z = x * x;
  const float pc = fmaf(z, fmaf(z, fmaf(z, fmaf(z, -2.7557319e-7f, 2.4801587e-5f), -1.3888889e-3f), 4.1666668e-2f), -0.5f);
  *cm1 = z * pc;
  const float ps = fmaf(z, fmaf(z, fmaf(z, 2.7557319e-6f, -1.9841270e-4f), 8.3333333e-3f), -0.16666667f);
  *s = fmaf(x * z, ps, x);
}

// N(s): a * exp(-i coef (|a|^2 - shift)).  For a small phase the product is formed as
// a + [a (cos - 1 - i sin)]: the two small terms of each component are summed first and the
// component is added last, in one rounding.  Adding the sine term to the component first and
// the shrink a (cos - 1) after it would round the shrink away whenever it is below half an ulp
// of the component -- with the same sign at every step at points where |a|^2 stays near the
// shift, a steady gain of mass (emulated: 1.1e-8 per step at ||a|^2 - 1| = 4e-3).
// The large-phase branch (|phase| > 1/2, i.e. ||a|^2 - shift| > 1/(2 coef): rare) is kept out of
// line.  Inlined at every element of a thread's unrolled pencil data it would repeat sincosf's
// argument reduction dozens of times in the kernel, and the instruction fetch of the common
// small-phase path would then miss in the instruction cache.
static __device__ __noinline__ float2 nonlinear_large(float2 a, float ph) {
  float sn, cs;
  sincosf(ph, &sn, &cs);
  return unit_rotate(a, cs, -sn);
}

template <typename V, typename S> __device__ __forceinline__ V nonlinear(V a, S coef, S shift) {
  S r2;
  if constexpr (sizeof(S) == 4) r2 = fmaf(a.x, a.x, a.y * a.y);   // explicit: see rotk
  else r2 = a.x * a.x + a.y * a.y;
  S ph = coef * (r2 - shift);
  S sn, cs;
  if constexpr (sizeof(S) == 4) {
    if (fabsf(ph) <= 0.5f) {
      float cm1;
      sincos_m1_small(ph, &sn, &cm1);
      const float ur = fmaf(a.y, sn, __fmul_rn(a.x, cm1));
      const float ui = fmaf(-a.x, sn, __fmul_rn(a.y, cm1));
      return V{__fadd_rn(a.x, ur), __fadd_rn(a.y, ui)};
    }
    return nonlinear_large(a, ph);
  } else {
    sincos(ph, &sn, &cs);
    return V{a.x * cs + a.y * sn, a.y * cs - a.x * sn};
  }
}

// N(s) on all E elements of a thread (float32 in pairs).  Two elements at a time through packed
// FP32x2 operations whose lanes round exactly as the scalar ones of nonlinear(): the same
// results, about half the instructions of the small-phase path.  A pair with a large phase
// takes the scalar path for both.
__device__ __forceinline__ float2 f2c(float c) { return float2{c, c}; }
__device__ __forceinline__ void nonlinear_pair(float2& a, float2& b, float coef, float shift) {
  const float2 X{a.x, b.x}, Y{a.y, b.y};
  const float2 r2 = __ffma2_rn(X, X, __fmul2_rn(Y, Y));
  const float2 ph = __fmul2_rn(f2c(coef), __fadd2_rn(r2, f2c(-shift)));
  if (fabsf(ph.x) <= 0.5f && fabsf(ph.y) <= 0.5f) {
    const float2 z = __fmul2_rn(ph, ph);
    float2 pc = __ffma2_rn(z, f2c(-2.7557319e-7f), f2c(2.4801587e-5f));
    pc = __ffma2_rn(z, pc, f2c(-1.3888889e-3f));
    pc = __ffma2_rn(z, pc, f2c(4.1666668e-2f));
    pc = __ffma2_rn(z, pc, f2c(-0.5f));
    const float2 cm1 = __fmul2_rn(z, pc);
    float2 ps = __ffma2_rn(z, f2c(2.7557319e-6f), f2c(-1.9841270e-4f));
    ps = __ffma2_rn(z, ps, f2c(8.3333333e-3f));
    ps = __ffma2_rn(z, ps, f2c(-0.16666667f));
    const float2 sn = __ffma2_rn(__fmul2_rn(ph, z), ps, ph);
    const float2 ur = __ffma2_rn(Y, sn, __fmul2_rn(X, cm1));
    const float2 ui = __ffma2_rn(X, __fmul2_rn(sn, f2c(-1.0f)), __fmul2_rn(Y, cm1));
    const float2 rx = __fadd2_rn(X, ur), ry = __fadd2_rn(Y, ui);
    a = float2{rx.x, ry.x};
    b = float2{rx.y, ry.y};
  } else {
    a = nonlinear(a, coef, shift);
    b = nonlinear(b, coef, shift);
  }
}
template <int E, typename V, typename S> __device__ __forceinline__ void nonlinear_all(V* v, S coef, S shift) {
  if constexpr (sizeof(S) == 4 && E % 2 == 0) {
#pragma unroll
    for (int e = 0; e < E; e += 2) nonlinear_pair(v[e], v[e + 1], coef, shift);
  } else {
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = nonlinear(v[e], coef, shift);
  }
}

template <typename T, int L, bool INV, class GetAddr>
__device__ __forceinline__ void load_pattern(cpx<T>* v, int t, const GetAddr& addr) {
  constexpr int E = Plan<L>::E;
#pragma unroll
  for (int e = 0; e < E; ++e) v[e] = *addr(in_pos<L, INV>(e, t));
}
template <typename T, int L, bool INV, class GetAddr>
__device__ __forceinline__ void store_pattern(const cpx<T>* v, int t, const GetAddr& addr) {
  constexpr int E = Plan<L>::E;
#pragma unroll
  for (int e = 0; e < E; ++e) *addr(out_pos<L, INV>(e, t)) = v[e];
}

// Body shared by both tile shapes.  (i1, i2) are the grid indices of the pencil's two other
// coordinates (only used by OP_FWD_K_INV).
// TILE_IN_SMEM: the tile addressed by addr() lives in the same shared memory that the
// passes use for their exchanges, so the block synchronises after reading it (and, with
// warp-private exchanges, before writing it back).  WARP_X: see fft_regs.
template <int OP, typename T, int L, int B, class Lay, class GetAddr, bool TILE_IN_SMEM = false, bool WARP_X = false,
          bool TW_SH = false, int NB = 0>
__device__ __forceinline__ void sweep_op_body(const SweepArgs<T>& a, int t, int p, cpx<T>* sm, const Lay& lay,
                                              const GetAddr& addr, int i1, int i2) {
  using V = cpx<T>;
  constexpr int E = Plan<L>::E;
  constexpr KConst inv_l = kconst(1.0 / L);
  constexpr bool IN_INV = OP == OP_INV || OP == OP_INV_N || OP == OP_INV_N_FWD;
  constexpr bool OUT_INV = OP == OP_INV || OP == OP_INV_N || OP == OP_FWD_K_INV;
  const bool sc = a.scale_inv != 0;
  // the row's kinetic factor of (y, z) is read before the forward transform, so that its latency
  // is hidden behind the transform's arithmetic
  [[maybe_unused]] float4 eo{};
  if constexpr (OP == OP_FWD_K_INV && sizeof(T) == 4) eo = __ldg(a.ek2 + i2 * L + i1);
  V v[E];
  load_pattern<T, L, IN_INV>(v, t, addr);
  if constexpr (TILE_IN_SMEM) bsync<NB>();
  if constexpr (OP == OP_N_FWD) nonlinear_all<E>(v, a.nl_coef, a.nl_shift);
  if constexpr (OP == OP_FWD || OP == OP_N_FWD || OP == OP_FWD_K_INV)
    fft_regs<T, L, B, Lay, false, WARP_X, TW_SH, NB>(v, t, p, sm, lay, a.tw_fwd);
  if constexpr (IN_INV) {
    fft_regs<T, L, B, Lay, true, WARP_X, TW_SH, NB>(v, t, p, sm, lay, a.tw_inv);
    if constexpr (OP == OP_INV) {
      if (sc) {
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = kscale(v[e], inv_l);
      }
    } else {
      if (sc) {
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = kscale(v[e], inv_l);
      }
      nonlinear_all<E>(v, a.nl_coef, a.nl_shift);
    }
  }
  if constexpr (OP == OP_INV_N_FWD) {
    xsync<WARP_X, NB>();  // shared memory is reused by the forward passes
    fft_regs<T, L, B, Lay, false, WARP_X, TW_SH, NB>(v, t, p, sm, lay, a.tw_fwd);
  }
  if constexpr (OP == OP_FWD_K_INV) {
    if constexpr (sizeof(T) == 4) {
      // two products by factors exact to float64 (hi + lo), each rounded once: the magnitude
      // of the field is not biased by the kinetic factor, which is the same for a given k in
      // every step
#pragma unroll
      for (int e = 0; e < E; ++e) v[e] = twmul_k(twmul_k(v[e], __ldg(a.ekx + out_pos<L, false>(e, t))), eo);
    } else {
      const V eo = cmul(__ldg(a.ek + i1), __ldg(a.ek + i2));
#pragma unroll
      for (int e = 0; e < E; ++e) v[e] = kinetic_apply(v[e], eo, __ldg(a.ek + out_pos<L, false>(e, t)), a.k_norm);
    }
    xsync<WARP_X, NB>();
    fft_regs<T, L, B, Lay, true, WARP_X, TW_SH, NB>(v, t, p, sm, lay, a.tw_inv);
  }
  if constexpr (TILE_IN_SMEM && WARP_X) bsync<NB>();
  store_pattern<T, L, OUT_INV>(v, t, addr);
}

// y or z pencils: a CTA owns B consecutive x of one (z) or (y) line.  One kernel per
// operation: a kernel holds only the code it runs (smaller than one with every operation
// behind a run-time switch, which missed in the instruction cache).
template <typename T, int L, int OP, int NB = 0>
__device__ __forceinline__ void strided_tile(const SweepArgs<T>& a, long tile, cpx<T>* psi, int tid, cpx<T>* sm) {
  // tile: B consecutive x of one (z) line for y pencils, of one (y) line for z pencils; tid: the
  // thread within the NB (0: all) threads that share the tile and its exchange memory sm
  using V = cpx<T>;
  constexpr int B = strided_batch<T, L>();
  const int p = tid % B, t = tid / B;
  const long st = (a.axis == 1) ? (long)L : (long)L * L;    // stride along the pencil
  const long sc = (a.axis == 1) ? (long)L * L : (long)L;    // stride of the other coordinate
  const int x0 = (int)(tile % (L / B)) * B;
  const int c = (int)(tile / (L / B));
  V* base = psi + x0 + p + (long)c * sc;
  auto addr = [&](int pos) { return base + (long)pos * st; };
  LayStrided lay{B};
  sweep_op_body<OP, T, L, B, LayStrided, decltype(addr), false, false, false, NB>(a, t, p, sm, lay, addr, x0 + p, c);
}
template <typename T, int L, int OP>
__global__ void __launch_bounds__(strided_batch<T, L>() * (L / Plan<L>::E)) k_sweep_strided(SweepArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  strided_tile<T, L, OP>(a, blockIdx.x, a.psi[blockIdx.y], threadIdx.x, reinterpret_cast<cpx<T>*>(smraw));
}
template <typename T, int L, int OP>
__global__ void __launch_bounds__(strided_batch<T, L>() * (L / Plan<L>::E), rcap_blocks<T, L>(false))
    k_sweep_strided_rc(SweepArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  strided_tile<T, L, OP>(a, blockIdx.x, a.psi[blockIdx.y], threadIdx.x, reinterpret_cast<cpx<T>*>(smraw));
}

// x rows: a tile is B consecutive rows (y, z); the exchanges of a row stay within one warp.
template <typename T, int L, int OP>
__device__ __forceinline__ void contig_tile(const SweepArgs<T>& a, long tile, cpx<T>* psi, int tid, cpx<T>* sm) {
  using V = cpx<T>;
  constexpr int TP = L / Plan<L>::E;
  constexpr int B = contig_batch<T, L>();
  const int p = tid / TP, t = tid % TP;
  const long row = tile * B + p;
  V* base = psi + row * L;
  auto addr = [&](int pos) { return base + pos; };
  LayContig<L> lay;
  sweep_op_body<OP, T, L, B, LayContig<L>, decltype(addr), false, (TP <= 32)>(a, t, p, sm, lay, addr,
                                                                              (int)(row % L), (int)(row / L));
}
template <typename T, int L, int OP>
__global__ void __launch_bounds__(contig_batch<T, L>() * (L / Plan<L>::E)) k_sweep_contig(SweepArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  contig_tile<T, L, OP>(a, blockIdx.x, a.psi[blockIdx.y], threadIdx.x, reinterpret_cast<cpx<T>*>(smraw));
}
template <typename T, int L, int OP>
__global__ void __launch_bounds__(contig_batch<T, L>() * (L / Plan<L>::E), rcap_blocks<T, L>(true))
    k_sweep_contig_rc(SweepArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  contig_tile<T, L, OP>(a, blockIdx.x, a.psi[blockIdx.y], threadIdx.x, reinterpret_cast<cpx<T>*>(smraw));
}

// Operations each axis supports: y/z pencils every operation but FWD_K_INV; x rows forward,
// inverse and forward-K-inverse.  Anything else is an invalid launch.
#define GP_STRIDED_OPS(X) X(OP_FWD) X(OP_INV) X(OP_N_FWD) X(OP_INV_N) X(OP_INV_N_FWD)
#define GP_CONTIG_OPS(X) X(OP_FWD) X(OP_INV) X(OP_FWD_K_INV)

template <typename T, int L> struct SweepLaunch {
  static constexpr int TP = L / Plan<L>::E;
  static constexpr int BS = strided_batch<T, L>();
  static constexpr int BC = contig_batch<T, L>();
  static constexpr bool RC = rcapped<T, L>();
  static size_t smem_strided() { return sizeof(cpx<T>) * (size_t)L * BS; }
  static size_t smem_contig() { return sizeof(cpx<T>) * (size_t)contig_pitch<L>() * BC; }
  // the shared-memory limit of every operation's kernel, set together on the first launch of
  // this length (never inside a stream capture: a step's first sweeps run directly)
  static void set_attributes() {
    static bool done = false;
    if (done) return;
    const size_t sc = smem_contig(), ss = smem_strided();
#define GP_ATTR_C(OPV)                                                                                        \
  if constexpr (RC) cudaFuncSetAttribute(k_sweep_contig_rc<T, L, OPV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sc); \
  else if (sc > 48 * 1024) cudaFuncSetAttribute(k_sweep_contig<T, L, OPV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sc);
#define GP_ATTR_S(OPV)                                                                                        \
  if constexpr (RC) cudaFuncSetAttribute(k_sweep_strided_rc<T, L, OPV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ss); \
  else if (ss > 48 * 1024) cudaFuncSetAttribute(k_sweep_strided<T, L, OPV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ss);
    GP_CONTIG_OPS(GP_ATTR_C)
    GP_STRIDED_OPS(GP_ATTR_S)
#undef GP_ATTR_C
#undef GP_ATTR_S
    done = true;
  }
  template <int OP> static cudaError_t contig(const SweepArgs<T>& a, cudaStream_t s) {
    const size_t sm = smem_contig();
    set_attributes();
    const long rows = (long)L * L;
    const dim3 grid((unsigned)(rows / BC), (unsigned)a.count);
    if constexpr (RC) k_sweep_contig_rc<T, L, OP><<<grid, BC * TP, sm, s>>>(a);
    else k_sweep_contig<T, L, OP><<<grid, BC * TP, sm, s>>>(a);
    return cudaGetLastError();
  }
  template <int OP> static cudaError_t strided(const SweepArgs<T>& a, cudaStream_t s) {
    const size_t sm = smem_strided();
    set_attributes();
    const long tiles = (long)(L / BS) * L;
    const dim3 grid((unsigned)tiles, (unsigned)a.count);
    if constexpr (RC) k_sweep_strided_rc<T, L, OP><<<grid, BS * TP, sm, s>>>(a);
    else k_sweep_strided<T, L, OP><<<grid, BS * TP, sm, s>>>(a);
    return cudaGetLastError();
  }
  static cudaError_t launch(const SweepArgs<T>& a, cudaStream_t s) {
#define GP_OP_CASE_C(OPV) \
  case OPV: return contig<OPV>(a, s);
#define GP_OP_CASE_S(OPV) \
  case OPV: return strided<OPV>(a, s);
    if (a.axis == 0) {
      switch (a.op) { GP_CONTIG_OPS(GP_OP_CASE_C) default: return cudaErrorInvalidValue; }
    }
    switch (a.op) { GP_STRIDED_OPS(GP_OP_CASE_S) default: return cudaErrorInvalidValue; }
#undef GP_OP_CASE_C
#undef GP_OP_CASE_S
  }
};

}  // namespace gp

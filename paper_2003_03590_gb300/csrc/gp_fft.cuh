// gp_fft.cuh -- register-resident Stockham FFT along one axis of a tile of pencils.
//
// The pseudo-spectral step of Sec. 4.3 (eq:adi_looptime) needs 1D DFTs along
// x, y and z of an N^3 complex field, unnormalised forward
//   X[k] = sum_j x[j] exp(-2 pi i j k / N)
// and inverse with exp(+...) and a 1/N factor.  A CTA owns B pencils of
// length L.  Each thread owns E = L / TP elements of one pencil in registers;
// a radix-R pass turns those into E/R radix-R butterflies, and consecutive
// passes exchange data through shared memory.  The pass with radix R and
// "span" NS (product of the radices already applied) follows the autosort
// (Stockham) indexing: butterfly j reads x[j + r L/R] (r < R), multiplies by
// w^(r (j mod NS)) with w = exp(-+ 2 pi i / (NS R)), does a radix-R DFT and
// writes y[(j / NS) NS R + (j mod NS) + r NS].  The first pass reads and the
// last pass writes natural order, so
//   * the inverse transform uses the radices in reverse order; its last pass
//     then leaves in registers exactly the element pattern the first forward
//     pass reads, and a pointwise operation between them (the nonlinear phase
//     of Sec. 4.3) costs no data movement;
//   * the same holds between a forward transform and an inverse one (the
//     kinetic propagator of Sec. 4.3).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace gp {

template <typename T> struct CT;
template <> struct CT<float> { using v = float2; };
template <> struct CT<double> { using v = double2; };
template <typename T> using cpx = typename CT<T>::v;

template <typename V> __device__ __forceinline__ V cadd(V a, V b) { return V{a.x + b.x, a.y + b.y}; }
template <typename V> __device__ __forceinline__ V csub(V a, V b) { return V{a.x - b.x, a.y - b.y}; }
// float32: one packed FP32x2 instruction per complex operation.  Each lane rounds exactly as the
// scalar operation would (b * -1 is exact, so fma(b, -1, a) is a - b rounded once).
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return __ffma2_rn(b, float2{-1.0f, -1.0f}, a); }
__device__ __forceinline__ float2 swap2(float2 a) { return float2{a.y, a.x}; }
template <typename V> __device__ __forceinline__ V cmul(V a, V b) {
  return V{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename V> __device__ __forceinline__ V cmulconj(V a, V b) {  // a * conj(b)
  return V{a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y};
}
template <typename V, typename S> __device__ __forceinline__ V cscale(V a, S s) { return V{a.x * s, a.y * s}; }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return __fmul2_rn(a, float2{s, s}); }
template <typename V> __device__ __forceinline__ V cneg(V a) { return V{-a.x, -a.y}; }
// a * (-i) for the forward direction, a * (+i) for the inverse one
template <bool INV, typename V> __device__ __forceinline__ V mul_mi(V a) {
  return INV ? V{-a.y, a.x} : V{a.y, -a.x};
}
// ---------------------------------------------------------------- unbiased constants
// A float32 constant is carried as hi + lo (hi = nearest float, lo = the rest) and
// multiplied as fma(x, hi, x * lo): the product is then rounded once, without the
// fixed relative error of the rounded constant.  A fixed error would bias |w|^2
// the same way in every step and make the mass (conserved exactly by the
// scheme) drift linearly in time; the compensated product leaves only unbiased
// round-off.  float64 uses the constant directly.
struct KConst {
  double v;
  float hi, lo;
};
__host__ __device__ constexpr KConst kconst(double v) {
  return KConst{v, (float)v, (float)(v - (double)(float)v)};
}
__device__ __forceinline__ float kmul(float x, KConst k) { return fmaf(x, k.hi, x * k.lo); }
__device__ __forceinline__ double kmul(double x, KConst k) { return x * k.v; }
// both lanes of a float2 times the constants sa * k (lane 0) and sb * k (lane 1), sa, sb = +-1:
// per lane fma(x, +-hi, x * +-lo), the negation of kmul(x, k) when the sign is -1
__device__ __forceinline__ float2 kmul2(float2 x, KConst k, float sa, float sb) {
  return __ffma2_rn(x, float2{sa * k.hi, sb * k.hi}, __fmul2_rn(x, float2{sa * k.lo, sb * k.lo}));
}

// a * (c - i s) forward, a * (c + i s) inverse, for constants c = cos(theta), s = sin(theta)
// (float: every product-sum is an explicit fma, so that the rounding does not depend on how the
// compiler would contract a*b + c*d in a given kernel -- all kernel variants agree bitwise)
// NEG: the negated product (float: the constants negated, which rounds to exactly the negation).
template <bool INV, typename V, bool NEG = false> __device__ __forceinline__ V rotk(V a, KConst c, KConst s) {
  if constexpr (sizeof(a.x) == 4) {
    // lanes (re, im): lo = a c.lo + (+-a.y, -+a.x) s.lo;  result = a c.hi + ((+-a.y, -+a.x) s.hi + lo)
    const float2 b = swap2(a);
    const float sg = INV ? -1.0f : 1.0f, ng = NEG ? -1.0f : 1.0f;
    const float2 lo = __ffma2_rn(a, float2{ng * c.lo, ng * c.lo}, __fmul2_rn(b, float2{ng * sg * s.lo, -ng * sg * s.lo}));
    return __ffma2_rn(a, float2{ng * c.hi, ng * c.hi}, __ffma2_rn(b, float2{ng * sg * s.hi, -ng * sg * s.hi}, lo));
  } else {
    const V r = INV ? V{a.x * c.v - a.y * s.v, a.y * c.v + a.x * s.v} : V{a.x * c.v + a.y * s.v, a.y * c.v - a.x * s.v};
    return NEG ? cneg(r) : r;
  }
}
// multiplication by exp(-+ i pi/4) and exp(-+ 3 i pi/4): one constant, 1/sqrt(2)
constexpr KConst K_R2 = kconst(0.70710678118654752440);
constexpr KConst K_C16 = kconst(0.92387953251128675613);   // cos(pi/8)
constexpr KConst K_S16 = kconst(0.38268343236508977173);   // sin(pi/8)
constexpr KConst K_H3 = kconst(0.86602540378443864676);    // sqrt(3)/2
template <bool INV, typename V> __device__ __forceinline__ V rot45(V a) {   // * exp(-+ i pi/4)
  if constexpr (sizeof(a.x) == 4) {
    // forward (a.x + a.y, -(a.x - a.y)) K;  inverse (a.x - a.y, a.x + a.y) K
    if constexpr (INV) return kmul2(__ffma2_rn(swap2(a), float2{-1.0f, 1.0f}, a), K_R2, 1.0f, 1.0f);
    else return kmul2(__ffma2_rn(a, float2{1.0f, -1.0f}, swap2(a)), K_R2, 1.0f, -1.0f);
  } else {
    return INV ? V{kmul(a.x - a.y, K_R2), kmul(a.x + a.y, K_R2)} : V{kmul(a.x + a.y, K_R2), kmul(a.y - a.x, K_R2)};
  }
}
template <bool INV, typename V> __device__ __forceinline__ V rot135(V a) {  // * exp(-+ 3 i pi/4)
  if constexpr (sizeof(a.x) == 4) {
    // forward (a.y - a.x, -(a.x + a.y)) K;  inverse (-(a.x + a.y), a.x - a.y) K
    if constexpr (INV) return kmul2(__ffma2_rn(a, float2{1.0f, -1.0f}, swap2(a)), K_R2, -1.0f, 1.0f);
    else return kmul2(__ffma2_rn(a, float2{-1.0f, 1.0f}, swap2(a)), K_R2, 1.0f, -1.0f);
  } else {
    return INV ? V{kmul(-a.x - a.y, K_R2), kmul(a.x - a.y, K_R2)} : V{kmul(a.y - a.x, K_R2), kmul(-a.x - a.y, K_R2)};
  }
}

// Stockham twiddle storage: float32 keeps hi (x, y) and lo (z, w) parts, float64 the value.
template <typename T> struct TwT;
template <> struct TwT<float> { using v = float4; };
template <> struct TwT<double> { using v = double2; };
template <typename T> using tw_t = typename TwT<T>::v;

__device__ __forceinline__ float2 twmul(float2 a, float4 w) {   // a * (w.hi + w.lo), one rounding
  const float re_lo = fmaf(a.x, w.z, -a.y * w.w);
  const float im_lo = fmaf(a.x, w.w, a.y * w.z);
  return float2{fmaf(a.x, w.x, fmaf(-a.y, w.y, re_lo)), fmaf(a.x, w.y, fmaf(a.y, w.x, im_lo))};
}
__device__ __forceinline__ double2 twmul(double2 a, double2 w) { return cmul(a, w); }
// a * w as twmul, but with the larger of the two products of each component added last.  The
// kinetic factor turns a slowly rotating mode by the same tiny angle at every step; summing its
// small terms against the larger product alone first (as twmul's imaginary part does) would round
// the shrink a (1 - cos) away with the same sign at every step -- a steady gain of |a|^2 (emulated:
// +2.8e-6 over 200 steps at 2.5e-4 rad; with this order ~1e-9, the rounding noise).
__device__ __forceinline__ float2 twmul_k(float2 a, float4 w) {
  const float re_lo = fmaf(a.x, w.z, -a.y * w.w);
  const float im_lo = fmaf(a.x, w.w, a.y * w.z);
  const bool cb = fabsf(w.x) >= fabsf(w.y);
  // re = a.x c - a.y s, im = a.y c + a.x s: the c products are the larger when |c| >= |s|
  const float rb = cb ? a.x : -a.y, rbw = cb ? w.x : w.y, rs = cb ? -a.y : a.x, rsw = cb ? w.y : w.x;
  const float ib = cb ? a.y : a.x, ibw = cb ? w.x : w.y, is = cb ? a.x : a.y, isw = cb ? w.y : w.x;
  return float2{fmaf(rb, rbw, fmaf(rs, rsw, re_lo)), fmaf(ib, ibw, fmaf(is, isw, im_lo))};
}

// v * w / |w| for a float unit-ish w = c + i s.  |w|^2 - 1 is formed exactly (error-free
// products; the subtraction is exact by Sterbenz's lemma) and the product uses
// w (1 - e/2) as a hi + lo pair, so |result| = |v| (1 + O(e^2)) up to one unbiased rounding.
// A rounded w would scale |v| by the same factor at every step (for the kinetic factor, which
// is the same for a given k in every step) and make the conserved mass drift.
__device__ __forceinline__ float2 unit_rotate(float2 v, float c, float s) {
  const float pc = c * c, ec = fmaf(c, c, -pc);
  const float ps = s * s, es = fmaf(s, s, -ps);
  const float big = fmaxf(pc, ps), small = fminf(pc, ps);
  const float t = (big >= 0.5f) ? ((big - 1.0f) + small) : ((pc - 0.5f) + (ps - 0.5f));
  const float h = -0.5f * (t + (ec + es));
  const float dc = c * h, ds = s * h;
  const float re = fmaf(v.x, c, fmaf(-v.y, s, fmaf(v.x, dc, -v.y * ds)));
  const float im = fmaf(v.x, s, fmaf(v.y, c, fmaf(v.x, ds, v.y * dc)));
  return float2{re, im};
}
__device__ __forceinline__ double2 unit_rotate(double2 v, double c, double s) { return cmul(v, double2{c, s}); }


// ---------------------------------------------------------------- butterflies
// In-register DFTs of size 2, 3, 4, 8, 16, 32, natural order in and out.
template <bool INV, typename V> __device__ __forceinline__ void dft2(V& a, V& b) {
  V t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

// p = e + m, q = e - m with m = -+i o (forward -i, inverse +i)
template <bool INV, typename V> __device__ __forceinline__ void add_sub_mi(V e, V o, V& p, V& q) {
  if constexpr (sizeof(e.x) == 4) {
    // -i o = (o.y, -o.x), i o = (-o.y, o.x): both lanes from the swapped o with signs
    const float2 os = swap2(o);
    p = __ffma2_rn(os, INV ? float2{-1.0f, 1.0f} : float2{1.0f, -1.0f}, e);
    q = __ffma2_rn(os, INV ? float2{1.0f, -1.0f} : float2{-1.0f, 1.0f}, e);
  } else {
    const V m = mul_mi<INV>(o);
    p = cadd(e, m);
    q = csub(e, m);
  }
}

template <bool INV, typename V> __device__ __forceinline__ void dft4(V& a0, V& a1, V& a2, V& a3) {
  V s0 = cadd(a0, a2), d0 = csub(a0, a2), s1 = cadd(a1, a3), d1 = csub(a1, a3);
  a0 = cadd(s0, s1);
  a2 = csub(s0, s1);
  add_sub_mi<INV>(d0, d1, a1, a3);
}

template <bool INV, typename V> __device__ __forceinline__ void dft3(V& a0, V& a1, V& a2) {
  using S = decltype(a0.x);
  V t1 = cadd(a1, a2);
  V d = csub(a1, a2);
  V t2, t3;
  if constexpr (sizeof(S) == 4) {
    t2 = __ffma2_rn(t1, float2{-0.5f, -0.5f}, a0);   // a0 - t1 / 2 (the product is exact)
    t3 = kmul2(d, K_H3, 1.0f, 1.0f);                  // (a1 - a2) sqrt(3)/2
  } else {
    t2 = V{a0.x - S(0.5) * t1.x, a0.y - S(0.5) * t1.y};
    t3 = V{kmul(d.x, K_H3), kmul(d.y, K_H3)};
  }
  V it3 = V{-t3.y, t3.x};  // i t3
  a0 = cadd(a0, t1);
  if (!INV) { a1 = csub(t2, it3); a2 = cadd(t2, it3); }
  else      { a1 = cadd(t2, it3); a2 = csub(t2, it3); }
}

template <bool INV, typename V> __device__ __forceinline__ void dft8(V* v) {
  V e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  V o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4<INV>(e0, e1, e2, e3);
  dft4<INV>(o0, o1, o2, o3);
  o1 = rot45<INV>(o1);          // w8^1
  o3 = rot135<INV>(o3);         // w8^3
  v[0] = cadd(e0, o0); v[4] = csub(e0, o0);
  v[1] = cadd(e1, o1); v[5] = csub(e1, o1);
  add_sub_mi<INV>(e2, o2, v[2], v[6]);   // w8^2 = -+i
  v[3] = cadd(e3, o3); v[7] = csub(e3, o3);
}

// 16 = 4 x 4: DFT4 over the stride-4 subsequences, twiddles w16^(n2 k1), DFT4 over n2.
template <bool INV, typename V> __device__ __forceinline__ void dft16(V* v) {
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) dft4<INV>(v[n2], v[4 + n2], v[8 + n2], v[12 + n2]);
  // now v[4 k1 + n2] = Y[n2][k1]; multiply by w16^(n2 k1)
  v[5] = rotk<INV>(v[5], K_C16, K_S16);    // n2=1,k1=1: w^1
  v[6] = rot45<INV>(v[6]);                 // n2=2,k1=1: w^2
  v[7] = rotk<INV>(v[7], K_S16, K_C16);    // n2=3,k1=1: w^3
  v[9] = rot45<INV>(v[9]);                 // n2=1,k1=2: w^2
  v[10] = mul_mi<INV>(v[10]);              // n2=2,k1=2: w^4
  v[11] = rot135<INV>(v[11]);              // n2=3,k1=2: w^6
  v[13] = rotk<INV>(v[13], K_S16, K_C16);  // n2=1,k1=3: w^3
  v[14] = rot135<INV>(v[14]);              // n2=2,k1=3: w^6
  v[15] = rotk<INV, V, true>(v[15], K_C16, K_S16);  // n2=3,k1=3: w^9 = -w^1
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) dft4<INV>(v[4 * k1], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]);
  // v[4 k1 + k2] = X[k1 + 4 k2]: transpose to natural order
  V t[16];
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) t[k1 + 4 * k2] = v[4 * k1 + k2];
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = t[i];
}

// cos(k pi / 16), k = 0..8, and cos / sin of any multiple of pi / 16 by symmetry
constexpr double COS_PI16[9] = {1.0,
                                0.98078528040323044913,
                                0.92387953251128675613,
                                0.83146961230254523708,
                                0.70710678118654752440,
                                0.55557023301960222474,
                                0.38268343236508977173,
                                0.19509032201612826785,
                                0.0};
__host__ __device__ constexpr double cos_pi16(int e) {
  e = ((e % 32) + 32) % 32;
  return e <= 8 ? COS_PI16[e] : (e <= 16 ? -COS_PI16[16 - e] : (e <= 24 ? -COS_PI16[e - 16] : COS_PI16[32 - e]));
}
__host__ __device__ constexpr double sin_pi16(int e) { return cos_pi16(8 - e); }

// a * w32^EXP (forward, w32 = exp(-2 pi i / 32)) or a * conj(w32^EXP) (inverse)
template <bool INV, int EXP, typename V> __device__ __forceinline__ V rot32(V a) {
  constexpr int e = EXP % 32;
  if constexpr (e == 0) return a;
  else if constexpr (e == 8) return mul_mi<INV>(a);
  else if constexpr (e == 16) return cneg(a);
  else if constexpr (e == 24) return mul_mi<!INV>(a);
  else if constexpr (e == 4) return rot45<INV>(a);
  else if constexpr (e == 12) return rot135<INV>(a);
  else {
    constexpr KConst c = kconst(cos_pi16(e)), s = kconst(sin_pi16(e));
    return rotk<INV>(a, c, s);
  }
}

// 32 = 8 x 4: DFT8 over the four stride-4 subsequences, twiddles w32^(n2 k1), DFT4 over n2:
//   X[k1 + 8 k2] = sum_n2 w4^(n2 k2) w32^(n2 k1) sum_n1 w8^(n1 k1) x[4 n1 + n2]
template <bool INV, typename V> __device__ __forceinline__ void dft32(V* v) {
  V y[32];
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) {
    V u[8];
#pragma unroll
    for (int n1 = 0; n1 < 8; ++n1) u[n1] = v[4 * n1 + n2];
    dft8<INV>(u);
#pragma unroll
    for (int k1 = 0; k1 < 8; ++k1) y[4 * k1 + n2] = u[k1];
  }
  // y[4 k1 + n2] = Y[n2][k1]; multiply by w32^(n2 k1)
  y[5] = rot32<INV, 1>(y[5]);   y[6] = rot32<INV, 2>(y[6]);   y[7] = rot32<INV, 3>(y[7]);
  y[9] = rot32<INV, 2>(y[9]);   y[10] = rot32<INV, 4>(y[10]); y[11] = rot32<INV, 6>(y[11]);
  y[13] = rot32<INV, 3>(y[13]); y[14] = rot32<INV, 6>(y[14]); y[15] = rot32<INV, 9>(y[15]);
  y[17] = rot32<INV, 4>(y[17]); y[18] = rot32<INV, 8>(y[18]); y[19] = rot32<INV, 12>(y[19]);
  y[21] = rot32<INV, 5>(y[21]); y[22] = rot32<INV, 10>(y[22]); y[23] = rot32<INV, 15>(y[23]);
  y[25] = rot32<INV, 6>(y[25]); y[26] = rot32<INV, 12>(y[26]); y[27] = rot32<INV, 18>(y[27]);
  y[29] = rot32<INV, 7>(y[29]); y[30] = rot32<INV, 14>(y[30]); y[31] = rot32<INV, 21>(y[31]);
#pragma unroll
  for (int k1 = 0; k1 < 8; ++k1) dft4<INV>(y[4 * k1], y[4 * k1 + 1], y[4 * k1 + 2], y[4 * k1 + 3]);
  // y[4 k1 + k2] = X[k1 + 8 k2]: natural order
#pragma unroll
  for (int k1 = 0; k1 < 8; ++k1)
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) v[k1 + 8 * k2] = y[4 * k1 + k2];
}

template <int R, bool INV, typename V> __device__ __forceinline__ void dft(V* v) {
  if constexpr (R == 2) dft2<INV>(v[0], v[1]);
  else if constexpr (R == 3) dft3<INV>(v[0], v[1], v[2]);
  else if constexpr (R == 4) dft4<INV>(v[0], v[1], v[2], v[3]);
  else if constexpr (R == 8) dft8<INV>(v);
  else if constexpr (R == 16) dft16<INV>(v);
  else if constexpr (R == 32) dft32<INV>(v);
  else static_assert(R == 2, "unsupported radix");
}

// ---------------------------------------------------------------- radix plans
// Forward radix order per length; E = elements per thread (a multiple of every radix).
template <int L> struct Plan;
template <> struct Plan<8>    { static constexpr int NP = 1, E = 8,  R0 = 8,  R1 = 1,  R2 = 1; };
template <> struct Plan<12>   { static constexpr int NP = 2, E = 12, R0 = 4,  R1 = 3,  R2 = 1; };
template <> struct Plan<16>   { static constexpr int NP = 1, E = 16, R0 = 16, R1 = 1,  R2 = 1; };
template <> struct Plan<24>   { static constexpr int NP = 2, E = 24, R0 = 8,  R1 = 3,  R2 = 1; };
template <> struct Plan<32>   { static constexpr int NP = 2, E = 8,  R0 = 8,  R1 = 4,  R2 = 1; };
template <> struct Plan<48>   { static constexpr int NP = 3, E = 12, R0 = 4,  R1 = 4,  R2 = 3; };
template <> struct Plan<64>   { static constexpr int NP = 2, E = 8,  R0 = 8,  R1 = 8,  R2 = 1; };
template <> struct Plan<96>   { static constexpr int NP = 3, E = 24, R0 = 8,  R1 = 4,  R2 = 3; };
template <> struct Plan<128>  { static constexpr int NP = 2, E = 16, R0 = 16, R1 = 8,  R2 = 1; };
template <> struct Plan<192>  { static constexpr int NP = 3, E = 24, R0 = 8,  R1 = 8,  R2 = 3; };
template <> struct Plan<256>  { static constexpr int NP = 2, E = 16, R0 = 16, R1 = 16, R2 = 1; };
template <> struct Plan<512>  { static constexpr int NP = 2, E = 32, R0 = 16, R1 = 32, R2 = 1; };
template <> struct Plan<1024> { static constexpr int NP = 2, E = 32, R0 = 32, R1 = 32, R2 = 1; };

template <int L> __host__ __device__ constexpr int radix_fwd(int i) {
  return i == 0 ? Plan<L>::R0 : (i == 1 ? Plan<L>::R1 : Plan<L>::R2);
}
// pass i of the inverse transform uses the forward radices in reverse order
template <int L, bool INV> __host__ __device__ constexpr int radix_of(int i) {
  return INV ? radix_fwd<L>(Plan<L>::NP - 1 - i) : radix_fwd<L>(i);
}
template <int L, bool INV> __host__ __device__ constexpr int span_of(int i) {
  int ns = 1;
  for (int k = 0; k < i; ++k) ns *= radix_of<L, INV>(k);
  return ns;
}
// offset of pass i's twiddles in the direction's table: sum over earlier passes of NS (R - 1)
template <int L, bool INV> __host__ __device__ constexpr int tw_offset(int i) {
  int off = 0;
  for (int k = 0; k < i; ++k) off += span_of<L, INV>(k) * (radix_of<L, INV>(k) - 1);
  return off;
}
template <int L, bool INV> __host__ __device__ constexpr int tw_size() { return tw_offset<L, INV>(Plan<L>::NP); }

// ---------------------------------------------------------------- pencil engine
// Layout functor Lay: int smem_index(int pencil, int pos).  Registers v[E]:
// at the input of pass i (radix R) v[b R + r] holds x[t + b TP + r L/R].
// TW_SH: the twiddle table has been copied to shared memory (plain loads), else read through
// the read-only data cache.
template <typename T, int L, int B, class Lay, bool INV, int I, bool TW_SH = false>
__device__ __forceinline__ void pass_compute(cpx<T>* v, int t, const tw_t<T>* __restrict__ tw) {
  constexpr int R = radix_of<L, INV>(I);
  constexpr int NS = span_of<L, INV>(I);
  constexpr int E = Plan<L>::E;
  constexpr int TP = L / E;
  if constexpr (NS > 1) {
    constexpr int OFF = tw_offset<L, INV>(I);
#pragma unroll
    for (int b = 0; b < E / R; ++b) {
      const int j = t + b * TP;
      const int jm = j % NS;
#pragma unroll
      for (int r = 1; r < R; ++r) {
        const tw_t<T>* q = tw + OFF + jm * (R - 1) + (r - 1);
        if constexpr (TW_SH) v[b * R + r] = twmul(v[b * R + r], *q);
        else v[b * R + r] = twmul(v[b * R + r], __ldg(q));
      }
    }
  }
#pragma unroll
  for (int b = 0; b < E / R; ++b) dft<R, INV>(v + b * R);
}

// Write pass I's outputs to shared memory at their Stockham positions.
template <typename T, int L, class Lay, bool INV, int I>
__device__ __forceinline__ void pass_store(const cpx<T>* v, int t, int p, cpx<T>* sm, const Lay& lay) {
  constexpr int R = radix_of<L, INV>(I);
  constexpr int NS = span_of<L, INV>(I);
  constexpr int E = Plan<L>::E;
  constexpr int TP = L / E;
#pragma unroll
  for (int b = 0; b < E / R; ++b) {
    const int j = t + b * TP;
    const int idxD = (j / NS) * NS * R + (j % NS);
#pragma unroll
    for (int r = 0; r < R; ++r) sm[lay(p, idxD + r * NS)] = v[b * R + r];
  }
}

// Read pass I's inputs (natural Stockham input pattern) from shared memory.
template <typename T, int L, class Lay, bool INV, int I>
__device__ __forceinline__ void pass_load(cpx<T>* v, int t, int p, const cpx<T>* sm, const Lay& lay) {
  constexpr int R = radix_of<L, INV>(I);
  constexpr int E = Plan<L>::E;
  constexpr int TP = L / E;
#pragma unroll
  for (int b = 0; b < E / R; ++b) {
    const int j = t + b * TP;
#pragma unroll
    for (int r = 0; r < R; ++r) v[b * R + r] = sm[lay(p, j + r * (L / R))];
  }
}

// Position (along the pencil) of register e at the input of the first pass of
// direction INV, equal to the position of register e at the output of the
// last pass of the opposite direction.
template <int L, bool INV> __device__ __forceinline__ int in_pos(int e, int t) {
  constexpr int R = radix_of<L, INV>(0);
  constexpr int TP = L / Plan<L>::E;
  return t + (e / R) * TP + (e % R) * (L / R);
}
// Position of register e at the output of the last pass of direction INV.
template <int L, bool INV> __device__ __forceinline__ int out_pos(int e, int t) {
  constexpr int R = radix_of<L, INV>(Plan<L>::NP - 1);
  constexpr int TP = L / Plan<L>::E;
  return t + (e / R) * TP + (e % R) * (L / R);
}

// Full 1D transform of the registers: input pattern in_pos<INV>, output pattern out_pos<INV>.
// Uses shared memory for the exchanges between passes (two barriers each).  WARP_X: every
// pencil's threads lie in one warp and its exchange region is private to it, so the
// exchanges only need warp-level barriers.
// NB: 0 = the block barrier; otherwise a named barrier over a group of NB consecutive threads,
// barrier 1 + threadIdx.x / NB (kernels whose last warps do other work than the transforms use
// group 0; kernels with several compute groups, one barrier per group).
template <int NB> __device__ __forceinline__ int group_bar() { return 1 + (int)threadIdx.x / NB; }
template <int NB> __device__ __forceinline__ void bsync() {
  if constexpr (NB == 0) __syncthreads();
  else asm volatile("bar.sync %0, %1;" ::"r"(group_bar<NB>()), "n"(NB) : "memory");
}
template <bool WARP_X, int NB = 0> __device__ __forceinline__ void xsync() {
  if constexpr (WARP_X) __syncwarp();
  else bsync<NB>();
}
template <typename T, int L, int B, class Lay, bool INV, bool WARP_X = false, bool TW_SH = false, int NB = 0>
__device__ __forceinline__ void fft_regs(cpx<T>* v, int t, int p, cpx<T>* sm, const Lay& lay,
                                         const tw_t<T>* __restrict__ tw) {
  constexpr int NP = Plan<L>::NP;
  pass_compute<T, L, B, Lay, INV, 0, TW_SH>(v, t, tw);
  if constexpr (NP > 1) {
    pass_store<T, L, Lay, INV, 0>(v, t, p, sm, lay);
    xsync<WARP_X, NB>();
    pass_load<T, L, Lay, INV, 1>(v, t, p, sm, lay);
    xsync<WARP_X, NB>();
    pass_compute<T, L, B, Lay, INV, 1, TW_SH>(v, t, tw);
  }
  if constexpr (NP > 2) {
    pass_store<T, L, Lay, INV, 1>(v, t, p, sm, lay);
    xsync<WARP_X, NB>();
    pass_load<T, L, Lay, INV, 2>(v, t, p, sm, lay);
    xsync<WARP_X, NB>();
    pass_compute<T, L, B, Lay, INV, 2, TW_SH>(v, t, tw);
  }
}

}  // namespace gp

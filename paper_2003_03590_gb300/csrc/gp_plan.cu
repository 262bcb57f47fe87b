// gp_plan.cu -- plan object, float64-generated tables, dispatch and error handling of the C ABI.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "gp_internal.h"

namespace gp {

bool supported_n(int n) {
  switch (n) {
#define GP_CASE(L) case L:
    GP_SIZES(GP_CASE)
#undef GP_CASE
    return true;
    default:
      return false;
  }
}

int plan_np(int n) {
  switch (n) {
#define GP_CASE(L) case L: return Plan<L>::NP;
    GP_SIZES(GP_CASE)
#undef GP_CASE
    default: return 0;
  }
}

int plan_radix_fwd(int n, int i) {
  switch (n) {
#define GP_CASE(L) case L: return radix_fwd<L>(i);
    GP_SIZES(GP_CASE)
#undef GP_CASE
    default: return 0;
  }
}

cudaError_t sweep(int n, const SweepArgs<float>& a, cudaStream_t s) {
  switch (n) {
#define GP_CASE(L) case L: return sweep_f32_##L(a, s);
    GP_SIZES(GP_CASE)
#undef GP_CASE
    default: return cudaErrorInvalidValue;
  }
}
cudaError_t sweep(int n, const SweepArgs<double>& a, cudaStream_t s) {
  switch (n) {
#define GP_CASE(L) case L: return sweep_f64_##L(a, s);
    GP_SIZES(GP_CASE)
#undef GP_CASE
    default: return cudaErrorInvalidValue;
  }
}

gp_status fail(gp_plan* p, gp_status st, const std::string& msg) {
  if (p) p->err = msg;
  return st;
}

gp_status check_status(gp_plan* p) {
  GP_CUDA(p, p->stream ? cudaStreamSynchronize(p->stream) : cudaDeviceSynchronize());
  int st = 0;
  GP_CUDA(p, cudaMemcpy(&st, p->flag + 1, sizeof(int), cudaMemcpyDeviceToHost));
  if (st) {
    GP_CUDA(p, cudaMemset(p->flag + 1, 0, sizeof(int)));
    return fail(p, GP_ERR_TIMEOUT, "a bounded wait in a sweep kernel gave up: fields written since the last check are invalid");
  }
  return GP_OK;
}
gp_status cuda_fail(gp_plan* p, cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  return fail(p, e == cudaErrorMemoryAllocation ? GP_ERR_OOM : GP_ERR_CUDA, m);
}

// ---------------------------------------------------------------- tables
// Stockham twiddles of one direction: for pass i (radix R, span NS), entry
// jm (R-1) + (r-1) holds exp(sign 2 pi i r jm / (NS R)), jm < NS, 1 <= r < R.
static void twiddles(int n, bool inv, std::vector<double>& re, std::vector<double>& im) {
  const int np = plan_np(n);
  re.clear();
  im.clear();
  int ns = 1;
  for (int i = 0; i < np; ++i) {
    const int R = plan_radix_fwd(n, inv ? np - 1 - i : i);
    for (int jm = 0; jm < ns; ++jm)
      for (int r = 1; r < R; ++r) {
        // reduce r jm / (ns R) exactly in integers before forming the angle
        long long num = (long long)r * jm, den = (long long)ns * R;
        num %= den;
        double ang = (inv ? 2.0 : -2.0) * M_PI * (double)num / (double)den;
        re.push_back(std::cos(ang));
        im.push_back(std::sin(ang));
      }
    ns *= R;
  }
}

// v = hi + lo, hi = v rounded to 12 significant bits, lo = the float remainder (hi + lo = v to
// about 2^-36).  The compensated multiply fma(a, c_hi, fma(b, s_hi, lo_terms)) rounds twice; its
// inner rounding must not depend on the value of hi in a fixed way.  With a full-precision hi a
// product a*hi can be exact (hi = 1/2, the 30-degree twiddles of radix-3 lengths) or sit on a
// rounding midpoint (hi = 0.49999997 = 1/2 - 2^-25), and the lo terms are then rounded away with
// the same sign at every step, which makes the conserved mass drift.  A 12-bit hi leaves at least
// 12 bits of every product below the float32 ulp, set by the datum's low bits: unbiased rounding.
void split_hilo(double v, float* hi, float* lo) {
  if (v == 0.0) {
    *hi = 0.0f;
    *lo = 0.0f;
    return;
  }
  int e = 0;
  const double m = std::frexp(v, &e);                    // v = m 2^e, 1/2 <= |m| < 1
  const double h = std::ldexp(std::nearbyint(m * 4096.0) / 4096.0, e);
  *hi = (float)h;
  *lo = (float)(v - h);
}

template <typename V> static V pack(double c, double s);
// float32 twiddles keep the rounded value and the remainder, (hi.x, hi.y, lo.x, lo.y)
template <> float4 pack<float4>(double c, double s) {
  float ch, cl, sh, sl;
  split_hilo(c, &ch, &cl);
  split_hilo(s, &sh, &sl);
  return make_float4(ch, sh, cl, sl);
}
template <> double2 pack<double2>(double c, double s) { return make_double2(c, s); }
template <> float2 pack<float2>(double c, double s) { return make_float2((float)c, (float)s); }

template <typename V> static cudaError_t upload(const std::vector<double>& re, const std::vector<double>& im, void** dev) {
  std::vector<V> h(re.size() > 0 ? re.size() : 1);
  for (size_t i = 0; i < re.size(); ++i) h[i] = pack<V>(re[i], im[i]);
  cudaError_t e = cudaMalloc(dev, h.size() * sizeof(V));
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*dev, h.data(), h.size() * sizeof(V), cudaMemcpyHostToDevice);
}

static cudaError_t build_tables(FieldPlan& F) {
  std::vector<double> re, im;
  cudaError_t e;
  for (int inv = 0; inv < 2; ++inv) {
    twiddles(F.n, inv != 0, re, im);
    e = upload<float4>(re, im, inv ? &F.t32.tw_inv : &F.t32.tw_fwd);
    if (e != cudaSuccess) return e;
    e = upload<double2>(re, im, inv ? &F.t64.tw_inv : &F.t64.tw_fwd);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// exp(-i alpha k^2 s) for grid index i (k = i for i < N/2, else i - N; Nyquist k^2 = (N/2)^2).
// The phase alpha k^2 s is reduced modulo 2 pi in float64 before rounding.
static void ktable_values(int n, double alpha, double s, std::vector<double>& re, std::vector<double>& im) {
  re.resize(n);
  im.resize(n);
  for (int i = 0; i < n; ++i) {
    double k = (i < (n + 1) / 2) ? i : i - n;
    double ph = std::fmod(alpha * k * k * s, 2.0 * M_PI);
    re[i] = std::cos(ph);
    im[i] = -std::sin(ph);
  }
}

// float64 fields: N entries exp(-i alpha k^2 s).  float32 fields: N hi/lo entries of the same,
// followed by N^2 hi/lo entries of exp(-i alpha (k1^2 + k2^2) s) / N^3 (index i2 N + i1),
// each formed in float64 and split into hi + lo.
const void* ktable(gp_plan* p, int field, double s, bool fp64) {
  FieldPlan& F = p->f[field];
  std::vector<KTable>& cache = fp64 ? F.k64 : F.k32;
  for (auto& k : cache)
    if (k.s == s) return k.dev;
  std::vector<double> re, im;
  ktable_values(F.n, F.alpha, s, re, im);
  KTable kt;
  kt.s = s;
  cudaError_t e;
  if (fp64) {
    e = upload<double2>(re, im, &kt.dev);
  } else {
    const int n = F.n;
    const double norm = 1.0 / (double)F.npts;
    std::vector<double> r2((size_t)n + (size_t)n * n), i2((size_t)n + (size_t)n * n);
    for (int i = 0; i < n; ++i) {
      r2[i] = re[i];
      i2[i] = im[i];
    }
    for (int b = 0; b < n; ++b)
      for (int a = 0; a < n; ++a) {
        const size_t q = (size_t)n + (size_t)b * n + a;
        r2[q] = (re[a] * re[b] - im[a] * im[b]) * norm;
        i2[q] = (re[a] * im[b] + im[a] * re[b]) * norm;
      }
    e = upload<float4>(r2, i2, &kt.dev);
  }
  if (e != cudaSuccess) return nullptr;
  cache.push_back(kt);
  return kt.dev;
}

gp_status ensure_ws(gp_plan* p, int field, size_t bytes) {
  FieldPlan& F = p->f[field];
  if (F.ws_bytes >= bytes) return GP_OK;
  if (F.ws) cudaFree(F.ws);
  F.ws = nullptr;
  F.ws_bytes = 0;
  cudaError_t e = cudaMalloc(&F.ws, bytes);
  if (e != cudaSuccess) return cuda_fail(p, e, "workspace allocation");
  F.ws_bytes = bytes;
  return GP_OK;
}

template <> const Tables& tables<float>(FieldPlan& F) { return F.t32; }
template <> const Tables& tables<double>(FieldPlan& F) { return F.t64; }

template <typename T> cudaError_t fft3(FieldPlan& F, cpx<T>* x, bool inverse, cudaStream_t s) {
  const Tables& tb = tables<T>(F);
  SweepArgs<T> a{};
  a.psi[0] = x;
  a.count = 1;
  a.tw_fwd = (const tw_t<T>*)tb.tw_fwd;
  a.tw_inv = (const tw_t<T>*)tb.tw_inv;
  a.op = inverse ? OP_INV : OP_FWD;
  a.scale_inv = 1;
  const int order_f[3] = {0, 1, 2}, order_i[3] = {2, 1, 0};
  for (int i = 0; i < 3; ++i) {
    a.axis = inverse ? order_i[i] : order_f[i];
    cudaError_t e = sweep(F.n, a, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}
template cudaError_t fft3<float>(FieldPlan&, cpx<float>*, bool, cudaStream_t);
template cudaError_t fft3<double>(FieldPlan&, cpx<double>*, bool, cudaStream_t);

template <typename T> cudaError_t kinetic3(FieldPlan& F, cpx<T>* x, const cpx<T>* ek, cudaStream_t s) {
  const Tables& tb = tables<T>(F);
  SweepArgs<T> a{};
  a.psi[0] = x;
  a.count = 1;
  a.tw_fwd = (const tw_t<T>*)tb.tw_fwd;
  a.tw_inv = (const tw_t<T>*)tb.tw_inv;
  if constexpr (sizeof(T) == 4) {
    a.ekx = (const float4*)ek;
    a.ek2 = (const float4*)ek + F.n;
  } else {
    a.ek = ek;
    a.k_norm = kconst(1.0 / (double)F.npts);
  }
  a.scale_inv = 0;
  const int axes[5] = {2, 1, 0, 1, 2};
  const int ops[5] = {OP_FWD, OP_FWD, OP_FWD_K_INV, OP_INV, OP_INV};
  for (int i = 0; i < 5; ++i) {
    a.axis = axes[i];
    a.op = ops[i];
    cudaError_t e = sweep(F.n, a, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}
template cudaError_t kinetic3<float>(FieldPlan&, cpx<float>*, const cpx<float>*, cudaStream_t);
template cudaError_t kinetic3<double>(FieldPlan&, cpx<double>*, const cpx<double>*, cudaStream_t);

static void free_field(FieldPlan& F) {
  void* ptrs[] = {F.t32.tw_fwd, F.t32.tw_inv, F.t64.tw_fwd, F.t64.tw_inv, F.host_buf, F.ws};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  for (auto& k : F.k32)
    if (k.dev) cudaFree(k.dev);
  for (auto& k : F.k64)
    if (k.dev) cudaFree(k.dev);
  F = FieldPlan();
}

}  // namespace gp

using namespace gp;

extern "C" {

const char* gp_status_string(gp_status st) {
  switch (st) {
    case GP_OK: return "GP_OK";
    case GP_ERR_INVALID_ARG: return "GP_ERR_INVALID_ARG";
    case GP_ERR_UNSUPPORTED_SIZE: return "GP_ERR_UNSUPPORTED_SIZE";
    case GP_ERR_OOM: return "GP_ERR_OOM";
    case GP_ERR_CUDA: return "GP_ERR_CUDA";
    case GP_ERR_TIMEOUT: return "GP_ERR_TIMEOUT";
    case GP_ERR_NONFINITE: return "GP_ERR_NONFINITE";
  }
  return "GP_ERR_UNKNOWN";
}

const char* gp_last_error(const gp_plan* p) { return p ? p->err.c_str() : "null plan"; }

gp_status gp_plan_create(const gp_field_params* fields, int nfields, void* stream, gp_plan** out) {
  if (!out) return GP_ERR_INVALID_ARG;
  *out = nullptr;
  if (!fields || nfields <= 0) return GP_ERR_INVALID_ARG;
  for (int i = 0; i < nfields; ++i) {
    const gp_field_params& q = fields[i];
    if (!supported_n(q.n)) return GP_ERR_UNSUPPORTED_SIZE;
    if (!std::isfinite(q.dt) || !std::isfinite(q.xi) || !std::isfinite(q.alpha) || !std::isfinite(q.beta))
      return GP_ERR_INVALID_ARG;
    if (q.precision != GP_FP32 && q.precision != GP_FP64) return GP_ERR_INVALID_ARG;
    if (q.split != GP_SPLIT_NKN && q.split != GP_SPLIT_KNK) return GP_ERR_INVALID_ARG;
    if (q.alpha == 0.0 && q.beta == 0.0 && !(q.xi > 0.0)) return GP_ERR_INVALID_ARG;
  }
  gp_plan* p = new gp_plan();
  p->stream = (cudaStream_t)stream;
  // GP_SWEEPS=plain selects the non-TMA float32 sweep kernels (for comparisons)
  const char* env = std::getenv("GP_SWEEPS");
  p->use_tma = !(env && std::strcmp(env, "plain") == 0);
  p->f.resize(nfields);
  for (int i = 0; i < nfields; ++i) {
    FieldPlan& F = p->f[i];
    F.prm = fields[i];
    F.n = fields[i].n;
    F.npts = (long long)F.n * F.n * F.n;
    F.fp64 = fields[i].precision == GP_FP64;
    if (fields[i].alpha == 0.0 && fields[i].beta == 0.0) {
      F.alpha = std::sqrt(2.0) * fields[i].xi;
      F.beta = 2.0 / F.alpha;
    } else {
      F.alpha = fields[i].alpha;
      F.beta = fields[i].beta;
    }
    cudaError_t e = build_tables(F);
    if (e != cudaSuccess) {
      gp_status st = cuda_fail(p, e, "table upload");
      gp_plan_destroy(p);
      return st;
    }
  }
  cudaError_t e = cudaMalloc(&p->acc, 64 * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&p->flag, 16 * sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(p->flag, 0, 16 * sizeof(int));
  if (e != cudaSuccess) {
    gp_status st = cuda_fail(p, e, "plan allocation");
    gp_plan_destroy(p);
    return st;
  }
  *out = p;
  return GP_OK;
}

gp_status gp_plan_sync(gp_plan* p) {
  if (!p) return GP_ERR_INVALID_ARG;
  return gp::check_status(p);
}

gp_status gp_plan_destroy(gp_plan* p) {
  if (!p) return GP_OK;
  if (p->stream) cudaStreamSynchronize(p->stream);
  else cudaDeviceSynchronize();
  for (auto& F : p->f) free_field(F);
  if (p->acc) cudaFree(p->acc);
  if (p->flag) cudaFree(p->flag);
  if (p->adj_ws) cudaFree(p->adj_ws);
  if (p->plane_sync) cudaFree(p->plane_sync);
  if (p->cycle_graph) cudaGraphExecDestroy(p->cycle_graph);
  if (p->run_graph) cudaGraphExecDestroy(p->run_graph);
  delete p;
  return GP_OK;
}

int gp_plan_nbins(const gp_plan* p, int field) {
  if (!p || field < 0 || field >= (int)p->f.size()) return -1;
  int n = p->f[field].n;
  return (int)std::floor(std::sqrt(3.0) * n / 2.0 + 0.5) + 1;
}

gp_status gp_plan_coefficients(const gp_plan* p, int field, double* alpha, double* beta) {
  if (!p || field < 0 || field >= (int)p->f.size() || !alpha || !beta) return GP_ERR_INVALID_ARG;
  *alpha = p->f[field].alpha;
  *beta = p->f[field].beta;
  return GP_OK;
}

}  // extern "C"

// gp_ensemble.cu -- a whole NKN run of a ragged ensemble (fields of several small lengths) in one
// persistent launch.
//
// The run is a sequence of stages, each a sweep over every field: per step z (N(dt/2) and forward
// z on the first step, inverse z, N(dt), forward z after it), forward y, forward x with K(dt) and
// inverse x, inverse y; after the last step z (inverse z, N(dt/2)) -- the schedule of the
// per-sweep launches (Sec. 4.3, the merged half steps), so the results are bitwise theirs.  An
// item is one tile of one stage of one field (y and z: as many 16-pencil tiles as the CTA's
// threads hold; x: one tile of rows).  Items are handed out from one ticket counter in the order
// (chunk of fields, step, stage, field, tile); an item of stage g of field f waits until every
// item of stage g - 1 of f is counted.  Those items have lower tickets, held by running CTAs whose
// own waits point to lower tickets still, so the oldest unfinished item can always proceed; and
// between the two stages of one field lie the chunk's other fields' items of the same stage, so
// waits are rare.  A chunk (a few tens of MB) stays in L2 through all its steps.  Every wait is
// bounded (~1 s): a wait that gives up sets the status word, and its item is counted anyway so
// that the launch ends (its results are then invalid).
#include <cstring>

#include "gp_internal.h"

namespace gp {

namespace {

constexpr int ENS_THREADS = 256;

// per field: its device array, length and the parameters of the sweep operations
struct EnsField {
  cpx<float>* psi;
  const tw_t<float>* tw_fwd;
  const tw_t<float>* tw_inv;
  const float4* ekx;      // K(dt) along x (hi/lo), length n
  const float4* ek2;      // K(dt) of (y, z) with 1/n^3 (hi/lo), n^2
  float nl_h, nl_dt;      // beta dt/2 and beta dt
  float nl_shift;
  int n;
};

struct EnsArgs {
  EnsField f[GP_ENS_MAXF];
  int nf;
  int off_s[GP_ENS_MAXF + 1];   // items of a y/z stage before field f
  int off_c[GP_ENS_MAXF + 1];   // items of the x stage before field f
  int nch;                      // chunks: fields ch_f0[c] .. ch_f0[c + 1] - 1
  int ch_f0[GP_ENS_MAXF + 1];
  long long ch_t0[GP_ENS_MAXF + 1];   // first ticket of chunk c
  int steps;
  int skip;                     // leading tickets never handed out (a test of the bounded waits)
  int* ticket;
  int* done;                    // [stage][field] items counted
  int* status;
};

__device__ __forceinline__ void red_release_gpu_add_ens(int* p, int v) {
  asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// items of one stage of a field of length L: y/z 16-pencil tiles grouped by the threads that fit
// in a CTA; x tiles of rows
template <int L> __host__ __device__ constexpr int ens_sub() {
  return ENS_THREADS / (strided_batch<float, L>() * (L / Plan<L>::E));
}
template <int L> __host__ __device__ constexpr int ens_items_strided() {
  return (L / strided_batch<float, L>()) * L / ens_sub<L>();
}
template <int L> __host__ __device__ constexpr int ens_items_contig() { return L * L / contig_batch<float, L>(); }
template <int L> __host__ __device__ constexpr size_t ens_smem() {
  const size_t s = sizeof(float2) * (size_t)L * strided_batch<float, L>() * ens_sub<L>();
  const size_t c = sizeof(float2) * (size_t)contig_pitch<L>() * contig_batch<float, L>();
  return s > c ? s : c;
}

#define GP_ENS_SIZES(X) X(32) X(64) X(96) X(128)

// not inlined: each length keeps its own register allocation within the kernel's budget
template <int L> __device__ __noinline__ void ens_stage_item(const EnsField& F, int kind, bool first, bool last,
                                                                int item, float2* sm) {
  SweepArgs<float> a{};
  a.tw_fwd = F.tw_fwd;
  a.tw_inv = F.tw_inv;
  a.ekx = F.ekx;
  a.ek2 = F.ek2;
  a.nl_shift = F.nl_shift;
  a.scale_inv = 0;
  static_assert(contig_batch<float, L>() * (L / Plan<L>::E) == ENS_THREADS, "one x tile per CTA");
  if (kind == 2) {   // x rows: forward x, K(dt) with 1/n^3, inverse x
    a.axis = 0;
    contig_tile<float, L, OP_FWD_K_INV>(a, item, F.psi, threadIdx.x, sm);
    return;
  }
  static_assert(ENS_THREADS % (strided_batch<float, L>() * (L / Plan<L>::E)) == 0, "whole tiles per CTA");
  constexpr int NB = strided_batch<float, L>() * (L / Plan<L>::E);   // threads per tile
  const int sub = threadIdx.x / NB, tid = threadIdx.x % NB;
  const long tile = (long)item * ens_sub<L>() + sub;
  float2* ssm = sm + (size_t)sub * L * strided_batch<float, L>();
  a.axis = kind == 0 ? 2 : 1;
  if (kind == 1) strided_tile<float, L, OP_FWD, NB>(a, tile, F.psi, tid, ssm);
  else if (kind == 3) strided_tile<float, L, OP_INV, NB>(a, tile, F.psi, tid, ssm);
  else if (last) {
    a.nl_coef = F.nl_h;
    strided_tile<float, L, OP_INV_N, NB>(a, tile, F.psi, tid, ssm);
  } else if (first) {
    a.nl_coef = F.nl_h;
    strided_tile<float, L, OP_N_FWD, NB>(a, tile, F.psi, tid, ssm);
  } else {
    a.nl_coef = F.nl_dt;
    strided_tile<float, L, OP_INV_N_FWD, NB>(a, tile, F.psi, tid, ssm);
  }
}

// ticket -> (field f, stage g = 4 step + kind, kind, step, item within the field's stage)
__device__ __forceinline__ void ens_decode(const EnsArgs& a, long long tk, int& f, int& g, int& kind, int& step,
                                           int& item) {
  int c = 0;
  while (a.ch_t0[c + 1] <= tk) ++c;
  const int f0 = a.ch_f0[c], f1 = a.ch_f0[c + 1];
  const int ns = a.off_s[f1] - a.off_s[f0], nc = a.off_c[f1] - a.off_c[f0];
  const int per_step = 3 * ns + nc;                        // z, y forward, x, y inverse
  const long long tl = tk - a.ch_t0[c];
  step = (int)(tl / per_step);
  int r = (int)(tl - (long long)step * per_step);
  if (step == a.steps) kind = 0;                           // the closing z stage
  else if (r < ns) kind = 0;
  else if (r < 2 * ns) { kind = 1; r -= ns; }
  else if (r < 2 * ns + nc) { kind = 2; r -= 2 * ns; }
  else { kind = 3; r -= 2 * ns + nc; }
  const int* off = kind == 2 ? a.off_c : a.off_s;
  r += off[f0];
  f = f0;
  while (off[f + 1] <= r) ++f;
  item = r - off[f];
  g = 4 * step + kind;
}

__global__ void __launch_bounds__(ENS_THREADS, 2) k_ensemble_run(const __grid_constant__ EnsArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* sm = reinterpret_cast<float2*>(smraw);
  __shared__ long long s_ticket;
  __shared__ int s_ok;
  const long long total = a.ch_t0[a.nch];
  // thread 0 holds the CTA's next ticket while the current item runs (the atomic's latency is
  // hidden); the oldest unfinished ticket is then always an item in progress, never one held
  long long next = 0;
  if (threadIdx.x == 0) next = (long long)(unsigned)atomicAdd(a.ticket, 1) + a.skip;
  for (;;) {
    // thread 0 takes the ticket, decodes it and waits for the item's inputs; one barrier then
    // hands (ticket, ok) to the CTA
    if (threadIdx.x == 0) {
      const long long tk = next;
      if (next < total) next = (long long)(unsigned)atomicAdd(a.ticket, 1) + a.skip;
      int ok = 1;
      if (tk < total) {
        int f, g, kind, step, item;
        ens_decode(a, tk, f, g, kind, step, item);
        if (g > 0) {
          const int pk = (g - 1) % 4;
          const int need = pk == 2 ? a.off_c[f + 1] - a.off_c[f] : a.off_s[f + 1] - a.off_s[f];
          const int* c = a.done + (long)(g - 1) * a.nf + f;
          ok = 0;
          for (int i = 0; i < (1 << 20); ++i) {   // about a second
            if (ld_acquire_gpu(c) >= need) {
              ok = 1;
              break;
            }
            __nanosleep(64);
          }
          if (!ok) atomicExch(a.status, 1);
        }
      }
      s_ticket = tk;
      s_ok = ok;
    }
    __syncthreads();
    const long long tk = s_ticket;
    if (tk >= total) break;
    int f, g, kind, step, item;
    ens_decode(a, tk, f, g, kind, step, item);
    const bool first = g == 0, last = step == a.steps;
    if (s_ok) {
      const EnsField& F = a.f[f];
      switch (F.n) {
#define GP_ENS_CASE(L) \
  case L: ens_stage_item<L>(F, kind, first, last, item, sm); break;
        GP_ENS_SIZES(GP_ENS_CASE)
#undef GP_ENS_CASE
        default: break;
      }
    }
    __syncthreads();   // every thread's stores of the item, and the CTA's shared memory is free again
    // counted by a thread of the second warp with a release reduction (the barrier above orders
    // every thread's stores before it), overlapping thread 0's work on the next ticket (that work
    // may wait for this very count: it is not blocked by it)
    if (threadIdx.x == 32) red_release_gpu_add_ens(a.done + (long)g * a.nf + f, 1);
  }
}

size_t ens_smem_of(int n) {
  switch (n) {
#define GP_ENS_CASE(L) case L: return ens_smem<L>();
    GP_ENS_SIZES(GP_ENS_CASE)
#undef GP_ENS_CASE
    default: return 0;
  }
}
int ens_items(int n, bool contig) {
  switch (n) {
#define GP_ENS_CASE(L) case L: return contig ? ens_items_contig<L>() : ens_items_strided<L>();
    GP_ENS_SIZES(GP_ENS_CASE)
#undef GP_ENS_CASE
    default: return 0;
  }
}

}  // namespace

bool ensemble_supported(int n) { return ens_smem_of(n) > 0; }

// Fields are taken in chunks of at most this many bytes, each chunk through all its steps before
// the next: a chunk stays in L2 (129 MB) for its whole run, so HBM sees each field read and
// written about once per call.
constexpr size_t ENS_CHUNK_BYTES = 40u << 20;

// Counters: one ticket, then [4 steps + 1][fields] stage counts.
size_t ensemble_sync_ints(int nsteps, int nf) { return 1 + (size_t)(4 * nsteps + 1) * (size_t)nf; }

cudaError_t ensemble_run(gp_plan* p, const std::vector<int>& fields, void* const* psi, int nsteps, int* sync,
                         cudaStream_t s, int skip) {
  static thread_local EnsArgs a;   // large: off the stack, one per host thread
  std::memset(&a, 0, sizeof(a));
  const int nf = (int)fields.size();
  if (nf < 1 || nf > GP_ENS_MAXF || nsteps < 1) return cudaErrorInvalidValue;
  size_t smem = 0;
  a.off_s[0] = a.off_c[0] = 0;
  for (int i = 0; i < nf; ++i) {
    FieldPlan& F = p->f[fields[i]];
    const float4* kt = (const float4*)ktable(p, fields[i], F.prm.dt, false);
    if (!kt || !ensemble_supported(F.n)) return cudaErrorInvalidValue;
    EnsField& e = a.f[i];
    e.psi = (cpx<float>*)psi[fields[i]];
    e.tw_fwd = (const tw_t<float>*)F.t32.tw_fwd;
    e.tw_inv = (const tw_t<float>*)F.t32.tw_inv;
    e.ekx = kt;
    e.ek2 = kt + F.n;
    e.nl_h = (float)(F.beta * 0.5 * F.prm.dt);
    e.nl_dt = (float)(F.beta * F.prm.dt);
    e.nl_shift = F.prm.nonlin_minus_one ? 1.0f : 0.0f;
    e.n = F.n;
    a.off_s[i + 1] = a.off_s[i] + ens_items(F.n, false);
    a.off_c[i + 1] = a.off_c[i] + ens_items(F.n, true);
    const size_t sm = ens_smem_of(F.n);
    if (sm > smem) smem = sm;
  }
  a.nf = nf;
  a.steps = nsteps;
  a.skip = skip;
  // chunks of consecutive fields
  a.nch = 0;
  a.ch_f0[0] = 0;
  a.ch_t0[0] = 0;
  size_t bytes = 0;
  for (int i = 0; i < nf; ++i) {
    const size_t b = (size_t)a.f[i].n * a.f[i].n * a.f[i].n * sizeof(float2);
    if (i > a.ch_f0[a.nch] && bytes + b > ENS_CHUNK_BYTES) {
      ++a.nch;
      a.ch_f0[a.nch] = i;
      bytes = 0;
    }
    bytes += b;
  }
  ++a.nch;
  a.ch_f0[a.nch] = nf;
  for (int c = 0; c < a.nch; ++c) {
    const int f0 = a.ch_f0[c], f1 = a.ch_f0[c + 1];
    const long long ns = a.off_s[f1] - a.off_s[f0], nc = a.off_c[f1] - a.off_c[f0];
    a.ch_t0[c + 1] = a.ch_t0[c] + (long long)nsteps * (3 * ns + nc) + ns;
  }
  if (a.ch_t0[a.nch] >= (1ll << 31)) return cudaErrorInvalidValue;   // tickets are 32-bit counts
  a.ticket = sync;
  a.done = sync + 1;
  a.status = p->flag + 1;
  cudaError_t e = cudaMemsetAsync(sync, 0, ensemble_sync_ints(nsteps, nf) * sizeof(int), s);
  if (e != cudaSuccess) return e;
  // the shared-memory limit and the CTAs per SM, for the largest tile any length here may need
  // (set once per process, thread-safely, on the first launch, which is never inside a capture)
  static const size_t smax = [] {
    size_t m = 0;
#define GP_ENS_CASE(L) m = ens_smem<L>() > m ? ens_smem<L>() : m;
    GP_ENS_SIZES(GP_ENS_CASE)
#undef GP_ENS_CASE
    return m;
  }();
  static const int occ = [] {
    int o = 0;
    if (cudaFuncSetAttribute(k_ensemble_run, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smax) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_ensemble_run, ENS_THREADS, smax) != cudaSuccess)
      return 0;
    return o;
  }();
  if (occ < 1 || smem > smax) return cudaErrorInvalidConfiguration;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  k_ensemble_run<<<sms * occ, ENS_THREADS, smax, s>>>(a);
  return cudaGetLastError();
}

}  // namespace gp

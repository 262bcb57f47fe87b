// gp_internal.h -- declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <string>
#include <utility>
#include <vector>

#include "gp.h"
#include "gp_sweep.cuh"

namespace gp {

#define GP_SIZES(X) X(8) X(12) X(16) X(24) X(32) X(48) X(64) X(96) X(128) X(192) X(256) X(512) X(1024)
#define GP_DECL_SWEEP(L)                                                   \
  cudaError_t sweep_f32_##L(const SweepArgs<float>&, cudaStream_t);        \
  cudaError_t sweep_f64_##L(const SweepArgs<double>&, cudaStream_t);
GP_SIZES(GP_DECL_SWEEP)
#undef GP_DECL_SWEEP

#define GP_TMA_SIZES(X) X(32) X(48) X(64) X(96) X(128) X(192) X(256) X(512) X(1024)
struct TmaSweepArgs;
struct TmaPlaneArgs;
#define GP_DECL_TMA(L)                                                     \
  cudaError_t tma_sweep_##L(const TmaSweepArgs&, int, int, int, cudaStream_t);   \
  cudaError_t tma_plane_##L(TmaPlaneArgs&, int, int, int, cudaStream_t);
GP_TMA_SIZES(GP_DECL_TMA)
#undef GP_DECL_TMA
bool tma_supported(int n);
// launch one TMA sweep for the fields psi[0..count) of length n (float32 fused path)
cudaError_t tma_sweep(int n, const SweepArgs<float>& a, void* const* psi, int* status, cudaStream_t s,
                      int ctas_req = 0,    // CTAs per SM; 0: as many as fit
                      int stages = 3,      // shared-memory stages of the y/z kernels: 3 or 2
                      int groups = 1);     // compute groups per CTA: 1, or 2 (lengths >= 512)
// launch the fused plane kernel (forward y, forward x + K + inverse x, inverse y) for the
// fields psi[0..count) of length n; sync: device ints, at least plane_sync_ints(n, count)
cudaError_t tma_plane(int n, const SweepArgs<float>& a, void* const* psi, int* sync, int* status, cudaStream_t s,
                      int stages = 3,       // shared-memory stages: 3, or 2 (twiddles through L1)
                      int skip = 0,         // leading tickets never handed out (test of the bounded waits)
                      int ctas_per_sm = 0,  // 0: as many CTAs per SM as fit; else at most that many
                      int groups = 1);      // compute groups per CTA: 1, or the grouped kernel (lengths >= 512)
inline size_t plane_sync_ints(int n, int count) { return 1 + 2 * (size_t)n * (size_t)count; }
// a whole NKN run of float32 fields of small lengths in one persistent launch (gp_ensemble.cu)
constexpr int GP_ENS_MAXF = 64;   // fields of one such launch
bool ensemble_supported(int n);
size_t ensemble_sync_ints(int nsteps, int nf);
cudaError_t ensemble_run(gp_plan* p, const std::vector<int>& fields, void* const* psi, int nsteps, int* sync,
                         cudaStream_t s, int skip = 0);

bool supported_n(int n);
void split_hilo(double v, float* hi, float* lo);   // see gp_plan.cu
int plan_np(int n);           // number of radix passes for length n
int plan_radix_fwd(int n, int i);
cudaError_t sweep(int n, const SweepArgs<float>& a, cudaStream_t s);
cudaError_t sweep(int n, const SweepArgs<double>& a, cudaStream_t s);

// Device tables of one grid length in one precision.
struct Tables {
  void* tw_fwd = nullptr;  // Stockham twiddles, forward direction
  void* tw_inv = nullptr;  // inverse direction
};

// Kinetic propagator table exp(-i alpha k^2 s) for a given s, per storage type.
struct KTable {
  double s = 0.0;
  void* dev = nullptr;
};

struct FieldPlan {
  gp_field_params prm{};
  int n = 0;
  long long npts = 0;
  double alpha = 0.0, beta = 0.0;
  bool fp64 = false;
  Tables t32, t64;                  // both precisions (init and diagnostics use float64)
  std::vector<KTable> k32, k64;     // cached propagator tables
  void* host_buf = nullptr;         // device buffer used by gp_step_host
  void* ws = nullptr;               // general workspace (lazily sized)
  size_t ws_bytes = 0;
};

}  // namespace gp

struct gp_plan {
  std::vector<gp::FieldPlan> f;
  cudaStream_t stream = nullptr;
  std::string err;
  double* acc = nullptr;            // device accumulators for reductions
  int* flag = nullptr;              // device status flags
  void* adj_ws = nullptr;           // adjoint recompute workspace
  size_t adj_bytes = 0;
  cudaGraphExec_t cycle_graph = nullptr;   // captured steady-state cycle of gp_step
  std::vector<void*> cycle_key;            // field pointers the graph was captured for
  int cycle_len = 0;
  cudaGraphExec_t run_graph = nullptr;     // a whole gp_step call, captured when it repeats
  std::vector<void*> run_key, last_key;
  int run_steps = -1, last_steps = -1;
  long long launches = 0;                  // kernels launched or replayed
  bool use_tma = true;                     // float32 sweeps through the TMA-pipelined kernels
  std::vector<std::pair<long long, int>> tune;   // (n, axis, op) key -> sweep variant (gp_plan_autotune)
  int* plane_sync = nullptr;               // counters of the fused plane kernel
  size_t plane_sync_ints = 0;
  int plane_skip = 0;                      // gp_plan_test_timeout: tickets the next launch skips
  bool prof = false;                       // per-launch event timing (gp_profile)
  bool fused_batch = false;                // gp_plan_set_fused_batch: whole NKN runs in one launch
  std::vector<cudaEvent_t> ev_pool;        // recorded events, two per profiled launch
  std::vector<int> ev_kind;                // kind index of each profiled launch
  std::vector<std::string> kinds;          // names of the kinds seen
};

namespace gp {

gp_status fail(gp_plan* p, gp_status st, const std::string& msg);
gp_status cuda_fail(gp_plan* p, cudaError_t e, const char* what);
// synchronise the plan's stream and report (and clear) the sweep kernels' status word
gp_status check_status(gp_plan* p);
#define GP_CUDA(p, call)                                   \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return gp::cuda_fail(p, e_, #call); \
  } while (0)

const void* ktable(gp_plan* p, int field, double s, bool fp64);   // device pointer or nullptr
gp_status ensure_ws(gp_plan* p, int field, size_t bytes);

// 3D transforms of a whole field through the pencil sweeps (unfused).
template <typename T> cudaError_t fft3(FieldPlan& F, cpx<T>* x, bool inverse, cudaStream_t s);
// K with fused sweeps: fwd z, fwd y, [fwd x, K (table ek), 1/N^3, inv x], inv y, inv z.
template <typename T> cudaError_t kinetic3(FieldPlan& F, cpx<T>* x, const cpx<T>* ek, cudaStream_t s);
template <typename T> const Tables& tables(FieldPlan& F);

// pointwise kernels (gp_pointwise.cu)
template <typename T> cudaError_t launch_nonlinear(cpx<T>* psi, long long npts, double coef, double shift, cudaStream_t s);
template <typename T> cudaError_t launch_kinetic_mul(cpx<T>* psi, int n, const cpx<T>* ek, cudaStream_t s);
template <typename T> cudaError_t launch_vjp_nonlinear(const cpx<T>* psi_in, cpx<T>* lam, long long npts, double coef,
                                                       double shift, cudaStream_t s);

// sweep variants (gp_step.cu): 0 TMA persistent, 1 TMA one CTA per SM, 2 plain, 3 TMA with two
// stages, 4 TMA with two compute groups per CTA (lengths >= 512); for OP_PLANE 0 means the fused
// plane kernel, 3 the same with two stages and 2 the three separate sweeps it replaces
enum { VARIANT_TMA = 0, VARIANT_TMA_ONE = 1, VARIANT_PLAIN = 2, VARIANT_TMA_2STAGE = 3, VARIANT_TMA_GROUPS = 4 };
int sweep_variant(gp_plan* p, int n, int axis, int op);
bool plane_on(gp_plan* p, int n);
gp_status ensure_plane_sync(gp_plan* p, size_t ints);
// one float32 sweep of the given kind with the given variant (used by the autotuner)
cudaError_t launch_sweep_variant(gp_plan* p, int n, const SweepArgs<float>& a, void* const* psi, int variant,
                                 cudaStream_t s);

// 3D transforms of several float32 fields of one length through the tuned sweep kernels
cudaError_t fft3_many(gp_plan* p, FieldPlan& F, cpx<float>* const* xs, int count, bool inverse, cudaStream_t s);

// the time step (gp_step.cu): advance one field by nsteps on the plan's stream
gp_status step_field(gp_plan* p, int field, void* psi, int nsteps);

}  // namespace gp

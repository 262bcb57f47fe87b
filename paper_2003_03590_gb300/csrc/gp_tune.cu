// gp_tune.cu -- autotuner of the float32 sweep kernels.
//
// For every grid length of the plan's float32 fields and every sweep kind its time step uses
// (axis and fused operation), the tuner times the candidate kernels on a scratch field:
//   0  TMA-pipelined persistent kernel, as many CTAs per SM as fit
//   1  the same with one CTA per SM (a larger share of L2 and shared-memory bandwidth each)
//   2  the non-persistent kernel (one tile per CTA, loads and stores by the threads)
//   3  (y and z) the TMA kernel with two shared-memory stages instead of three: one tile of
//      look-ahead, one more CTA per SM
// and keeps the fastest; the fused plane kernel (op 7) is timed against the three sweeps it
// replaces.  Choices are cached in a small JSON file keyed by the GPU's name.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "gp_internal.h"

namespace gp {

static std::string cache_key(const char* gpu, int n, int axis, int op) {
  return std::string(gpu) + "|" + std::to_string(n) + "|" + std::to_string(axis) + "|" + std::to_string(op);
}

// candidates per kind: 0-2 everywhere, 3 (two stages) for y, z and the plane kernel; the plane
// kernel has no one-CTA variant
static bool variant_ok(int axis, int op, int v, int n) {
  if (op == OP_PLANE)
    return v == VARIANT_TMA || v == VARIANT_TMA_ONE || v == VARIANT_PLAIN || v == VARIANT_TMA_2STAGE ||
           (v == VARIANT_TMA_GROUPS && n >= 512);
  if (v == VARIANT_TMA_2STAGE) return axis != 0;
  if (v == VARIANT_TMA_GROUPS) return n >= 512;
  return v >= 0 && v <= 2;
}

// minimal reader/writer for {"key": int, ...}
static bool cache_lookup(const std::string& text, const std::string& key, int* v) {
  const std::string pat = "\"" + key + "\":";
  size_t at = text.find(pat);
  if (at == std::string::npos) return false;
  return std::sscanf(text.c_str() + at + pat.size(), "%d", v) == 1;
}

}  // namespace gp

using namespace gp;

extern "C" gp_status gp_plan_autotune(gp_plan* p, const char* cache_path) {
  if (!p) return GP_ERR_INVALID_ARG;
  cudaDeviceProp prop{};
  int dev = 0;
  GP_CUDA(p, cudaGetDevice(&dev));
  GP_CUDA(p, cudaGetDeviceProperties(&prop, dev));
  for (char* c = prop.name; *c; ++c)
    if (*c == '"' || *c == '|') *c = '_';
  const bool verbose = std::getenv("GP_TUNE_VERBOSE") != nullptr;   // per-candidate times on stderr
  std::string text;
  if (cache_path) {
    if (FILE* f = std::fopen(cache_path, "r")) {
      char buf[4096];
      size_t got;
      while ((got = std::fread(buf, 1, sizeof buf, f)) > 0) text.append(buf, got);
      std::fclose(f);
    }
  }
  // the fused plane kernel comes last: it is timed against the three sweeps it replaces, each
  // with the variant chosen for it just before
  const int kinds[9][2] = {{2, OP_N_FWD}, {2, OP_INV_N_FWD}, {2, OP_INV_N}, {2, OP_FWD}, {2, OP_INV},
                           {1, OP_FWD},   {1, OP_INV},       {0, OP_FWD_K_INV}, {1, OP_PLANE}};
  std::vector<int> done;
  std::string out_entries;
  for (size_t fi = 0; fi < p->f.size(); ++fi) {
    FieldPlan& F = p->f[fi];
    if (F.fp64 || !tma_supported(F.n)) continue;
    bool seen = false;
    for (int n : done) seen |= n == F.n;
    if (seen) continue;
    done.push_back(F.n);
    const float4* kt = (const float4*)ktable(p, (int)fi, F.prm.dt, false);
    if (!kt) return fail(p, GP_ERR_OOM, "kinetic table allocation");
    void* scratch = nullptr;
    bool timed = false;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    for (const auto& kind : kinds) {
      const int axis = kind[0], op = kind[1];
      const long long key = (long long)F.n * 64 + axis * 8 + op;
      int best = -1;
      if (!cache_lookup(text, cache_key(prop.name, F.n, axis, op), &best) || !variant_ok(axis, op, best, F.n)) {
        best = 0;
        if (!scratch) {
          GP_CUDA(p, cudaMalloc(&scratch, (size_t)F.npts * 8));
          GP_CUDA(p, cudaMemset(scratch, 0, (size_t)F.npts * 8));
          GP_CUDA(p, cudaEventCreate(&e0));
          GP_CUDA(p, cudaEventCreate(&e1));
        }
        timed = true;
        SweepArgs<float> a{};
        a.psi[0] = (cpx<float>*)scratch;
        a.count = 1;
        a.tw_fwd = (const tw_t<float>*)F.t32.tw_fwd;
        a.tw_inv = (const tw_t<float>*)F.t32.tw_inv;
        a.op = op;
        a.axis = axis;
        a.nl_coef = (float)(F.beta * F.prm.dt);
        a.nl_shift = 1.0f;
        a.ekx = kt;
        a.ek2 = kt + F.n;
        a.scale_inv = 0;
        if (op == OP_PLANE) {
          gp_status st = ensure_plane_sync(p, plane_sync_ints(F.n, 1));
          if (st != GP_OK) return st;
        }
        float best_ms = 1e30f;
        for (int var = 0; var < 5; ++var) {
          if (!variant_ok(axis, op, var, F.n)) continue;
          auto run = [&]() -> cudaError_t { return launch_sweep_variant(p, F.n, a, &scratch, var, p->stream); };
          for (int w = 0; w < 2; ++w) GP_CUDA(p, run());
          GP_CUDA(p, cudaEventRecord(e0, p->stream));
          for (int r = 0; r < 5; ++r) GP_CUDA(p, run());
          GP_CUDA(p, cudaEventRecord(e1, p->stream));
          GP_CUDA(p, cudaEventSynchronize(e1));
          float ms = 0.f;
          GP_CUDA(p, cudaEventElapsedTime(&ms, e0, e1));
          if (verbose) std::fprintf(stderr, "gp_plan_autotune: n %d axis %d op %d variant %d: %.2f us\n", F.n, axis, op, var, ms * 200.f);
          if (ms < best_ms) {
            best_ms = ms;
            best = var;
          }
        }
      }
      bool found = false;
      for (auto& e : p->tune)
        if (e.first == key) {
          e.second = best;
          found = true;
        }
      if (!found) p->tune.push_back({key, best});
      out_entries += (out_entries.empty() ? "" : ",\n") + std::string(" \"") + cache_key(prop.name, F.n, axis, op) +
                     "\": " + std::to_string(best);
    }
    if (scratch) cudaFree(scratch);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    (void)timed;
  }
  if (cache_path && !out_entries.empty()) {
    // keep the entries of other GPUs and lengths already in the file
    std::string merged = "{\n" + out_entries;
    size_t pos = 0;
    while ((pos = text.find('"', pos)) != std::string::npos) {
      const size_t end = text.find('"', pos + 1);
      if (end == std::string::npos) break;
      const std::string k = text.substr(pos + 1, end - pos - 1);
      int v = 0;
      if (out_entries.find("\"" + k + "\"") == std::string::npos && cache_lookup(text, k, &v))
        merged += ",\n \"" + k + "\": " + std::to_string(v);
      pos = end + 1;
    }
    merged += "\n}\n";
    if (FILE* f = std::fopen(cache_path, "w")) {
      std::fwrite(merged.data(), 1, merged.size(), f);
      std::fclose(f);
    }
  }
  // a change of kernels invalidates captured graphs
  if (p->cycle_graph) {
    cudaGraphExecDestroy(p->cycle_graph);
    p->cycle_graph = nullptr;
    p->cycle_key.clear();
  }
  if (p->run_graph) {
    cudaGraphExecDestroy(p->run_graph);
    p->run_graph = nullptr;
    p->run_key.clear();
  }
  return GP_OK;
}

extern "C" int gp_plan_sweep_variant(gp_plan* p, int n, int axis, int op) {
  if (!p) return -1;
  return sweep_variant(p, n, axis, op);
}

extern "C" gp_status gp_plan_set_sweep_variant(gp_plan* p, int n, int axis, int op, int variant) {
  if (!p) return GP_ERR_INVALID_ARG;
  const bool kind_ok = (axis == 2 && op >= OP_FWD && op <= OP_INV_N) || (axis == 1 && (op == OP_FWD || op == OP_INV)) ||
                       (axis == 0 && op == OP_FWD_K_INV) || (axis == 1 && op == OP_PLANE);
  if (!kind_ok || !variant_ok(axis, op, variant, n))
    return fail(p, GP_ERR_INVALID_ARG, "gp_plan_set_sweep_variant: unknown sweep kind or variant");
  if (p->stream) GP_CUDA(p, cudaStreamSynchronize(p->stream));
  const long long key = (long long)n * 64 + axis * 8 + op;
  bool found = false;
  for (auto& e : p->tune)
    if (e.first == key) {
      e.second = variant;
      found = true;
    }
  if (!found) p->tune.push_back({key, variant});
  if (p->cycle_graph) {
    cudaGraphExecDestroy(p->cycle_graph);
    p->cycle_graph = nullptr;
  }
  if (p->run_graph) {
    cudaGraphExecDestroy(p->run_graph);
    p->run_graph = nullptr;
  }
  p->run_key.clear();
  p->last_key.clear();
  return GP_OK;
}

extern "C" gp_status gp_plan_set_fused_batch(gp_plan* p, int on) {
  if (!p) return GP_ERR_INVALID_ARG;
  if (on != 0 && on != 1) return fail(p, GP_ERR_INVALID_ARG, "gp_plan_set_fused_batch: on must be 0 or 1");
  if (on) {
    if ((int)p->f.size() > GP_ENS_MAXF)
      return fail(p, GP_ERR_INVALID_ARG, "gp_plan_set_fused_batch: more fields than one fused run holds");
    for (const auto& F : p->f)
      if (F.fp64 || F.prm.split != GP_SPLIT_NKN || !ensemble_supported(F.n))
        return fail(p, GP_ERR_INVALID_ARG,
                    "gp_plan_set_fused_batch: needs float32 NKN fields of lengths 32, 64, 96 or 128");
  }
  if (p->stream) GP_CUDA(p, cudaStreamSynchronize(p->stream));
  p->fused_batch = on == 1;
  if (p->cycle_graph) {
    cudaGraphExecDestroy(p->cycle_graph);
    p->cycle_graph = nullptr;
  }
  if (p->run_graph) {
    cudaGraphExecDestroy(p->run_graph);
    p->run_graph = nullptr;
  }
  p->run_key.clear();
  p->last_key.clear();
  return GP_OK;
}

extern "C" gp_status gp_plan_test_timeout(gp_plan* p, int tiles) {
  if (!p) return GP_ERR_INVALID_ARG;
  if (tiles < 0) return fail(p, GP_ERR_INVALID_ARG, "gp_plan_test_timeout: negative tile count");
  if (p->stream) GP_CUDA(p, cudaStreamSynchronize(p->stream));
  p->plane_skip = tiles;
  // the setting must reach a direct launch, not a graph captured before it
  if (p->cycle_graph) {
    cudaGraphExecDestroy(p->cycle_graph);
    p->cycle_graph = nullptr;
    p->cycle_key.clear();
  }
  if (p->run_graph) {
    cudaGraphExecDestroy(p->run_graph);
    p->run_graph = nullptr;
  }
  p->run_key.clear();
  p->last_key.clear();
  return GP_OK;
}

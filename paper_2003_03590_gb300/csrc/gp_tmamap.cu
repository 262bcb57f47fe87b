// gp_tmamap.cu -- tensor maps and dispatch of the TMA-pipelined float32 sweeps.
#include <cudaTypedefs.h>

#include <cstring>

#include "gp_internal.h"
#include "gp_plane.cuh"

namespace gp {

bool tma_supported(int n) {
  switch (n) {
#define GP_CASE(L) case L:
    GP_TMA_SIZES(GP_CASE)
#undef GP_CASE
    return true;
    default:
      return false;
  }
}

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

template <int L> static void box_of(int axis, cuuint32_t box[3]) {
  if (axis == 0) {
    box[0] = TmaContig<L>::BOX; box[1] = TmaContig<L>::B; box[2] = 1;
  } else if (axis == 1) {
    box[0] = TmaStrided<L>::B; box[1] = TmaStrided<L>::BOX; box[2] = 1;
  } else {
    box[0] = TmaStrided<L, 3, z_wide<L>()>::B; box[1] = 1; box[2] = TmaStrided<L>::BOX;
  }
}

template <int L> static bool swizzled(int axis) { return axis != 0 && TmaStrided<L>::SWZ; }

static bool encode_box(CUtensorMap* m, void* base, int n, const cuuint32_t box[3], bool swz) {
  auto enc = encode_fn();
  if (!enc) return false;
  cuuint64_t dims[3] = {(cuuint64_t)n, (cuuint64_t)n, (cuuint64_t)n};
  cuuint64_t strides[2] = {(cuuint64_t)n * 8, (cuuint64_t)n * n * 8};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   swz ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

static bool make_map(CUtensorMap* m, void* base, int n, int axis) {
  cuuint32_t box[3];
  bool swz = false;
  switch (n) {
#define GP_CASE(L) case L: box_of<L>(axis, box); swz = swizzled<L>(axis); break;
    GP_TMA_SIZES(GP_CASE)
#undef GP_CASE
    default: return false;
  }
  return encode_box(m, base, n, box, swz);
}

cudaError_t tma_sweep(int n, const SweepArgs<float>& a, void* const* psi, int* status, cudaStream_t s,
                      int ctas_req, int stages, int groups) {
  if (a.axis == 0) stages = 3;
  // large: kept off the stack (a launch copies it); one per host thread, so plans stepped from
  // several threads never share an argument block between its set-up and its launch
  static thread_local TmaSweepArgs t;
  std::memset(&t, 0, sizeof(t));
  t.count = a.count;
  for (int f = 0; f < a.count; ++f)
    if (!make_map(&t.map[f], psi[f], n, a.axis)) return cudaErrorInvalidValue;
  t.tw_fwd = a.tw_fwd;
  t.tw_inv = a.tw_inv;
  t.ekx = a.ekx;
  t.ek2 = a.ek2;
  t.nl_coef = a.nl_coef;
  t.nl_shift = a.nl_shift;
  t.op = a.op;
  t.axis = a.axis;
  t.scale_inv = a.scale_inv;
  t.status = status;
  switch (n) {
#define GP_CASE(L) case L: return tma_sweep_##L(t, ctas_req, stages, groups, s);
    GP_TMA_SIZES(GP_CASE)
#undef GP_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

// the fused plane kernel (gp_plane.cuh): forward y, forward x + K + inverse x, inverse y of
// every z-plane of the fields psi[0..count) in one launch
cudaError_t tma_plane(int n, const SweepArgs<float>& a, void* const* psi, int* sync, int* status, cudaStream_t s,
                      int stages, int skip, int ctas_per_sm, int groups) {
  static thread_local TmaPlaneArgs t;   // as in tma_sweep: one per host thread
  std::memset(&t, 0, sizeof(t));
  t.count = a.count;
  cuuint32_t by[3], bx[3];
  switch (n) {
#define GP_CASE(L)                                                                          \
  case L:                                                                                   \
    by[0] = TmaPlane<L>::B; by[1] = TmaPlane<L>::BOX; by[2] = 1;                            \
    bx[0] = TmaPlane<L>::BOX; bx[1] = TmaPlane<L>::B; bx[2] = 1;                            \
    break;
    GP_TMA_SIZES(GP_CASE)
#undef GP_CASE
    default:
      return cudaErrorInvalidValue;
  }
  for (int f = 0; f < a.count; ++f)
    if (!encode_box(&t.map_y[f], psi[f], n, by, false) || !encode_box(&t.map_x[f], psi[f], n, bx, false))
      return cudaErrorInvalidValue;
  t.tw_fwd = a.tw_fwd;
  t.tw_inv = a.tw_inv;
  t.ekx = a.ekx;
  t.ek2 = a.ek2;
  t.sync = sync;
  t.status = status;
  t.skip = skip;
  cudaError_t e = cudaMemsetAsync(sync, 0, plane_sync_ints(n, a.count) * sizeof(int), s);
  if (e != cudaSuccess) return e;
  switch (n) {
#define GP_CASE(L) case L: return tma_plane_##L(t, stages, ctas_per_sm, groups, s);
    GP_TMA_SIZES(GP_CASE)
#undef GP_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace gp

// Instantiations of the pencil sweeps for some grid lengths (compiled in parallel).
#include "gp_internal.h"
#include "gp_plane.cuh"

namespace gp {
cudaError_t sweep_f32_256(const SweepArgs<float>& a, cudaStream_t s) { return SweepLaunch<float, 256>::launch(a, s); }
cudaError_t sweep_f64_256(const SweepArgs<double>& a, cudaStream_t s) { return SweepLaunch<double, 256>::launch(a, s); }
cudaError_t tma_sweep_256(const TmaSweepArgs& a, int ctas, int stages, int groups, cudaStream_t s) {
  return TmaLaunch<256>::launch(a, ctas, stages, groups, s);
}
cudaError_t tma_plane_256(TmaPlaneArgs& a, int stages, int ctas_per_sm, int groups, cudaStream_t s) {
  return TmaPlaneLaunch<256>::launch(a, stages, ctas_per_sm, groups, s);
}
}  // namespace gp

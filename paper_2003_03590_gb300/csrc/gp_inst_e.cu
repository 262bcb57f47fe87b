// Instantiations of the pencil sweeps for some grid lengths (compiled in parallel).
#include "gp_internal.h"
#include "gp_plane.cuh"

namespace gp {
cudaError_t sweep_f32_1024(const SweepArgs<float>& a, cudaStream_t s) { return SweepLaunch<float, 1024>::launch(a, s); }
cudaError_t sweep_f64_1024(const SweepArgs<double>& a, cudaStream_t s) { return SweepLaunch<double, 1024>::launch(a, s); }
cudaError_t tma_sweep_1024(const TmaSweepArgs& a, int ctas, int stages, int groups, cudaStream_t s) {
  return TmaLaunch<1024>::launch(a, ctas, stages, groups, s);
}
cudaError_t tma_plane_1024(TmaPlaneArgs& a, int stages, int ctas_per_sm, int groups, cudaStream_t s) {
  return TmaPlaneLaunch<1024>::launch(a, stages, ctas_per_sm, groups, s);
}
}  // namespace gp

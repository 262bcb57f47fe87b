// Instantiations of the pencil sweeps for some grid lengths (compiled in parallel).
#include "gp_internal.h"
#include "gp_plane.cuh"

namespace gp {
cudaError_t sweep_f32_512(const SweepArgs<float>& a, cudaStream_t s) { return SweepLaunch<float, 512>::launch(a, s); }
cudaError_t sweep_f64_512(const SweepArgs<double>& a, cudaStream_t s) { return SweepLaunch<double, 512>::launch(a, s); }
cudaError_t tma_sweep_512(const TmaSweepArgs& a, int ctas, int stages, int groups, cudaStream_t s) {
  return TmaLaunch<512>::launch(a, ctas, stages, groups, s);
}
cudaError_t tma_plane_512(TmaPlaneArgs& a, int stages, int ctas_per_sm, int groups, cudaStream_t s) {
  return TmaPlaneLaunch<512>::launch(a, stages, ctas_per_sm, groups, s);
}
}  // namespace gp

// Instantiations of the pencil sweeps for some grid lengths (compiled in parallel).
#include "gp_internal.h"
#include "gp_plane.cuh"

namespace gp {
cudaError_t sweep_f32_64(const SweepArgs<float>& a, cudaStream_t s) { return SweepLaunch<float, 64>::launch(a, s); }
cudaError_t sweep_f64_64(const SweepArgs<double>& a, cudaStream_t s) { return SweepLaunch<double, 64>::launch(a, s); }
cudaError_t sweep_f32_96(const SweepArgs<float>& a, cudaStream_t s) { return SweepLaunch<float, 96>::launch(a, s); }
cudaError_t sweep_f64_96(const SweepArgs<double>& a, cudaStream_t s) { return SweepLaunch<double, 96>::launch(a, s); }
cudaError_t sweep_f32_128(const SweepArgs<float>& a, cudaStream_t s) { return SweepLaunch<float, 128>::launch(a, s); }
cudaError_t sweep_f64_128(const SweepArgs<double>& a, cudaStream_t s) { return SweepLaunch<double, 128>::launch(a, s); }
cudaError_t sweep_f32_192(const SweepArgs<float>& a, cudaStream_t s) { return SweepLaunch<float, 192>::launch(a, s); }
cudaError_t sweep_f64_192(const SweepArgs<double>& a, cudaStream_t s) { return SweepLaunch<double, 192>::launch(a, s); }
cudaError_t tma_sweep_32(const TmaSweepArgs& a, int ctas, int stages, int groups, cudaStream_t s) {
  return TmaLaunch<32>::launch(a, ctas, stages, groups, s);
}
cudaError_t tma_plane_32(TmaPlaneArgs& a, int stages, int ctas_per_sm, int groups, cudaStream_t s) {
  return TmaPlaneLaunch<32>::launch(a, stages, ctas_per_sm, groups, s);
}
cudaError_t tma_sweep_48(const TmaSweepArgs& a, int ctas, int stages, int groups, cudaStream_t s) {
  return TmaLaunch<48>::launch(a, ctas, stages, groups, s);
}
cudaError_t tma_plane_48(TmaPlaneArgs& a, int stages, int ctas_per_sm, int groups, cudaStream_t s) {
  return TmaPlaneLaunch<48>::launch(a, stages, ctas_per_sm, groups, s);
}
cudaError_t tma_sweep_64(const TmaSweepArgs& a, int ctas, int stages, int groups, cudaStream_t s) {
  return TmaLaunch<64>::launch(a, ctas, stages, groups, s);
}
cudaError_t tma_plane_64(TmaPlaneArgs& a, int stages, int ctas_per_sm, int groups, cudaStream_t s) {
  return TmaPlaneLaunch<64>::launch(a, stages, ctas_per_sm, groups, s);
}
cudaError_t tma_sweep_96(const TmaSweepArgs& a, int ctas, int stages, int groups, cudaStream_t s) {
  return TmaLaunch<96>::launch(a, ctas, stages, groups, s);
}
cudaError_t tma_plane_96(TmaPlaneArgs& a, int stages, int ctas_per_sm, int groups, cudaStream_t s) {
  return TmaPlaneLaunch<96>::launch(a, stages, ctas_per_sm, groups, s);
}
cudaError_t tma_sweep_128(const TmaSweepArgs& a, int ctas, int stages, int groups, cudaStream_t s) {
  return TmaLaunch<128>::launch(a, ctas, stages, groups, s);
}
cudaError_t tma_plane_128(TmaPlaneArgs& a, int stages, int ctas_per_sm, int groups, cudaStream_t s) {
  return TmaPlaneLaunch<128>::launch(a, stages, ctas_per_sm, groups, s);
}
cudaError_t tma_sweep_192(const TmaSweepArgs& a, int ctas, int stages, int groups, cudaStream_t s) {
  return TmaLaunch<192>::launch(a, ctas, stages, groups, s);
}
cudaError_t tma_plane_192(TmaPlaneArgs& a, int stages, int ctas_per_sm, int groups, cudaStream_t s) {
  return TmaPlaneLaunch<192>::launch(a, stages, ctas_per_sm, groups, s);
}
}  // namespace gp

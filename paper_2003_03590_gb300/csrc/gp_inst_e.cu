// Instantiations of the pencil sweeps for some grid lengths (compiled in parallel).
#include "gp_internal.h"

namespace gp {
cudaError_t sweep_f32_1024(const SweepArgs<float>& a, cudaStream_t s) { return SweepLaunch<float, 1024>::launch(a, s); }
cudaError_t sweep_f64_1024(const SweepArgs<double>& a, cudaStream_t s) { return SweepLaunch<double, 1024>::launch(a, s); }
}  // namespace gp

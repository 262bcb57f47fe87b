// Instantiations of the pencil sweeps for some grid lengths (compiled in parallel).
#include "gp_internal.h"

namespace gp {
cudaError_t sweep_f32_8(const SweepArgs<float>& a, cudaStream_t s) { return SweepLaunch<float, 8>::launch(a, s); }
cudaError_t sweep_f64_8(const SweepArgs<double>& a, cudaStream_t s) { return SweepLaunch<double, 8>::launch(a, s); }
cudaError_t sweep_f32_12(const SweepArgs<float>& a, cudaStream_t s) { return SweepLaunch<float, 12>::launch(a, s); }
cudaError_t sweep_f64_12(const SweepArgs<double>& a, cudaStream_t s) { return SweepLaunch<double, 12>::launch(a, s); }
cudaError_t sweep_f32_16(const SweepArgs<float>& a, cudaStream_t s) { return SweepLaunch<float, 16>::launch(a, s); }
cudaError_t sweep_f64_16(const SweepArgs<double>& a, cudaStream_t s) { return SweepLaunch<double, 16>::launch(a, s); }
cudaError_t sweep_f32_24(const SweepArgs<float>& a, cudaStream_t s) { return SweepLaunch<float, 24>::launch(a, s); }
cudaError_t sweep_f64_24(const SweepArgs<double>& a, cudaStream_t s) { return SweepLaunch<double, 24>::launch(a, s); }
cudaError_t sweep_f32_32(const SweepArgs<float>& a, cudaStream_t s) { return SweepLaunch<float, 32>::launch(a, s); }
cudaError_t sweep_f64_32(const SweepArgs<double>& a, cudaStream_t s) { return SweepLaunch<double, 32>::launch(a, s); }
cudaError_t sweep_f32_48(const SweepArgs<float>& a, cudaStream_t s) { return SweepLaunch<float, 48>::launch(a, s); }
cudaError_t sweep_f64_48(const SweepArgs<double>& a, cudaStream_t s) { return SweepLaunch<double, 48>::launch(a, s); }
}  // namespace gp

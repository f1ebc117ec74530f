// Instantiates the af_patch_step launchers for float state arrays (the
// kernels themselves live in af_step_kernels.cuh); one translation unit per
// precision so the two compile in parallel.
#include "af_step_kernels.cuh"

namespace af {
template af_status launch_step<float, AF_ACOUSTICS>(int, const StepArgs<float> &,
                                                    const WeightsOf<float, AF_ACOUSTICS>::type &, int, cudaStream_t);
template af_status launch_step<float, AF_ADVECTION>(int, const StepArgs<float> &,
                                                    const WeightsOf<float, AF_ADVECTION>::type &, int, cudaStream_t);
af_status wait_timeouts_f32(unsigned int *count, bool reset) { return wait_timeouts_here(count, reset); }
}  // namespace af

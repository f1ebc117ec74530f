// FP32 af_patch_step kernels specialised for 32 x 32-cell patches (plane
// strides and lattice widths known at compile time); a translation unit of
// their own so they compile in parallel with the others.
#include "af_step_kernels.cuh"

namespace af {
template af_status launch_step_nn<float, AF_ACOUSTICS, 32>(int, const StepArgs<float> &,
                                                           const WeightsOf<float, AF_ACOUSTICS>::type &, int,
                                                           cudaStream_t);
template af_status launch_step_nn<float, AF_ADVECTION, 32>(int, const StepArgs<float> &,
                                                           const WeightsOf<float, AF_ADVECTION>::type &, int,
                                                           cudaStream_t);
af_status wait_timeouts_f32_n32(unsigned int *count, bool reset) { return wait_timeouts_here(count, reset); }
}  // namespace af

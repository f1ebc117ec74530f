// FP32 af_patch_step kernels specialised for 16 x 16-cell patches (plane
// strides and lattice widths known at compile time); a translation unit of
// their own so they compile in parallel with the others.
#include "af_step_kernels.cuh"

namespace af {
template af_status launch_step_nn<float, AF_ACOUSTICS, 16>(int, const StepArgs<float> &,
                                                           const WeightsOf<float, AF_ACOUSTICS>::type &, int,
                                                           cudaStream_t);
template af_status launch_step_nn<float, AF_ADVECTION, 16>(int, const StepArgs<float> &,
                                                           const WeightsOf<float, AF_ADVECTION>::type &, int,
                                                           cudaStream_t);
af_status wait_timeouts_f32_n16(unsigned int *count, bool reset) { return wait_timeouts_here(count, reset); }
}  // namespace af

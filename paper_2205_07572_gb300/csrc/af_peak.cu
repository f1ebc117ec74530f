// af_fma_throughput: a probe of the fused multiply-add rate of this GPU in
// FP32 or FP64, the ALU roof the step kernels are measured against (the
// FP64 stencil is bound by it).  Every thread runs eight independent FMA
// chains in registers and stores one sum, so nothing can be removed.
#include <cuda_runtime.h>

#include <cstdint>

#include "af.h"

namespace af {
namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) fma_probe_kernel(int iters, T *sink) {
    T a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = T(1) + T(threadIdx.x + k) * T(1e-7);
    const T m = T(0.9999999), c = T(1e-7);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], m, c);
    }
    T s = T(0);
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    sink[(int64_t)blockIdx.x * kThreads + threadIdx.x] = s;
}

}  // namespace
}  // namespace af

extern "C" int32_t af_fma_probe_threads(void) { return af::kThreads * af::kChains; }

extern "C" af_status af_fma_throughput(int32_t prec, int32_t blocks, int32_t iters, void *d_sink, void *stream) {
    if ((prec != AF_F64 && prec != AF_F32) || blocks < 1 || iters < 1 || d_sink == nullptr) return AF_ERR_ARG;
    const uintptr_t esz = prec == AF_F64 ? 8 : 4;
    if (reinterpret_cast<uintptr_t>(d_sink) & (esz - 1)) return AF_ERR_LAYOUT;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (prec == AF_F64)
        af::fma_probe_kernel<double><<<blocks, af::kThreads, 0, s>>>(iters, static_cast<double *>(d_sink));
    else
        af::fma_probe_kernel<float><<<blocks, af::kThreads, 0, s>>>(iters, static_cast<float *>(d_sink));
    return cudaGetLastError() == cudaSuccess ? AF_OK : AF_ERR_CUDA;
}

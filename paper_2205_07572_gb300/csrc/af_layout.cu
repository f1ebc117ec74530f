// af_pack_owned / af_unpack_owned: the owned degrees of freedom of every
// patch (the cell averages and the corner, left-edge and bottom-edge point
// values of its n x n cells, Section 2, Fig. 1) between the lattice state
// layout and a compact [patch][comp][plane][n][n] array, so that a state kept
// in host memory carries no ghost ring and no plane padding.  Plain copies:
// one CTA per plane of one patch, threads over rows and columns.
#include <cuda_runtime.h>

#include <cstdint>

#include "af_internal.h"

namespace af {
namespace {

template <typename T, bool PACK>
__global__ void owned_copy_kernel(int n, int64_t plane, const T *__restrict__ src, T *__restrict__ dst) {
    const int64_t pl = blockIdx.x;  // (patch, comp, plane) flattened
    const int W = n + 2 * kGhost + 1;
    const int64_t lat = pl * plane, own = pl * (int64_t)n * n;
    for (int j = threadIdx.y; j < n; j += blockDim.y)
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const int64_t l = lat + (int64_t)(j + kGhost) * W + (i + kGhost), o = own + (int64_t)j * n + i;
            if (PACK)
                dst[o] = src[l];
            else
                dst[l] = src[o];
        }
}

af_status owned_copy(const af_config *cfg, int32_t npatch, const void *src, void *dst, bool pack, void *stream) {
    if (cfg == nullptr || npatch < 0) return AF_ERR_ARG;
    if (cfg->n < 2 || cfg->n > 64) return AF_ERR_ARG;
    if (cfg->prec != AF_F64 && cfg->prec != AF_F32) return AF_ERR_ARG;
    if (cfg->ncomp != (cfg->eq == AF_ADVECTION ? 1 : 3)) return AF_ERR_ARG;
    if (npatch == 0) return AF_OK;
    if (src == nullptr || dst == nullptr || src == dst) return AF_ERR_ARG;
    const void *state = pack ? src : dst;
    const void *owned = pack ? dst : src;
    const uintptr_t esz = cfg->prec == AF_F64 ? 8 : 4;
    if (reinterpret_cast<uintptr_t>(state) & 31u) return AF_ERR_LAYOUT;
    if (reinterpret_cast<uintptr_t>(owned) & (esz - 1)) return AF_ERR_LAYOUT;
    const int64_t blocks = (int64_t)npatch * cfg->ncomp * kPlanes;
    if (blocks > 0x7fffffff) return AF_ERR_ARG;
    const dim3 block(32, 8);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t plane = plane_stride(cfg->n);
    if (cfg->prec == AF_F64) {
        if (pack)
            owned_copy_kernel<double, true><<<(unsigned)blocks, block, 0, s>>>(
                cfg->n, plane, static_cast<const double *>(src), static_cast<double *>(dst));
        else
            owned_copy_kernel<double, false><<<(unsigned)blocks, block, 0, s>>>(
                cfg->n, plane, static_cast<const double *>(src), static_cast<double *>(dst));
    } else {
        if (pack)
            owned_copy_kernel<float, true><<<(unsigned)blocks, block, 0, s>>>(
                cfg->n, plane, static_cast<const float *>(src), static_cast<float *>(dst));
        else
            owned_copy_kernel<float, false><<<(unsigned)blocks, block, 0, s>>>(
                cfg->n, plane, static_cast<const float *>(src), static_cast<float *>(dst));
    }
    return cudaGetLastError() == cudaSuccess ? AF_OK : AF_ERR_CUDA;
}

}  // namespace
}  // namespace af

extern "C" af_status af_pack_owned(const af_config *cfg, int32_t npatch, const void *d_state, void *d_owned,
                                   void *stream) {
    return af::owned_copy(cfg, npatch, d_state, d_owned, true, stream);
}

extern "C" af_status af_unpack_owned(const af_config *cfg, int32_t npatch, const void *d_owned, void *d_state,
                                     void *stream) {
    return af::owned_copy(cfg, npatch, d_owned, d_state, false, stream);
}

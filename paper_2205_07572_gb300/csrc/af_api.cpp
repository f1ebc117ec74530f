// Host-only entry points of libaf.so: status names, layout sizes and the
// work-list builder of af_patch_step.
#include <cstring>

#include "af_internal.h"

extern "C" const char *af_status_string(af_status s) {
    switch (s) {
    case AF_OK: return "AF_OK";
    case AF_ERR_ARG: return "AF_ERR_ARG: invalid argument";
    case AF_ERR_CFL: return "AF_ERR_CFL: time step violates the CFL condition";
    case AF_ERR_LAYOUT: return "AF_ERR_LAYOUT: misaligned pointer or inconsistent layout";
    case AF_ERR_CUDA: return "AF_ERR_CUDA: a CUDA runtime call failed";
    case AF_ERR_TIMEOUT: return "AF_ERR_TIMEOUT: a bounded device wait gave up";
    case AF_ERR_UNIMPLEMENTED: return "AF_ERR_UNIMPLEMENTED";
    }
    return "unknown af_status";
}

extern "C" int64_t af_plane_stride(int32_t n) { return n < 1 ? 0 : af::plane_stride(n); }

extern "C" int64_t af_patch_words(int32_t n, int32_t ncomp) {
    return n < 1 || ncomp < 1 ? 0 : (int64_t)ncomp * af::kPlanes * af::plane_stride(n);
}

extern "C" af_status af_build_step_work_at(const af_config *cfg, int32_t tiling_index, int32_t npatch,
                                           const int32_t *h_patch, const int32_t *h_level, const int32_t *h_ix,
                                           const int32_t *h_iy, const int32_t *h_nbr, af_work *h_work,
                                           int32_t capacity, int32_t *nwork) {
    using namespace af;
    if (cfg == nullptr || nwork == nullptr || npatch < 0 || capacity < 0) return AF_ERR_ARG;
    if (cfg->n < 2 || cfg->n > 64) return AF_ERR_ARG;
    if (tiling_index < 0 || tiling_index >= kNumTilings) return AF_ERR_ARG;
    if (npatch > 0 && h_patch == nullptr) return AF_ERR_ARG;
    const int n = cfg->n;
    const Tiling tl = tiling(tiling_index);
    auto extended = [&](int k) {
        if (h_nbr == nullptr) return true;
        for (int d = 0; d < 8; ++d)
            if (h_nbr[8 * k + d] < 0) return true;
        return false;
    };
    int32_t count = 0;
    for (int k = 0; k < npatch; ++k) {
        const int w = extended(k) ? n + 2 : n;
        count += ((w + tl.tmx - 1) / tl.tmx) * ((w + tl.tmy - 1) / tl.tmy);
    }
    *nwork = count;
    if (count > capacity || (count > 0 && h_work == nullptr)) return AF_ERR_ARG;
    int32_t idx = 0;
    for (int k = 0; k < npatch; ++k) {
        if (h_patch[k] < 0) return AF_ERR_ARG;
        const bool ext = extended(k);
        const int lo = ext ? -1 : 0, w = ext ? n + 2 : n;
        const int ntx = (w + tl.tmx - 1) / tl.tmx, nty = (w + tl.tmy - 1) / tl.tmy;
        for (int ty = 0; ty < nty; ++ty)
            for (int tx = 0; tx < ntx; ++tx) {
                af_work &o = h_work[idx++];
                std::memset(&o, 0, sizeof(o));
                o.patch = h_patch[k];
                o.level = h_level ? h_level[k] : 0;
                for (int d = 0; d < 8; ++d) o.nbr[d] = h_nbr ? h_nbr[8 * k + d] : -1;
                // near-equal split of [lo, lo + w) into ntx x nty pieces
                o.x0 = (int16_t)(lo + (w * tx) / ntx);
                o.x1 = (int16_t)(lo + (w * (tx + 1)) / ntx);
                o.y0 = (int16_t)(lo + (w * ty) / nty);
                o.y1 = (int16_t)(lo + (w * (ty + 1)) / nty);
                o.flags = ext ? 1 : 0;
                o.ix = h_ix ? h_ix[k] : 0;
                o.iy = h_iy ? h_iy[k] : 0;
            }
    }
    return AF_OK;
}

extern "C" af_status af_build_step_work_tiled(const af_config *cfg, int32_t tiling_index, int32_t npatch,
                                              const int32_t *h_patch, const int32_t *h_level, const int32_t *h_nbr,
                                              af_work *h_work, int32_t capacity, int32_t *nwork) {
    return af_build_step_work_at(cfg, tiling_index, npatch, h_patch, h_level, nullptr, nullptr, h_nbr, h_work,
                                 capacity, nwork);
}

extern "C" af_status af_build_step_work(const af_config *cfg, int32_t npatch, const int32_t *h_patch,
                                        const int32_t *h_level, const int32_t *h_nbr, af_work *h_work,
                                        int32_t capacity, int32_t *nwork) {
    if (cfg == nullptr) return AF_ERR_ARG;
    return af_build_step_work_tiled(cfg, af::default_tiling(cfg->n), npatch, h_patch, h_level, h_nbr, h_work,
                                    capacity, nwork);
}

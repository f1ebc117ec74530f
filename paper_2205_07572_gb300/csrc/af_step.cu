// Host side of af_patch_step (Section 2 of arXiv 2205.07572): argument and
// CFL checks (Eq. cfl-adv, Eq. cfl-acoustics), the cached stencil weights,
// and the choice of compiled tiling.  The kernels are in
// af_step_kernels.cuh, instantiated per precision in af_step_f32.cu and
// af_step_f64.cu.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "af_step_kernels.cuh"

namespace af {
namespace {

struct WeightKey {
    int eq;
    double r0, r1;
    bool operator==(const WeightKey &o) const { return eq == o.eq && r0 == o.r0 && r1 == o.r1; }
};

std::mutex g_mu;

WeightKey g_skey{-1, 0, 0}, g_dkey{-1, 0, 0};
AcousticSymWeights<double> g_sw;
bool g_sw_ok = false;
AdvectionWeights<double> g_dw;

template <typename T>
bool get_acoustic(double rx, double ry, AcousticSymWeights<T> &out) {
    std::lock_guard<std::mutex> lk(g_mu);
    const WeightKey k{AF_ACOUSTICS, rx, ry};
    if (!(k == g_skey)) {
        g_sw_ok = acoustic_sym_weights(rx, ry, g_sw);
        g_skey = k;
    }
    constexpr int nw = sizeof(AcousticSymWeights<double>) / sizeof(double);
    static_assert(sizeof(AcousticSymWeights<T>) == nw * sizeof(T), "packed weight struct");
    const double *src = &g_sw.cA[0][0];
    T *dst = &out.cA[0][0];
    for (int i = 0; i < nw; ++i) dst[i] = (T)src[i];
    return g_sw_ok;
}

template <typename T>
void get_advection(double nx, double ny, AdvectionWeights<T> &out) {
    std::lock_guard<std::mutex> lk(g_mu);
    const WeightKey k{AF_ADVECTION, nx, ny};
    if (!(k == g_dkey)) {
        advection_weights(nx, ny, g_dw);
        g_dkey = k;
    }
    for (int t = 0; t < 3; ++t)
        for (int s = 0; s < 2; ++s) {
            for (int d = 0; d < 9; ++d) out.w[t][s][d] = (T)g_dw.w[t][s][d];
            out.off[t][s][0] = g_dw.off[t][s][0];
            out.off[t][s][1] = g_dw.off[t][s][1];
        }
}

// Interleave the two time combinations (T, Q^{n+1}) of every FP32 weight.
void pair_weights(const AcousticSymWeights<float> &s, AcousticPairWeights &p) {
    for (int k = 0; k < 9; ++k) for (int t = 0; t < 2; ++t) p.cA[k][t] = s.cA[t][k];
    for (int k = 0; k < 6; ++k) for (int t = 0; t < 2; ++t) p.cDx[k][t] = s.cDx[t][k], p.cDy[k][t] = s.cDy[t][k];
    for (int k = 0; k < 6; ++k) for (int t = 0; t < 2; ++t) p.xA[k][t] = s.xA[t][k], p.yA[k][t] = s.yA[t][k];
    for (int k = 0; k < 4; ++k) for (int t = 0; t < 2; ++t) p.xDx[k][t] = s.xDx[t][k], p.yDy[k][t] = s.yDy[t][k];
    for (int k = 0; k < 3; ++k) for (int t = 0; t < 2; ++t) p.xDy[k][t] = s.xDy[t][k], p.yDx[k][t] = s.yDx[t][k];
}

template <typename T, int EQ>
af_status launch(int k, const af_config &cfg, int nwork, const af_work *d_work, const void *d_in, void *d_out,
                 uint32_t swap, double dt0, double dx0, double dy0, double *d_freg, cudaStream_t stream) {
    StepArgs<T> A;
    A.swap = swap;
    A.work = d_work;
    A.in = static_cast<const T *>(d_in);
    A.out = static_cast<T *>(d_out);
    A.freg = d_freg;
    A.plane = plane_stride(cfg.n);
    A.n = cfg.n;
    A.ncomp = cfg.ncomp;
    A.dtdx = (T)(dt0 / dx0);
    A.dtdy = (T)(dt0 / dy0);
    A.dt0 = dt0;
    typename WeightsOf<T, EQ>::type W;
    if constexpr (EQ == AF_ACOUSTICS) {
        A.fx = A.fy = (T)(cfg.c / 36.0);
        if constexpr (sizeof(T) == 4) {
            AcousticSymWeights<float> sw;
            if (!get_acoustic<float>(cfg.c * dt0 / dx0, cfg.c * dt0 / dy0, sw)) return AF_ERR_UNIMPLEMENTED;
            pair_weights(sw, W);
        } else {
            if (!get_acoustic<T>(cfg.c * dt0 / dx0, cfg.c * dt0 / dy0, W)) return AF_ERR_UNIMPLEMENTED;
        }
    } else {
        A.fx = (T)(cfg.a / 36.0);
        A.fy = (T)(cfg.b / 36.0);
        get_advection<T>(cfg.a * dt0 / dx0, cfg.b * dt0 / dy0, W);
    }
    return launch_step<T, EQ>(k, A, W, nwork, stream);
}

}  // namespace
}  // namespace af

extern "C" int32_t af_step_tilings(af_tiling *out, int32_t capacity) {
    using namespace af;
    for (int k = 0; k < kNumTilings && k < capacity && out; ++k) {
        const Tiling t = tiling(k);
        out[k].tile_x = t.tmx;
        out[k].tile_y = t.tmy;
        out[k].threads = t.threads;
        out[k].persistent = t.persistent;
    }
    return kNumTilings;
}

extern "C" int32_t af_step_default_tiling(const af_config *cfg) {
    return cfg ? af::default_tiling(cfg->n) : -1;
}

namespace af {
namespace {

af_status step_checked(const af_config *cfg, int32_t tiling_index, int32_t nwork, const af_work *d_work,
                       const void *d_in, void *d_out, uint32_t swap, double dt0, double dx0, double dy0,
                       double *d_flux_reg, void *stream) {
    if (cfg == nullptr || nwork < 0) return AF_ERR_ARG;
    if (tiling_index < 0 || tiling_index >= kNumTilings) return AF_ERR_ARG;
    if (cfg->n < 2 || cfg->n > 64) return AF_ERR_ARG;
    if (cfg->eq != AF_ADVECTION && cfg->eq != AF_ACOUSTICS) return AF_ERR_ARG;
    if (cfg->prec != AF_F64 && cfg->prec != AF_F32) return AF_ERR_ARG;
    if (cfg->ncomp != (cfg->eq == AF_ADVECTION ? 1 : 3)) return AF_ERR_ARG;
    if (!(dt0 > 0.0) || !(dx0 > 0.0) || !(dy0 > 0.0)) return AF_ERR_ARG;
    if (nwork == 0) return AF_OK;
    if (d_work == nullptr || d_in == nullptr || d_out == nullptr) return AF_ERR_ARG;
    if (d_in == d_out) return AF_ERR_ARG;
    if ((reinterpret_cast<uintptr_t>(d_in) | reinterpret_cast<uintptr_t>(d_out)) & 31u) return AF_ERR_LAYOUT;
    if (reinterpret_cast<uintptr_t>(d_work) & 15u) return AF_ERR_LAYOUT;
    if (reinterpret_cast<uintptr_t>(d_flux_reg) & 7u) return AF_ERR_LAYOUT;
    const double tol = 1e-12;
    if (cfg->eq == AF_ADVECTION) {
        // strict: the foot of every characteristic must stay within one cell
        // of its node, which bounds the kernel's shared-memory window
        if (!(std::fabs(cfg->a) * dt0 / dx0 <= 1.0) || !(std::fabs(cfg->b) * dt0 / dy0 <= 1.0)) return AF_ERR_CFL;
    } else {
        if (!(cfg->c > 0.0)) return AF_ERR_ARG;
        if (cfg->c * dt0 / dx0 > 0.5 + tol || cfg->c * dt0 / dy0 > 0.5 + tol) return AF_ERR_CFL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int k = tiling_index;
    if (cfg->prec == AF_F64)
        return cfg->eq == AF_ACOUSTICS
                   ? launch<double, AF_ACOUSTICS>(k, *cfg, nwork, d_work, d_in, d_out, swap, dt0, dx0, dy0, d_flux_reg, s)
                   : launch<double, AF_ADVECTION>(k, *cfg, nwork, d_work, d_in, d_out, swap, dt0, dx0, dy0, d_flux_reg, s);
    return cfg->eq == AF_ACOUSTICS
               ? launch<float, AF_ACOUSTICS>(k, *cfg, nwork, d_work, d_in, d_out, swap, dt0, dx0, dy0, d_flux_reg, s)
               : launch<float, AF_ADVECTION>(k, *cfg, nwork, d_work, d_in, d_out, swap, dt0, dx0, dy0, d_flux_reg, s);
}

}  // namespace
}  // namespace af

extern "C" af_status af_patch_step_tiled(const af_config *cfg, int32_t tiling_index, int32_t nwork,
                                         const af_work *d_work, const void *d_in, void *d_out, double dt0,
                                         double dx0, double dy0, double *d_flux_reg, void *stream) {
    return af::step_checked(cfg, tiling_index, nwork, d_work, d_in, d_out, 0u, dt0, dx0, dy0, d_flux_reg, stream);
}

extern "C" af_status af_patch_step_pair(const af_config *cfg, int32_t tiling_index, int32_t nwork,
                                        const af_work *d_work, const af_state_pair *state, double dt0, double dx0,
                                        double dy0, double *d_flux_reg, void *stream) {
    if (state == nullptr) return AF_ERR_ARG;
    return af::step_checked(cfg, tiling_index, nwork, d_work, state->buf[0], state->buf[1], state->parity, dt0, dx0,
                            dy0, d_flux_reg, stream);
}

extern "C" af_status af_patch_step(const af_config *cfg, int32_t nwork, const af_work *d_work, const void *d_in,
                                   void *d_out, double dt0, double dx0, double dy0, double *d_flux_reg,
                                   void *stream) {
    if (cfg == nullptr) return AF_ERR_ARG;
    return af_patch_step_tiled(cfg, af::default_tiling(cfg->n), nwork, d_work, d_in, d_out, dt0, dx0, dy0,
                               d_flux_reg, stream);
}

extern "C" af_status af_step_wait_timeouts(uint32_t *count, int32_t reset) {
    if (count == nullptr) return AF_ERR_ARG;
    unsigned int a = 0, b = 0, c = 0, d = 0, e = 0, f = 0;
    af_status st = af::wait_timeouts_f32(&a, reset != 0);
    if (st == AF_OK) st = af::wait_timeouts_f64(&b, reset != 0);
    if (st == AF_OK) st = af::wait_timeouts_f32_n16(&c, reset != 0);
    if (st == AF_OK) st = af::wait_timeouts_f32_n32(&d, reset != 0);
    if (st == AF_OK) st = af::wait_timeouts_var(&e, reset != 0);
    if (st == AF_OK) st = af::wait_timeouts_cnn(&f, reset != 0);
    if (st != AF_OK) return st;
    *count = a + b + c + d + e + f;
    return AF_OK;
}

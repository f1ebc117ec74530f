// af_patch_step_var: one Active Flux step of variable-velocity advection
// (Sections 4.2 and 4.3 of arXiv 2205.07572) on GB300.
//
// The tile staging, the same-level halo and the whole-patch copy of patches
// that advance their ghost layer are those of the constant-velocity kernel
// (af_step_kernels.cuh).  The velocity depends on position (and, for the
// swirl, on time), so the evolved point values are no longer fixed stencils:
// every node traces its characteristic back to t^n -- an exact rotation for
// solid-body rotation, one classical Runge-Kutta step for the swirl -- and
// evaluates the reconstruction (Eq. poly) of the cell holding the foot.  The
// fluxes take the velocity at their quadrature points (solid body) or at the
// face centre for each time level (Eqs. swirlF, swirlG).
#include <cuda_runtime.h>

#include <cmath>

#include "af_step_kernels.cuh"

namespace af {
namespace dev {

template <typename T>
struct VarArgs {
    StepArgs<T> s;      // work list, buffers, flux registers, layout
    double x_lo, y_lo;  // node line 0 of patch (0, 0)
    double t;           // t^n
    double dx0, dy0;    // level-0 mesh widths
    // swirl, per level l (host-computed once per call): cos(pi t) at t^n,
    // t^n + dt_l/4, t^n + dt_l/2, t^n + dt_l, and sin(pi h) / (pi h) for
    // h = dx_l, dy_l
    double cl[AF_MAX_LEVEL + 1][4];
    double kl[AF_MAX_LEVEL + 1][2];
};

__device__ __forceinline__ float spi(float x) { return sinpif(x); }
__device__ __forceinline__ double spi(double x) { return sinpi(x); }
__device__ __forceinline__ float cpi(float x) { return cospif(x); }
__device__ __forceinline__ double cpi(double x) { return cospi(x); }

__device__ __forceinline__ void scpi(float x, float &s, float &c) { sincospif(x, &s, &c); }
__device__ __forceinline__ void scpi(double x, double &s, double &c) { sincospi(x, &s, &c); }

// Swirl velocity: the centred differences of Eq. swirlODE written as
// -sin^2(pi x) sin(2 pi y) cos(pi t) sin(pi dy) / (pi dy) and its mirror,
// with sin(2 pi y) = 2 sin(pi y) cos(pi y).  kx = sin(pi dx) / (pi dx), ky
// likewise; ct = cos(pi t).
template <typename T>
__device__ __forceinline__ void swirl_v(T x, T y, T ct, T kx, T ky, T &a, T &b) {
    T sx, cx, sy, cy;
    scpi(x, sx, cx);
    scpi(y, sy, cy);
    a = -sx * sx * (T(2) * sy * cy) * ct * ky;
    b = sy * sy * (T(2) * sx * cx) * ct * kx;
}

// Time-independent factor of the swirl velocity at a face centre:
// a(x, y, t) = ax * cos(pi t) (x-faces), b(x, y, t) = by * cos(pi t) (y-faces).
template <typename T>
__device__ __forceinline__ T swirl_ax(T x, T y, T ky) {
    T sx, cx, sy, cy;
    scpi(x, sx, cx);
    scpi(y, sy, cy);
    return -sx * sx * (T(2) * sy * cy) * ky;
}
template <typename T>
__device__ __forceinline__ T swirl_by(T x, T y, T kx) {
    T sx, cx, sy, cy;
    scpi(x, sx, cx);
    scpi(y, sy, cy);
    return sy * sy * (T(2) * sx * cx) * kx;
}

// Per-tile constants of one level.
template <typename T>
struct VarLevel {
    T dx, dy, dt;
    T c[4];     // cos(pi t) at t^n, t^n + dt/4, t^n + dt/2, t^n + dt
    T kx, ky;   // swirl difference factors
    T xo, yo;   // patch corner (node line 0)
};

// Foot at t^n of the characteristic through (x, y) at t^n + tau; `half`
// selects tau = dt/2 (else dt).
template <typename T, int FIELD>
__device__ __forceinline__ void foot(const VarLevel<T> &L, T x, T y, bool half, T &xf, T &yf) {
    const T tau = half ? T(0.5) * L.dt : L.dt;
    if constexpr (FIELD == AF_FIELD_SOLID_BODY) {
        const T c = cpi(tau), s = spi(tau);
        xf = x * c + y * s;
        yf = -x * s + y * c;
    } else {
        // stage times t + tau, t + tau/2, t + tau/2, t
        const T c1 = half ? L.c[2] : L.c[3], c2 = half ? L.c[1] : L.c[2], c3 = L.c[0];
        const T h = -tau;
        T k1a, k1b, k2a, k2b, k3a, k3b, k4a, k4b;
        swirl_v(x, y, c1, L.kx, L.ky, k1a, k1b);
        swirl_v(x + T(0.5) * h * k1a, y + T(0.5) * h * k1b, c2, L.kx, L.ky, k2a, k2b);
        swirl_v(x + T(0.5) * h * k2a, y + T(0.5) * h * k2b, c2, L.kx, L.ky, k3a, k3b);
        swirl_v(x + h * k3a, y + h * k3b, c3, L.kx, L.ky, k4a, k4b);
        xf = x + h / T(6) * (k1a + T(2) * k2a + T(2) * k3a + k4a);
        yf = y + h / T(6) * (k1b + T(2) * k2b + T(2) * k3b + k4b);
    }
}

// Reconstruction of the staged cell holding (xf, yf); cells x0-1 .. x1 and
// y0-1 .. y1 of the patch are in the window (pitch WX, plane size WSZ).
template <typename T, int WX, int WSZ>
__device__ __forceinline__ T eval_at(const VarLevel<T> &L, const T *Sin, int x0, int x1, int y0, int y1, T xf,
                                     T yf) {
    const T fx = (xf - L.xo) / L.dx, fy = (yf - L.yo) / L.dy;
    int ci = (int)floor(fx), cj = (int)floor(fy);
    ci = ci < x0 - 1 ? x0 - 1 : (ci > x1 ? x1 : ci);
    cj = cj < y0 - 1 ? y0 - 1 : (cj > y1 ? y1 : cj);
    const T xi = T(2) * (fx - (T)ci) - T(1), eta = T(2) * (fy - (T)cj) - T(1);
    const int o = (cj - y0 + 1) * WX + (ci - x0 + 1);
    const T *A = Sin + kAvg * WSZ, *Cr = Sin + kCorner * WSZ, *X = Sin + kXmid * WSZ, *Y = Sin + kYmid * WSZ;
    const T c00 = Cr[o], c10 = Cr[o + 1], c01 = Cr[o + WX], c11 = Cr[o + WX + 1];
    const T xl = X[o], xr = X[o + 1], yb = Y[o], yt = Y[o + WX];
    const T cen = T(2.25) * A[o] - T(0.0625) * (c00 + c10 + c01 + c11) - T(0.25) * (xl + xr + yb + yt);
    const T lx0 = T(0.5) * xi * (xi - T(1)), lx1 = T(1) - xi * xi, lx2 = T(0.5) * xi * (xi + T(1));
    const T ly0 = T(0.5) * eta * (eta - T(1)), ly1 = T(1) - eta * eta, ly2 = T(0.5) * eta * (eta + T(1));
    return ly0 * (lx0 * c00 + lx1 * yb + lx2 * c10) + ly1 * (lx0 * xl + lx1 * cen + lx2 * xr) +
           ly2 * (lx0 * c01 + lx1 * yt + lx2 * c11);
}

template <typename T, int FIELD, int NT, int TMX, int TMY>
__global__ void __launch_bounds__(NT) step_var_kernel(const __grid_constant__ VarArgs<T> V) {
    using Gm = Geo<TMX, TMY>;
    constexpr int WX = Gm::WX, WSZ = Gm::WSZ, TX = Gm::TX, TSZ = Gm::TSZ;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *const Sbase = reinterpret_cast<T *>(smem_raw);
    T *const Sin = Sbase + win_off<T, WX>();
    T *ST = Sbase + kPlanes * WSZ;  // [node type][half, full][TSZ]
    const StepArgs<T> &A = V.s;
    const af_work wk = A.work[blockIdx.x];
    if (wk.x1 - wk.x0 > TMX || wk.y1 - wk.y0 > TMY) return;
    const bool bulk = bulk_tile<T, WX>(A, wk);
    if (bulk) {  // bulk (TMA) copies of the window rows, as in the constant-velocity step
        __shared__ __align__(8) uint64_t bar;
        if (!stage_bulk<T, NT, WX, WSZ, 1>(A, wk, Sin, &bar)) return;  // counted in g_wait_timeouts
    } else {
        stage_issue<T, NT, WX, WSZ>(A, wk, Sin);
        cp_async_commit();
        cp_async_wait_all();
        __syncthreads();
    }
    if (wk.flags & 1) {
        stage_copy_out<T, NT, WX, WSZ>(A, wk, Sin);
        __syncthreads();
    }
    const int n = A.n, W_ = n + 2 * kGhost + 1, plane = (int)A.plane, level = wk.level;
    const int x0 = wk.x0, x1 = wk.x1, y0 = wk.y0, y1 = wk.y1, tw = x1 - x0, th = y1 - y0;
    VarLevel<T> L;
    L.dx = (T)ldexp(V.dx0, -level);
    L.dy = (T)ldexp(V.dy0, -level);
    L.dt = (T)ldexp(A.dt0, -level);
    L.xo = (T)(V.x_lo + (double)wk.ix * n * ldexp(V.dx0, -level));
    L.yo = (T)(V.y_lo + (double)wk.iy * n * ldexp(V.dy0, -level));
    if constexpr (FIELD == AF_FIELD_SWIRL) {
#pragma unroll
        for (int q = 0; q < 4; ++q) L.c[q] = (T)V.cl[level][q];
        L.kx = (T)V.kl[level][0];
        L.ky = (T)V.kl[level][1];
    }
    T *outp = dst_buf(A, level) + (int64_t)wk.patch * kPlanes * A.plane;
    const int sxhi = (x1 == n + 1) ? x1 : x1 - 1;
    const int syhi = (y1 == n + 1) ? y1 : y1 - 1;

    // ---- point values at t^{n+1/2}, t^{n+1}: node-cells (ii, jj) in [0, tw] x [0, th]
    for (int it = threadIdx.x; it < (tw + 1) * (th + 1); it += NT) {
        const int jj = it / (tw + 1), ii = it - jj * (tw + 1);
        const int i = x0 + ii, j = y0 + jj;
        const bool hx = j < y1, hy = i < x1;
        const bool st_x = i <= sxhi, st_y = j <= syhi;
        const int so = jj * TX + ii;
        T *const ob = outp + ((j + kGhost) * W_ + (i + kGhost));
#pragma unroll
        for (int ty = 0; ty < 3; ++ty) {
            if ((ty == 1 && !hx) || (ty == 2 && !hy)) continue;
            const T x = L.xo + ((T)i + (ty == 2 ? T(0.5) : T(0))) * L.dx;
            const T y = L.yo + ((T)j + (ty == 1 ? T(0.5) : T(0))) * L.dy;
            T xf, yf;
            foot<T, FIELD>(L, x, y, true, xf, yf);
            const T qh = eval_at<T, WX, WSZ>(L, Sin, x0, x1, y0, y1, xf, yf);
            foot<T, FIELD>(L, x, y, false, xf, yf);
            const T q1 = eval_at<T, WX, WSZ>(L, Sin, x0, x1, y0, y1, xf, yf);
            ST[(ty * 2 + 0) * TSZ + so] = qh;
            ST[(ty * 2 + 1) * TSZ + so] = q1;
            if (ty == 0 && st_x && st_y) ob[kCorner * plane] = q1;
            if (ty == 1 && st_x) ob[kXmid * plane] = q1;
            if (ty == 2 && st_y) ob[kYmid * plane] = q1;
        }
    }
    __syncthreads();

    // ---- fluxes and update of cells [x0, x1) x [y0, y1)
    const double dtl = ldexp(A.dt0, -level);
    const T w[3] = {T(1), T(4), T(1)};
    for (int it = threadIdx.x; it < tw * th; it += NT) {
        const int jj = it / tw, ii = it - jj * tw;
        const int i = x0 + ii, j = y0 + jj;
        const int so = jj * TX + ii, sw = (jj + 1) * WX + (ii + 1);
        const T *Cn = Sin + kCorner * WSZ, *Xn = Sin + kXmid * WSZ, *Yn = Sin + kYmid * WSZ;
        // the three face points at t^n, t^{n+1/2}, t^{n+1}: q(k, s)
        auto corner = [&](int k, int dq, int dw) -> T {
            return k == 0 ? Cn[sw + dw] : ST[(0 * 2 + k - 1) * TSZ + so + dq];
        };
        auto xmid = [&](int k, int dq, int dw) -> T {
            return k == 0 ? Xn[sw + dw] : ST[(1 * 2 + k - 1) * TSZ + so + dq];
        };
        auto ymid = [&](int k, int dq, int dw) -> T {
            return k == 0 ? Yn[sw + dw] : ST[(2 * 2 + k - 1) * TSZ + so + dq];
        };
        // x-face on node line i + di (di = 0 left, 1 right); y-face on j + dj
        auto xflux = [&](int di) -> T {
            const T xs = L.xo + (T)(i + di) * L.dx;
            T ax = T(0);
            if constexpr (FIELD == AF_FIELD_SWIRL) ax = swirl_ax(xs, L.yo + ((T)j + T(0.5)) * L.dy, L.ky);
            T acc = T(0);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const T ql = corner(k, di, di), qm = xmid(k, di, di), qu = corner(k, di + TX, di + WX);
                if constexpr (FIELD == AF_FIELD_SOLID_BODY) {
                    const T y0s = L.yo + (T)j * L.dy;
                    acc += w[k] * (-T(M_PI)) *
                           (y0s * ql + T(4) * (y0s + T(0.5) * L.dy) * qm + (y0s + L.dy) * qu);
                } else {
                    const T a = ax * L.c[k == 0 ? 0 : (k == 1 ? 2 : 3)];
                    acc += w[k] * a * (ql + T(4) * qm + qu);
                }
            }
            return acc / T(36);
        };
        auto yflux = [&](int dj) -> T {
            const T ys = L.yo + (T)(j + dj) * L.dy;
            T by = T(0);
            if constexpr (FIELD == AF_FIELD_SWIRL) by = swirl_by(L.xo + ((T)i + T(0.5)) * L.dx, ys, L.kx);
            T acc = T(0);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const T ql = corner(k, dj * TX, dj * WX), qm = ymid(k, dj * TX, dj * WX),
                        qr = corner(k, dj * TX + 1, dj * WX + 1);
                if constexpr (FIELD == AF_FIELD_SOLID_BODY) {
                    const T x0s = L.xo + (T)i * L.dx;
                    acc += w[k] * T(M_PI) * (x0s * ql + T(4) * (x0s + T(0.5) * L.dx) * qm + (x0s + L.dx) * qr);
                } else {
                    const T b = by * L.c[k == 0 ? 0 : (k == 1 ? 2 : 3)];
                    acc += w[k] * b * (ql + T(4) * qm + qr);
                }
            }
            return acc / T(36);
        };
        const T fl = xflux(0), fr = xflux(1), gb = yflux(0), gt = yflux(1);
        const T q = Sin[kAvg * WSZ + sw];
        outp[(j + kGhost) * W_ + (i + kGhost)] = q - L.dt / L.dx * (fr - fl) - L.dt / L.dy * (gt - gb);
        if (A.freg != nullptr) {
            double *fr_p = A.freg + (int64_t)wk.patch * 4 * n;
            const bool iny = (j >= 0 && j < n), inx = (i >= 0 && i < n);
            if (iny && i == 0) fr_p[0 * n + j] += dtl * (double)fl;
            if (iny && i == n - 1) fr_p[1 * n + j] += dtl * (double)fr;
            if (inx && j == 0) fr_p[2 * n + i] += dtl * (double)gb;
            if (inx && j == n - 1) fr_p[3 * n + i] += dtl * (double)gt;
        }
    }
    if (bulk) write_ghost_columns<T, NT, WX, WSZ, 1>(A, wk, Sin);
}

template <typename T, int FIELD, int NT, int TMX, int TMY>
af_status launch_var_tiling(const VarArgs<T> &V, int nwork, cudaStream_t stream) {
    using Gm = Geo<TMX, TMY>;
    const size_t smem = sizeof(T) * ((size_t)kPlanes * Gm::WSZ + 6 * (size_t)Gm::TSZ);
    if (smem > 227 * 1024) return AF_ERR_UNIMPLEMENTED;
    auto kern = step_var_kernel<T, FIELD, NT, TMX, TMY>;
    if (ensure_smem(kern, smem) != cudaSuccess) return AF_ERR_CUDA;
    kern<<<nwork, NT, smem, stream>>>(V);
    return cudaGetLastError() == cudaSuccess ? AF_OK : AF_ERR_CUDA;
}

// The persistent tiling (a CTA looping over tiles) runs here as one tile per CTA.
#define AF_VAR_CASE(K) \
    case K:            \
        return launch_var_tiling<T, FIELD, tiling(K).threads, tiling(K).tmx, tiling(K).tmy>(V, nwork, stream);

template <typename T, int FIELD>
af_status launch_var(int k, const VarArgs<T> &V, int nwork, cudaStream_t stream) {
    static_assert(kNumTilings == 10, "one case per compiled tiling");
    switch (k) {
        AF_VAR_CASE(0)
        AF_VAR_CASE(1)
        AF_VAR_CASE(2)
        AF_VAR_CASE(3)
        AF_VAR_CASE(4)
        AF_VAR_CASE(5)
        AF_VAR_CASE(6)
        AF_VAR_CASE(7)
        AF_VAR_CASE(8)
        AF_VAR_CASE(9)
    }
    return AF_ERR_ARG;
}

}  // namespace dev
}  // namespace af

extern "C" af_status af_patch_step_var(const af_config *cfg, int32_t tiling_index, int32_t nwork,
                                       const af_work *d_work, const af_state_pair *state, const af_velocity *vel,
                                       double dt0, double dx0, double dy0, double *d_flux_reg, void *stream) {
    using namespace af;
    if (cfg == nullptr || state == nullptr || vel == nullptr || nwork < 0) return AF_ERR_ARG;
    if (tiling_index < 0 || tiling_index >= kNumTilings) return AF_ERR_ARG;
    if (cfg->eq != AF_ADVECTION || cfg->ncomp != 1 || cfg->n < 2 || cfg->n > 64) return AF_ERR_ARG;
    if (cfg->prec != AF_F64 && cfg->prec != AF_F32) return AF_ERR_ARG;
    if (vel->field != AF_FIELD_SOLID_BODY && vel->field != AF_FIELD_SWIRL) return AF_ERR_ARG;
    if (!(dt0 > 0.0) || !(dx0 > 0.0) || !(dy0 > 0.0)) return AF_ERR_ARG;
    if (!(vel->x_hi > vel->x_lo) || !(vel->y_hi > vel->y_lo)) return AF_ERR_ARG;
    if (nwork == 0) return AF_OK;
    void *b0 = state->buf[0], *b1 = state->buf[1];
    if (d_work == nullptr || b0 == nullptr || b1 == nullptr || b0 == b1) return AF_ERR_ARG;
    if ((reinterpret_cast<uintptr_t>(b0) | reinterpret_cast<uintptr_t>(b1)) & 31u) return AF_ERR_LAYOUT;
    if (reinterpret_cast<uintptr_t>(d_work) & 15u) return AF_ERR_LAYOUT;
    if (reinterpret_cast<uintptr_t>(d_flux_reg) & 7u) return AF_ERR_LAYOUT;
    // speed bound over the domain and its two ghost layers at level 0
    double vmax;
    if (vel->field == AF_FIELD_SOLID_BODY) {
        const double ex = 3.0 * dx0, ey = 3.0 * dy0;
        const double mx = std::fmax(std::fabs(vel->x_lo - ex), std::fabs(vel->x_hi + ex));
        const double my = std::fmax(std::fabs(vel->y_lo - ey), std::fabs(vel->y_hi + ey));
        vmax = M_PI * std::fmax(mx, my);
    } else {
        vmax = 1.0;  // |sin^2 sin| <= 1 and sin(pi h) / (pi h) <= 1
    }
    if (!(vmax * dt0 <= std::fmin(dx0, dy0))) return AF_ERR_CFL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int k = tiling_index;
    auto fill = [&](auto &V) {
        V.s.work = d_work;
        V.s.freg = d_flux_reg;
        V.s.plane = plane_stride(cfg->n);
        V.s.n = cfg->n;
        V.s.ncomp = 1;
        V.s.dt0 = dt0;
        V.s.swap = state->parity;
        V.x_lo = vel->x_lo;
        V.y_lo = vel->y_lo;
        V.t = vel->t;
        V.dx0 = dx0;
        V.dy0 = dy0;
        for (int l = 0; l <= AF_MAX_LEVEL; ++l) {
            const double dtl = std::ldexp(dt0, -l), hx = std::ldexp(dx0, -l), hy = std::ldexp(dy0, -l);
            V.cl[l][0] = std::cos(M_PI * vel->t);
            V.cl[l][1] = std::cos(M_PI * (vel->t + 0.25 * dtl));
            V.cl[l][2] = std::cos(M_PI * (vel->t + 0.5 * dtl));
            V.cl[l][3] = std::cos(M_PI * (vel->t + dtl));
            V.kl[l][0] = std::sin(M_PI * hx) / (M_PI * hx);
            V.kl[l][1] = std::sin(M_PI * hy) / (M_PI * hy);
        }
    };
    if (cfg->prec == AF_F64) {
        dev::VarArgs<double> V{};
        fill(V);
        V.s.in = static_cast<const double *>(b0);
        V.s.out = static_cast<double *>(b1);
        return vel->field == AF_FIELD_SOLID_BODY ? dev::launch_var<double, AF_FIELD_SOLID_BODY>(k, V, nwork, s)
                                                 : dev::launch_var<double, AF_FIELD_SWIRL>(k, V, nwork, s);
    }
    dev::VarArgs<float> V{};
    fill(V);
    V.s.in = static_cast<const float *>(b0);
    V.s.out = static_cast<float *>(b1);
    return vel->field == AF_FIELD_SOLID_BODY ? dev::launch_var<float, AF_FIELD_SOLID_BODY>(k, V, nwork, s)
                                             : dev::launch_var<float, AF_FIELD_SWIRL>(k, V, nwork, s);
}

namespace af {
af_status wait_timeouts_var(unsigned int *count, bool reset) { return wait_timeouts_here(count, reset); }
}  // namespace af

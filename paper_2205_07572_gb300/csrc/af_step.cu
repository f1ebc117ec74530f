// af_patch_step: one Active Flux time step (Section 2 of arXiv 2205.07572)
// on GB300 (sm_103a).
//
// One CTA advances one tile (<= 32 x 32 cells) of one patch:
//   stage  - the tile's degrees of freedom plus a one-cell halo are copied to
//            shared memory; halo entries in a direction with a same-level
//            neighbour are read straight from that neighbour's interior (the
//            same-level ghost copy of Section 3.1 fused into the load), other
//            directions from the patch's own ghost ring;
//   nodes  - one thread per node-cell evolves the corner, left-edge midpoint
//            and bottom-edge midpoint of its cell to t^{n+1/2} and t^{n+1}
//            (Eq. advection-update / Eq. ERFormula) as constant-weight
//            stencils, keeps T = Q^n + 4 Q^{n+1/2} + Q^{n+1} in shared memory
//            and writes Q^{n+1} to the output;
//   update - one thread per cell forms the four face fluxes by the space-time
//            Simpson rule (Eq. Simpson-2d: f is linear, so the 3 x 3 sum is
//            f((T_lo + 4 T_mid + T_hi) / 36)) and applies Eq. 2dfv.
// No tensor cores: the stencil is not a dense contraction.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "af_internal.h"

namespace af {
namespace {

template <typename T>
struct StepArgs {
    const af_work *work;
    const T *in;
    T *out;
    double *freg;
    int64_t plane;   // plane stride (elements)
    int n, ncomp;
    int wn;          // shared-memory pitch of a staged plane (tile max + 3)
    int tp;          // pitch of the T arrays (tile max + 1)
    T dtdx, dtdy;    // dt/dx and dt/dy (the same on every level)
    T fx, fy;        // flux scale: advection a/36, b/36; acoustics c/36
    double dt0;      // level-0 time step (flux registers)
};

__device__ __forceinline__ int dir_index(int sx, int sy) {
    if (sy == 0) return sx < 0 ? 0 : 1;
    if (sx == 0) return sy < 0 ? 2 : 3;
    return 4 + (sx > 0 ? 1 : 0) + (sy > 0 ? 2 : 0);
}

__device__ __forceinline__ void cp_async(float *smem, const float *gmem) {
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async(double *smem, const double *gmem) {
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\n" ::);
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// Lattice offset (within the state) of window entry (li, lj) of `patch`:
// from the same-level neighbour in that direction if there is one, else
// from the patch itself (its interior or its ghost ring).
template <typename T>
__device__ __forceinline__ int64_t window_source(const StepArgs<T> &A, int patch, const int *s_nbr, int li, int lj) {
    const int n = A.n, W = n + 2 * kGhost + 1;
    const int64_t pw = (int64_t)A.ncomp * kPlanes * A.plane;
    const int sx = li < 0 ? -1 : (li >= n ? 1 : 0);
    const int sy = lj < 0 ? -1 : (lj >= n ? 1 : 0);
    int src = patch, si = li, sj = lj;
    if (sx | sy) {
        const int nb = s_nbr[dir_index(sx, sy)];
        if (nb >= 0) {
            src = nb;
            si = li - sx * n;
            sj = lj - sy * n;
        }
    }
    return (int64_t)src * pw + (int64_t)(sj + kGhost) * W + (si + kGhost);
}

// Stage the window of node lines [x0-1, x1+1] x [y0-1, y1+1] of every plane
// with asynchronous global->shared copies (all in flight at once), then wait.
// For a patch that advances its ghost layer (copy_all), the tile also writes
// the staged entries of its share of the patch's lattice to the output, so
// the output holds a complete patch (advanced entries are overwritten later).
template <typename T, int NT, int WN>
__device__ __forceinline__ void stage(const StepArgs<T> &A, int patch, const int *s_nbr, int x0, int y0,
                                      int x1, int y1, int ww, int wh, bool copy_all, T *Sin) {
    const int ncp = A.ncomp * kPlanes;
    constexpr int wsz = WN * WN;
    for (int pos = threadIdx.x; pos < ww * wh; pos += NT) {
        const int row = pos / ww, col = pos - row * ww;
        const T *g = A.in + window_source(A, patch, s_nbr, x0 - 1 + col, y0 - 1 + row);
        T *s = Sin + row * WN + col;
#pragma unroll 4
        for (int cp = 0; cp < ncp; ++cp) cp_async(s + cp * wsz, g + cp * A.plane);
    }
    cp_async_wait_all();
    __syncthreads();
    if (copy_all) {
        const int n = A.n, W = n + 2 * kGhost + 1;
        const int64_t pw = (int64_t)A.ncomp * kPlanes * A.plane;
        // share of the lattice [-2, n+2]^2 this tile copies
        const int cxlo = x0 == -1 ? -2 : x0, cxhi = x1 == n + 1 ? n + 3 : x1;
        const int cylo = y0 == -1 ? -2 : y0, cyhi = y1 == n + 1 ? n + 3 : y1;
        for (int pos = threadIdx.x; pos < ww * wh; pos += NT) {
            const int row = pos / ww, col = pos - row * ww;
            const int li = x0 - 1 + col, lj = y0 - 1 + row;
            if (li >= cxlo && li < cxhi && lj >= cylo && lj < cyhi) {
                T *o = A.out + (int64_t)patch * pw + (int64_t)(lj + kGhost) * W + (li + kGhost);
                const T *s = Sin + row * WN + col;
                for (int cp = 0; cp < ncp; ++cp) o[cp * A.plane] = s[cp * wsz];
            }
        }
    }
}

// Position of block entry k (see af_internal.h) relative to (i-1, j-1).
__host__ __device__ constexpr int blk_plane(int k) {
    return k < 4 ? kAvg : (k < 13 ? kCorner : (k < 19 ? kXmid : kYmid));
}
__host__ __device__ constexpr int blk_a(int k) {
    return k < 4 ? (k & 1) : (k < 13 ? (k - 4) % 3 : (k < 19 ? (k - 13) % 3 : (k - 19) % 2));
}
__host__ __device__ constexpr int blk_b(int k) {
    return k < 4 ? (k >> 1) : (k < 13 ? (k - 4) / 3 : (k < 19 ? (k - 13) / 3 : (k - 19) / 2));
}

// Orbit sums of a quad (++, +-, -+, --): symmetric, x-antisymmetric,
// y-antisymmetric parts.
template <typename T>
__device__ __forceinline__ void quad(T pp, T pm, T mp, T mm, T &ss, T &as, T &sa) {
    const T a = pp + pm, b = mp + mm;
    ss = a + b;
    as = a - b;
    sa = (pp - pm) + (mp - mm);
}

template <int N, typename T>
__device__ __forceinline__ T dot(const T *w, const T *v) {
    T s = w[0] * v[0];
#pragma unroll
    for (int k = 1; k < N; ++k) s = fma(w[k], v[k], s);
    return s;
}

// Acoustic node evaluation of one node-cell item (window coords qi, rj of
// node line (i, j)) with the mirror-folded weights: the 25 block values of
// each input component are combined into the orbit sums of the three nodes,
// then p += A.SS_p + Dx.AS_u + Dy.SA_v, u += A.SS_u + Dx.AS_p,
// v += A.SS_v + Dy.SA_p (the evolution operators of Eq. ERFormula).
// out: T and Q^{n+1} of corner (tc, nc), left-edge mid (tx, nx) and
// bottom-edge mid (ty, ny) for p, u, v.
template <typename T, int WN>
__device__ __forceinline__ void acoustic_item(const AcousticSymWeights<T> &W, const T *Sin, int qi, int rj,
                                              T tc[3], T nc[3], T tx[3], T nx[3], T ty[3], T ny[3]) {
    constexpr int WSZ = WN * WN;
#pragma unroll
    for (int o = 0; o < 3; ++o) tc[o] = nc[o] = tx[o] = nx[o] = ty[o] = ny[o] = T(0);
    const T *base = Sin + (rj - 1) * WN + (qi - 1);
#pragma unroll
    for (int ci = 0; ci < 3; ++ci) {
        T b[25];
#pragma unroll
        for (int k = 0; k < 25; ++k) b[k] = base[(ci * kPlanes + blk_plane(k)) * WSZ + blk_b(k) * WN + blk_a(k)];
        // ---- corner node
        T css[9], cas[6], csa[6];
        quad(b[3], b[1], b[2], b[0], css[0], cas[0], csa[0]);
        quad(b[12], b[6], b[10], b[4], css[1], cas[1], csa[1]);
        quad(b[18], b[15], b[16], b[13], css[2], cas[2], csa[2]);
        quad(b[24], b[20], b[23], b[19], css[3], cas[3], csa[3]);
        css[4] = b[9] + b[7];   cas[4] = b[9] - b[7];
        css[5] = b[22] + b[21]; cas[5] = b[22] - b[21];
        css[6] = b[11] + b[5];  csa[4] = b[11] - b[5];
        css[7] = b[17] + b[14]; csa[5] = b[17] - b[14];
        css[8] = b[8];
        // ---- left-edge midpoint
        T xss[6], xas[4], xsa[3];
        quad(b[12], b[9], b[10], b[7], xss[0], xas[0], xsa[0]);
        quad(b[24], b[22], b[23], b[21], xss[1], xas[1], xsa[1]);
        xss[2] = b[3] + b[2];   xas[2] = b[3] - b[2];
        xss[3] = b[18] + b[16]; xas[3] = b[18] - b[16];
        xss[4] = b[11] + b[8];  xsa[2] = b[11] - b[8];
        xss[5] = b[17];
        // ---- bottom-edge midpoint
        T yss[6], yas[3], ysa[4];
        quad(b[12], b[6], b[11], b[5], yss[0], yas[0], ysa[0]);
        quad(b[18], b[15], b[17], b[14], yss[1], yas[1], ysa[1]);
        yss[2] = b[9] + b[8];   yas[2] = b[9] - b[8];
        yss[3] = b[3] + b[1];   ysa[2] = b[3] - b[1];
        yss[4] = b[24] + b[20]; ysa[3] = b[24] - b[20];
        yss[5] = b[22];
        if (ci == 0) {  // p: A on p; Dx.AS_p -> u; Dy.SA_p -> v
            tc[0] += dot<9>(W.cA[0], css); nc[0] += dot<9>(W.cA[1], css);
            tx[0] += dot<6>(W.xA[0], xss); nx[0] += dot<6>(W.xA[1], xss);
            ty[0] += dot<6>(W.yA[0], yss); ny[0] += dot<6>(W.yA[1], yss);
            tc[1] += dot<6>(W.cDx[0], cas); nc[1] += dot<6>(W.cDx[1], cas);
            tx[1] += dot<4>(W.xDx[0], xas); nx[1] += dot<4>(W.xDx[1], xas);
            ty[1] += dot<3>(W.yDx[0], yas); ny[1] += dot<3>(W.yDx[1], yas);
            tc[2] += dot<6>(W.cDy[0], csa); nc[2] += dot<6>(W.cDy[1], csa);
            tx[2] += dot<3>(W.xDy[0], xsa); nx[2] += dot<3>(W.xDy[1], xsa);
            ty[2] += dot<4>(W.yDy[0], ysa); ny[2] += dot<4>(W.yDy[1], ysa);
        } else if (ci == 1) {  // u: A on u; Dx.AS_u -> p
            tc[1] += dot<9>(W.cA[0], css); nc[1] += dot<9>(W.cA[1], css);
            tx[1] += dot<6>(W.xA[0], xss); nx[1] += dot<6>(W.xA[1], xss);
            ty[1] += dot<6>(W.yA[0], yss); ny[1] += dot<6>(W.yA[1], yss);
            tc[0] += dot<6>(W.cDx[0], cas); nc[0] += dot<6>(W.cDx[1], cas);
            tx[0] += dot<4>(W.xDx[0], xas); nx[0] += dot<4>(W.xDx[1], xas);
            ty[0] += dot<3>(W.yDx[0], yas); ny[0] += dot<3>(W.yDx[1], yas);
        } else {  // v: A on v; Dy.SA_v -> p
            tc[2] += dot<9>(W.cA[0], css); nc[2] += dot<9>(W.cA[1], css);
            tx[2] += dot<6>(W.xA[0], xss); nx[2] += dot<6>(W.xA[1], xss);
            ty[2] += dot<6>(W.yA[0], yss); ny[2] += dot<6>(W.yA[1], yss);
            tc[0] += dot<6>(W.cDy[0], csa); nc[0] += dot<6>(W.cDy[1], csa);
            tx[0] += dot<3>(W.xDy[0], xsa); nx[0] += dot<3>(W.xDy[1], xsa);
            ty[0] += dot<4>(W.yDy[0], ysa); ny[0] += dot<4>(W.yDy[1], ysa);
        }
    }
}

// Advection: value of the reconstruction of window cell (cq, cr) with weights w.
template <typename T, int wn>
__device__ __forceinline__ T adv_eval(const T *w, const T *Sin, int cq, int cr) {
    constexpr int wsz = wn * wn;
    const int o = cr * wn + cq;
    const T *A = Sin + kAvg * wsz, *C = Sin + kCorner * wsz, *X = Sin + kXmid * wsz, *Y = Sin + kYmid * wsz;
    T v = w[0] * A[o];
    v = fma(w[1], C[o], v);
    v = fma(w[2], C[o + 1], v);
    v = fma(w[3], C[o + wn], v);
    v = fma(w[4], C[o + wn + 1], v);
    v = fma(w[5], X[o], v);
    v = fma(w[6], X[o + 1], v);
    v = fma(w[7], Y[o], v);
    v = fma(w[8], Y[o + wn], v);
    return v;
}

template <typename T, int EQ, int NT>
struct WeightsOf;
template <typename T, int NT>
struct WeightsOf<T, AF_ACOUSTICS, NT> { using type = AcousticSymWeights<T>; };
template <typename T, int NT>
struct WeightsOf<T, AF_ADVECTION, NT> { using type = AdvectionWeights<T>; };

template <typename T, int EQ, int NT, int TM>
__global__ void __launch_bounds__(NT) step_kernel(const __grid_constant__ StepArgs<T> A,
                                                  const __grid_constant__ typename WeightsOf<T, EQ, NT>::type W) {
    constexpr int WN = TM + 3, TP = TM + 1;  // window pitch, T-array pitch
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_nbr[8];
    T *Sin = reinterpret_cast<T *>(smem_raw);
    constexpr int ncomp = (EQ == AF_ACOUSTICS) ? 3 : 1;
    T *ST = Sin + ncomp * kPlanes * WN * WN;
    constexpr int tp = TP, tsz = TP * TP;

    const af_work &wk = A.work[blockIdx.x];
    const int patch = wk.patch, level = wk.level;
    const int x0 = wk.x0, x1 = wk.x1, y0 = wk.y0, y1 = wk.y1;
    if (threadIdx.x < 8) s_nbr[threadIdx.x] = wk.nbr[threadIdx.x];
    __syncthreads();
    const int tw = x1 - x0, th = y1 - y0;
    stage<T, NT, WN>(A, patch, s_nbr, x0, y0, x1, y1, tw + 3, th + 3, (wk.flags & 1) != 0, Sin);
    __syncthreads();

    const int n = A.n, W_ = n + 2 * kGhost + 1;
    const int64_t pw = (int64_t)ncomp * kPlanes * A.plane;
    T *outp = A.out + (int64_t)patch * pw;
    // node lines stored by this tile: [x0, x1) plus x1 itself when the tile
    // ends on the outer edge of the advanced first ghost layer
    const int sxhi = (x1 == n + 1) ? x1 : x1 - 1;
    const int syhi = (y1 == n + 1) ? y1 : y1 - 1;
    constexpr int wn = WN, wsz = WN * WN;

    // ---- point values (Eq. advection-update / Eq. ERFormula)
    const int nitems = (tw + 1) * (th + 1);
    for (int it = threadIdx.x; it < nitems; it += NT) {
        const int jj = it / (tw + 1), ii = it - jj * (tw + 1);
        const int i = x0 + ii, j = y0 + jj;
        const int qi = ii + 1, rj = jj + 1;
        const bool hx = j < y1, hy = i < x1;            // edge midpoints that exist
        const bool st_x = i <= sxhi, st_y = j <= syhi;  // stored lines
        const int64_t lo = (int64_t)(j + kGhost) * W_ + (i + kGhost);
        if constexpr (EQ == AF_ACOUSTICS) {
            T tc[3], nc[3], tx[3], nx[3], ty[3], ny[3];
            acoustic_item<T, WN>(W, Sin, qi, rj, tc, nc, tx, nx, ty, ny);
#pragma unroll
            for (int o = 0; o < 3; ++o) {
                ST[(o * 3 + 0) * tsz + jj * tp + ii] = tc[o];
                ST[(o * 3 + 1) * tsz + jj * tp + ii] = tx[o];
                ST[(o * 3 + 2) * tsz + jj * tp + ii] = ty[o];
                T *po = outp + (int64_t)o * kPlanes * A.plane + lo;
                if (st_x && st_y) po[kCorner * A.plane] = nc[o];
                if (st_x && hx) po[kXmid * A.plane] = nx[o];
                if (hy && st_y) po[kYmid * A.plane] = ny[o];
            }
        } else {
            const int own = rj * wn + qi;
            {
                const T qh = adv_eval<T, WN>(W.w[0][0], Sin, qi + W.off[0][0][0], rj + W.off[0][0][1]);
                const T q1 = adv_eval<T, WN>(W.w[0][1], Sin, qi + W.off[0][1][0], rj + W.off[0][1][1]);
                ST[0 * tsz + jj * tp + ii] = Sin[kCorner * wsz + own] + T(4) * qh + q1;
                if (st_x && st_y) outp[kCorner * A.plane + lo] = q1;
            }
            if (hx) {
                const T qh = adv_eval<T, WN>(W.w[1][0], Sin, qi + W.off[1][0][0], rj + W.off[1][0][1]);
                const T q1 = adv_eval<T, WN>(W.w[1][1], Sin, qi + W.off[1][1][0], rj + W.off[1][1][1]);
                ST[1 * tsz + jj * tp + ii] = Sin[kXmid * wsz + own] + T(4) * qh + q1;
                if (st_x) outp[kXmid * A.plane + lo] = q1;
            }
            if (hy) {
                const T qh = adv_eval<T, WN>(W.w[2][0], Sin, qi + W.off[2][0][0], rj + W.off[2][0][1]);
                const T q1 = adv_eval<T, WN>(W.w[2][1], Sin, qi + W.off[2][1][0], rj + W.off[2][1][1]);
                ST[2 * tsz + jj * tp + ii] = Sin[kYmid * wsz + own] + T(4) * qh + q1;
                if (st_y) outp[kYmid * A.plane + lo] = q1;
            }
        }
    }
    __syncthreads();

    // ---- fluxes (Eq. Simpson-2d) and update (Eq. 2dfv)
    const double dtl = ldexp(A.dt0, -level);
    for (int it = threadIdx.x; it < tw * th; it += NT) {
        const int jj = it / tw, ii = it - jj * tw;
        const int i = x0 + ii, j = y0 + jj;
        const int s00 = jj * tp + ii;
        T Fl[3], Fr[3], Gb[3], Gt[3];
#pragma unroll
        for (int c = 0; c < ncomp; ++c) {
            const T *Tc = ST + (c * 3 + 0) * tsz, *Tx = ST + (c * 3 + 1) * tsz, *Ty = ST + (c * 3 + 2) * tsz;
            // time-Simpson sums at the three points of each face
            Fl[c] = Tc[s00] + T(4) * Tx[s00] + Tc[s00 + tp];
            Fr[c] = Tc[s00 + 1] + T(4) * Tx[s00 + 1] + Tc[s00 + tp + 1];
            Gb[c] = Tc[s00] + T(4) * Ty[s00] + Tc[s00 + 1];
            Gt[c] = Tc[s00 + tp] + T(4) * Ty[s00 + tp] + Tc[s00 + tp + 1];
        }
        T fl[3], fr[3], gb[3], gt[3];
        if constexpr (EQ == AF_ACOUSTICS) {
            // f = c (u, p, 0), g = c (v, 0, p)
            fl[0] = A.fx * Fl[1]; fl[1] = A.fx * Fl[0]; fl[2] = T(0);
            fr[0] = A.fx * Fr[1]; fr[1] = A.fx * Fr[0]; fr[2] = T(0);
            gb[0] = A.fy * Gb[2]; gb[1] = T(0); gb[2] = A.fy * Gb[0];
            gt[0] = A.fy * Gt[2]; gt[1] = T(0); gt[2] = A.fy * Gt[0];
        } else {
            fl[0] = A.fx * Fl[0]; fr[0] = A.fx * Fr[0];
            gb[0] = A.fy * Gb[0]; gt[0] = A.fy * Gt[0];
        }
        const int64_t lo = (int64_t)(j + kGhost) * W_ + (i + kGhost);
        const int sa = (jj + 1) * wn + (ii + 1);
#pragma unroll
        for (int c = 0; c < ncomp; ++c) {
            const T q = Sin[(c * kPlanes + kAvg) * wsz + sa];
            outp[(int64_t)(c * kPlanes + kAvg) * A.plane + lo] = q - A.dtdx * (fr[c] - fl[c]) - A.dtdy * (gt[c] - gb[c]);
        }
        if (A.freg != nullptr) {
            double *fr_p = A.freg + (int64_t)patch * 4 * ncomp * n;
            const bool iny = (j >= 0 && j < n), inx = (i >= 0 && i < n);
#pragma unroll
            for (int c = 0; c < ncomp; ++c) {
                if (iny && i == 0) fr_p[(0 * ncomp + c) * n + j] += dtl * (double)fl[c];
                if (iny && i == n - 1) fr_p[(1 * ncomp + c) * n + j] += dtl * (double)fr[c];
                if (inx && j == 0) fr_p[(2 * ncomp + c) * n + i] += dtl * (double)gb[c];
                if (inx && j == n - 1) fr_p[(3 * ncomp + c) * n + i] += dtl * (double)gt[c];
            }
        }
    }
}

constexpr int kThreads = 256;

// ------------------------------------------------------------ weight cache
struct WeightKey {
    int eq;
    double r0, r1;
    bool operator==(const WeightKey &o) const { return eq == o.eq && r0 == o.r0 && r1 == o.r1; }
};
std::mutex g_wmu;
WeightKey g_akey{-1, 0, 0}, g_dkey{-1, 0, 0};
AcousticWeights<double> g_aw;
AdvectionWeights<double> g_dw;

std::mutex g_smu;
WeightKey g_skey{-1, 0, 0};
AcousticSymWeights<double> g_sw;
bool g_sw_ok = false;

template <typename T>
bool get_acoustic(double rx, double ry, AcousticSymWeights<T> &out) {
    std::lock_guard<std::mutex> lk(g_smu);
    WeightKey k{AF_ACOUSTICS, rx, ry};
    if (!(k == g_skey)) {
        g_sw_ok = acoustic_sym_weights(rx, ry, g_sw);
        g_skey = k;
    }
    const double *src = &g_sw.cA[0][0];
    T *dst = &out.cA[0][0];
    constexpr int nw = sizeof(AcousticSymWeights<double>) / sizeof(double);
    static_assert(sizeof(AcousticSymWeights<T>) == nw * sizeof(T), "packed weight struct");
    for (int i = 0; i < nw; ++i) dst[i] = (T)src[i];
    return g_sw_ok;
}

template <typename T>
void get_advection(double nx, double ny, AdvectionWeights<T> &out) {
    std::lock_guard<std::mutex> lk(g_wmu);
    WeightKey k{AF_ADVECTION, nx, ny};
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

template <typename Kern>
cudaError_t ensure_smem(Kern k, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Tile geometry compiled into the kernel: 10, 18 or 32 cells per side.
inline int tile_template_for(int n) {
    const int t = tile_max_for(n);
    return t <= 10 ? 10 : (t <= 18 ? 18 : 32);
}

template <typename T, int EQ, int TM>
af_status launch_tm(const StepArgs<T> &A, const typename WeightsOf<T, EQ, kThreads>::type &W, int ncomp, int nwork,
                    cudaStream_t stream) {
    constexpr int WN = TM + 3, TP = TM + 1;
    const size_t smem = sizeof(T) * ((size_t)ncomp * kPlanes * WN * WN + (size_t)ncomp * 3 * TP * TP);
    auto kern = step_kernel<T, EQ, kThreads, TM>;
    if (ensure_smem(kern, smem) != cudaSuccess) return AF_ERR_CUDA;
    kern<<<nwork, kThreads, smem, stream>>>(A, W);
    return cudaGetLastError() == cudaSuccess ? AF_OK : AF_ERR_CUDA;
}

template <typename T, int EQ>
af_status launch(const af_config &cfg, int nwork, const af_work *d_work, const void *d_in, void *d_out,
                 double dt0, double dx0, double dy0, double *d_freg, cudaStream_t stream) {
    StepArgs<T> A;
    A.work = d_work;
    A.in = static_cast<const T *>(d_in);
    A.out = static_cast<T *>(d_out);
    A.freg = d_freg;
    A.plane = plane_stride(cfg.n);
    A.n = cfg.n;
    A.ncomp = cfg.ncomp;
    const int tm = tile_template_for(cfg.n);
    A.wn = tm + 3;
    A.tp = tm + 1;
    A.dtdx = (T)(dt0 / dx0);
    A.dtdy = (T)(dt0 / dy0);
    A.dt0 = dt0;
    typename WeightsOf<T, EQ, kThreads>::type W;
    if constexpr (EQ == AF_ACOUSTICS) {
        A.fx = A.fy = (T)(cfg.c / 36.0);
        if (!get_acoustic<T>(cfg.c * dt0 / dx0, cfg.c * dt0 / dy0, W)) return AF_ERR_UNIMPLEMENTED;
    } else {
        A.fx = (T)(cfg.a / 36.0);
        A.fy = (T)(cfg.b / 36.0);
        get_advection<T>(cfg.a * dt0 / dx0, cfg.b * dt0 / dy0, W);
    }
    if (tm == 10) return launch_tm<T, EQ, 10>(A, W, cfg.ncomp, nwork, stream);
    if (tm == 18) return launch_tm<T, EQ, 18>(A, W, cfg.ncomp, nwork, stream);
    return launch_tm<T, EQ, 32>(A, W, cfg.ncomp, nwork, stream);
}

}  // namespace
}  // namespace af

extern "C" af_status af_patch_step(const af_config *cfg, int32_t nwork, const af_work *d_work, const void *d_in,
                                   void *d_out, double dt0, double dx0, double dy0, double *d_flux_reg,
                                   void *stream) {
    using namespace af;
    if (cfg == nullptr || nwork < 0) return AF_ERR_ARG;
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
    if (cfg->prec == AF_F64)
        return cfg->eq == AF_ACOUSTICS
                   ? launch<double, AF_ACOUSTICS>(*cfg, nwork, d_work, d_in, d_out, dt0, dx0, dy0, d_flux_reg, s)
                   : launch<double, AF_ADVECTION>(*cfg, nwork, d_work, d_in, d_out, dt0, dx0, dy0, d_flux_reg, s);
    return cfg->eq == AF_ACOUSTICS
               ? launch<float, AF_ACOUSTICS>(*cfg, nwork, d_work, d_in, d_out, dt0, dx0, dy0, d_flux_reg, s)
               : launch<float, AF_ADVECTION>(*cfg, nwork, d_work, d_in, d_out, dt0, dx0, dy0, d_flux_reg, s);
}

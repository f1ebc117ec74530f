// Learned refinement tagger of libaf.so: a 3-layer convolutional network
// that predicts, from a patch's cell averages with a two-cell halo, the tag
// the plain per-patch criterion (Section 3; the undivided-difference
// indicator of Sections 4.4 and 4.5.2) gives one coarse step later.  The
// paper has no such network; the definitions are with the declarations
// of the af_cnn_* entry points.
//
// Storage is BF16 (inputs, conv weights, layer-1 activations), arithmetic is
// FP32 with FP32 accumulation.  One CTA runs one patch through both
// convolutions in shared memory (the layer-1 map never leaves the SM); the
// backward pass uses that the global max-pool passes gradient to one pixel
// per channel, so it costs a small fraction of the forward pass, and it
// accumulates per-CTA partial gradients that a second kernel sums in a
// fixed order (deterministic).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>

#include "af_internal.h"

namespace af {
namespace {

constexpr int kF = 32;       // feature channels
constexpr int kLevels = 16;  // rows of the level embedding
constexpr int kW2Pitch = kF * 9 + 1;  // padded row of W2 in shared memory (bank spread)

__host__ __device__ constexpr int cnn_params(int C) { return kF * C * 9 + kLevels * kF + kF * kF * 9 + kF + kF + 1; }
// offsets of the parameter blocks in the flat vector
__host__ __device__ constexpr int off_w1() { return 0; }
__host__ __device__ constexpr int off_emb(int C) { return kF * C * 9; }
__host__ __device__ constexpr int off_w2(int C) { return off_emb(C) + kLevels * kF; }
__host__ __device__ constexpr int off_b2(int C) { return off_w2(C) + kF * kF * 9; }
__host__ __device__ constexpr int off_w3(int C) { return off_b2(C) + kF; }
__host__ __device__ constexpr int off_b3(int C) { return off_w3(C) + kF; }

__device__ __forceinline__ float rbf(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

// Shared-memory layout of one CTA (floats).
template <int C, int N>
struct Smem {
    static constexpr int S = N + 4, S1 = N + 2;
    static constexpr int w1 = 0;
    static constexpr int w2 = w1 + kF * C * 9;
    static constexpr int emb = w2 + kF * kW2Pitch;
    static constexpr int b2 = emb + kLevels * kF;
    static constexpr int w3 = b2 + kF;
    static constexpr int b3 = w3 + kF;
    static constexpr int m = b3 + 4;  // per-channel maxima of the current sample
    static constexpr int x = m + kF;
    static constexpr int a1 = x + C * S * S;
    static constexpr int fwd_end = a1 + kF * S1 * S1;
    static constexpr int da1 = fwd_end;
    static constexpr int gw1 = da1 + kF * S1 * S1;
    static constexpr int gemb = gw1 + kF * C * 9;
    static constexpr int gw2 = gemb + kLevels * kF;
    static constexpr int gb2 = gw2 + kF * kF * 9;
    static constexpr int gw3 = gb2 + kF;
    static constexpr int gb3 = gw3 + kF;
    static constexpr int bwd_end = gb3 + 4;
};

// Weights into shared memory (conv weights rounded to BF16).
template <int C, int N>
__device__ void load_weights(const float *__restrict__ P, float *sm) {
    using L = Smem<C, N>;
    for (int e = threadIdx.x; e < kF * C * 9; e += blockDim.x) sm[L::w1 + e] = rbf(P[off_w1() + e]);
    for (int e = threadIdx.x; e < kF * kF * 9; e += blockDim.x) {
        const int g = e / (kF * 9), r = e - g * kF * 9;
        sm[L::w2 + g * kW2Pitch + r] = rbf(P[off_w2(C) + e]);
    }
    for (int e = threadIdx.x; e < kLevels * kF; e += blockDim.x) sm[L::emb + e] = P[off_emb(C) + e];
    for (int e = threadIdx.x; e < kF; e += blockDim.x) {
        sm[L::b2 + e] = P[off_b2(C) + e];
        sm[L::w3 + e] = P[off_w3(C) + e];
    }
    if (threadIdx.x == 0) sm[L::b3] = P[off_b3(C)];
}

// Input of sample b and the layer-1 map A1 = bf16(relu(conv(X, W1) + emb)).
template <int C, int N>
__device__ void layer1(const __nv_bfloat16 *__restrict__ X, int b, int level, float *sm) {
    using L = Smem<C, N>;
    constexpr int S = L::S, S1 = L::S1;
    const __nv_bfloat16 *xb = X + (int64_t)b * C * S * S;
    for (int e = threadIdx.x; e < C * S * S; e += blockDim.x) sm[L::x + e] = __bfloat162float(xb[e]);
    __syncthreads();
    const float *emb = sm + L::emb + level * kF;
    for (int e = threadIdx.x; e < kF * S1 * S1; e += blockDim.x) {
        const int f = e / (S1 * S1), r = e - f * S1 * S1, y = r / S1, x = r - y * S1;
        float z = 0.f;
#pragma unroll
        for (int c = 0; c < C; ++c)
#pragma unroll
            for (int ky = 0; ky < 3; ++ky)
#pragma unroll
                for (int kx = 0; kx < 3; ++kx)
                    z = fmaf(sm[L::w1 + ((f * C + c) * 3 + ky) * 3 + kx], sm[L::x + (c * S + y + ky) * S + x + kx], z);
        z += emb[f];
        sm[L::a1 + e] = rbf(fmaxf(z, 0.f));
    }
    __syncthreads();
}

// Layer 2 and the global max-pool: thread (cg, row) computes channels
// 2cg, 2cg+1 of output row `row`; returns per channel the maximum of
// Z2 = conv(A1, W2) + b2 and its first row-major position.
template <int C, int N>
__device__ void layer2_max(const float *sm, float *mval, int *marg) {
    using L = Smem<C, N>;
    constexpr int S1 = L::S1;
    const int cg = threadIdx.x / N, row = threadIdx.x - cg * N;
    const bool active = cg < kF / 2;
    float acc[2][N];
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int x = 0; x < N; ++x) acc[h][x] = 0.f;
    if (active) {
        const float *w0 = sm + L::w2 + (2 * cg) * kW2Pitch, *w1 = w0 + kW2Pitch;
        for (int f = 0; f < kF; ++f) {
#pragma unroll
            for (int ky = 0; ky < 3; ++ky) {
                float a[N + 2];
                const float *src = sm + L::a1 + (f * S1 + row + ky) * S1;
#pragma unroll
                for (int x = 0; x < N + 2; ++x) a[x] = src[x];
#pragma unroll
                for (int kx = 0; kx < 3; ++kx) {
                    const float u = w0[f * 9 + ky * 3 + kx], v = w1[f * 9 + ky * 3 + kx];
#pragma unroll
                    for (int x = 0; x < N; ++x) {
                        acc[0][x] = fmaf(u, a[x + kx], acc[0][x]);
                        acc[1][x] = fmaf(v, a[x + kx], acc[1][x]);
                    }
                }
            }
        }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const float bias = active ? sm[L::b2 + 2 * cg + h] : 0.f;
        float best = -INFINITY;
        int bi = 0x7fffffff;
#pragma unroll
        for (int x = 0; x < N; ++x) {
            const float z = acc[h][x] + bias;
            if (z > best) {
                best = z;
                bi = row * N + x;
            }
        }
        // reduce over the N rows held by consecutive lanes
#pragma unroll
        for (int o = N / 2; o > 0; o >>= 1) {
            const float ob = __shfl_xor_sync(0xffffffffu, best, o, N);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o, N);
            if (ob > best || (ob == best && oi < bi)) {
                best = ob;
                bi = oi;
            }
        }
        if (active && row == 0) {
            mval[2 * cg + h] = best > 0.f ? best : 0.f;
            marg[2 * cg + h] = best > 0.f ? bi : -1;
        }
    }
}

template <int C, int N>
__global__ void __launch_bounds__(256) cnn_forward_kernel(int nsample, const __nv_bfloat16 *__restrict__ X,
                                                          const int32_t *__restrict__ level,
                                                          const float *__restrict__ P, float *__restrict__ logit,
                                                          float *__restrict__ Mout, int32_t *__restrict__ Aout) {
    using L = Smem<C, N>;
    extern __shared__ __align__(16) float sm[];
    __shared__ int s_arg[kF];
    load_weights<C, N>(P, sm);
    __syncthreads();
    for (int b = blockIdx.x; b < nsample; b += gridDim.x) {
        const int lv = min(max(level[b], 0), kLevels - 1);
        layer1<C, N>(X, b, lv, sm);
        layer2_max<C, N>(sm, sm + L::m, s_arg);
        __syncthreads();
        if (threadIdx.x < 32) {
            const int g = threadIdx.x;
            float v = sm[L::w3 + g] * sm[L::m + g];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            Mout[(int64_t)b * kF + g] = sm[L::m + g];
            Aout[(int64_t)b * kF + g] = s_arg[g];
            if (g == 0) logit[b] = v + sm[L::b3];
        }
        __syncthreads();
    }
}

template <int C, int N>
__global__ void __launch_bounds__(256) cnn_backward_kernel(int nsample, const __nv_bfloat16 *__restrict__ X,
                                                           const int32_t *__restrict__ level,
                                                           const float *__restrict__ P,
                                                           const float *__restrict__ logit,
                                                           const float *__restrict__ Min,
                                                           const int32_t *__restrict__ Ain,
                                                           const float *__restrict__ label,
                                                           const float *__restrict__ omega, float inv_omega_sum,
                                                           float *__restrict__ partial) {
    using L = Smem<C, N>;
    constexpr int S = L::S, S1 = L::S1;
    constexpr int NP = cnn_params(C);
    extern __shared__ __align__(16) float sm[];
    __shared__ float s_dz[kF];
    __shared__ int s_arg[kF];
    __shared__ float s_dlogit;
    load_weights<C, N>(P, sm);
    for (int e = threadIdx.x; e < L::bwd_end - L::gw1; e += blockDim.x) sm[L::gw1 + e] = 0.f;
    __syncthreads();
    for (int b = blockIdx.x; b < nsample; b += gridDim.x) {
        const int lv = min(max(level[b], 0), kLevels - 1);
        layer1<C, N>(X, b, lv, sm);
        if (threadIdx.x == 0) {
            const float l = logit[b];
            s_dlogit = omega[b] * (1.f / (1.f + expf(-l)) - label[b]) * inv_omega_sum;
        }
        __syncthreads();
        const float dl = s_dlogit;
        if (threadIdx.x < kF) {
            const int g = threadIdx.x;
            const float mg = Min[(int64_t)b * kF + g];
            const int ag = Ain[(int64_t)b * kF + g];
            sm[L::gw3 + g] += dl * mg;
            const float dz = ag >= 0 ? dl * sm[L::w3 + g] : 0.f;
            s_dz[g] = dz;
            s_arg[g] = ag;
            sm[L::gb2 + g] += dz;
            if (g == 0) sm[L::gb3] += dl;
        }
        __syncthreads();
        // dW2[g, f, ky, kx] += dz_g A1[f, y_g + ky, x_g + kx]
        for (int e = threadIdx.x; e < kF * kF * 9; e += blockDim.x) {
            const int g = e / (kF * 9), r = e - g * kF * 9, f = r / 9, k = r - f * 9;
            const int ag = s_arg[g];
            if (ag < 0) continue;
            const int yg = ag / N, xg = ag - yg * N;
            sm[L::gw2 + e] += s_dz[g] * sm[L::a1 + (f * S1 + yg + k / 3) * S1 + xg + k % 3];
        }
        // dA1 gathered per position (no write conflicts), masked by relu
        for (int e = threadIdx.x; e < kF * S1 * S1; e += blockDim.x) {
            const int f = e / (S1 * S1), r = e - f * S1 * S1, y = r / S1, x = r - y * S1;
            float d = 0.f;
            for (int g = 0; g < kF; ++g) {
                const int ag = s_arg[g];
                if (ag < 0) continue;
                const int ky = y - ag / N, kx = x - ag % N;
                if (ky < 0 || ky > 2 || kx < 0 || kx > 2) continue;
                d = fmaf(s_dz[g], sm[L::w2 + g * kW2Pitch + f * 9 + ky * 3 + kx], d);
            }
            sm[L::da1 + e] = sm[L::a1 + e] > 0.f ? d : 0.f;
        }
        __syncthreads();
        // level embedding and W1
        if (threadIdx.x < kF) {
            const int f = threadIdx.x;
            float s = 0.f;
            for (int r = 0; r < S1 * S1; ++r) s += sm[L::da1 + f * S1 * S1 + r];
            sm[L::gemb + lv * kF + f] += s;
        }
        for (int e = threadIdx.x; e < kF * C * 9; e += blockDim.x) {
            const int f = e / (C * 9), r = e - f * C * 9, c = r / 9, k = r - c * 9, ky = k / 3, kx = k % 3;
            float s = 0.f;
            for (int y = 0; y < S1; ++y)
                for (int x = 0; x < S1; ++x)
                    s = fmaf(sm[L::da1 + (f * S1 + y) * S1 + x], sm[L::x + (c * S + y + ky) * S + x + kx], s);
            sm[L::gw1 + e] += s;
        }
        __syncthreads();
    }
    // partial gradient of this CTA, in parameter order
    float *out = partial + (int64_t)blockIdx.x * NP;
    for (int e = threadIdx.x; e < NP; e += blockDim.x) {
        float v;
        if (e < off_emb(C)) v = sm[L::gw1 + e];
        else if (e < off_w2(C)) v = sm[L::gemb + e - off_emb(C)];
        else if (e < off_b2(C)) v = sm[L::gw2 + e - off_w2(C)];
        else if (e < off_w3(C)) v = sm[L::gb2 + e - off_b2(C)];
        else if (e < off_b3(C)) v = sm[L::gw3 + e - off_w3(C)];
        else v = sm[L::gb3];
        out[e] = v;
    }
}

__global__ void sum_partials(const float *__restrict__ partial, int nblocks, int np, float *__restrict__ grad) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= np) return;
    float s = 0.f;
    for (int k = 0; k < nblocks; ++k) s += partial[(int64_t)k * np + e];
    grad[e] = s;
}

__global__ void adam_kernel(int64_t n, float *__restrict__ p, float *__restrict__ m, float *__restrict__ v,
                            const float *__restrict__ g, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
}

// Inputs: cell averages of leaf p with two ghost layers, minus the interior
// mean, times 1 / (2 h_l thr), rounded to BF16.  Cells outside the patch come
// from the same-level neighbour in that direction, or from the leaf's own
// (exchanged) ghost ring where there is none.
template <typename T, int C>
__global__ void cnn_inputs_kernel(int n, int64_t plane, const int32_t *__restrict__ lev, T *b0, T *b1,
                                  uint32_t parity, const int32_t *__restrict__ nbr, double dx0, double thr,
                                  __nv_bfloat16 *__restrict__ X) {
    const int p = blockIdx.x, S = n + 4, W = n + 2 * kGhost + 1;
    const int lp = lev[p];
    const int64_t pw = (int64_t)C * kPlanes * plane;
    T *base = ((parity >> lp) & 1u) ? b1 : b0;
    __shared__ double red[256];
    __shared__ double s_mu;
    int nb[8];
#pragma unroll
    for (int d = 0; d < 8; ++d) nb[d] = nbr[8 * (int64_t)p + d];
    const double scale = 1.0 / (2.0 * (dx0 / (double)(1LL << lp)) * thr);
    for (int c = 0; c < C; ++c) {
        double s = 0.0;
        for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
            const int j = e / n, i = e - j * n;
            s += (double)base[(int64_t)p * pw + (c * kPlanes + kAvg) * plane + (j + kGhost) * W + (i + kGhost)];
        }
        red[threadIdx.x] = s;
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) s_mu = red[0] / (double)(n * n);
        __syncthreads();
        const double mu = s_mu;
        for (int e = threadIdx.x; e < S * S; e += blockDim.x) {
            const int y = e / S, x = e - y * S, i = x - 2, j = y - 2;
            const int sx = i < 0 ? -1 : (i >= n ? 1 : 0), sy = j < 0 ? -1 : (j >= n ? 1 : 0);
            int src = p, si = i, sj = j;
            if (sx | sy) {
                const int d = sy == 0 ? (sx < 0 ? 0 : 1) : (sx == 0 ? (sy < 0 ? 2 : 3) : 4 + (sx > 0) + 2 * (sy > 0));
                if (nb[d] >= 0) {
                    src = nb[d];
                    si = i - sx * n;
                    sj = j - sy * n;
                }
            }
            const double q = (double)base[(int64_t)src * pw + (c * kPlanes + kAvg) * plane + (sj + kGhost) * W +
                                          (si + kGhost)];
            X[((int64_t)p * C + c) * S * S + e] = __float2bfloat16_rn((float)((q - mu) * scale));
        }
        __syncthreads();
    }
}

__global__ void combine_kernel(int n, const float *__restrict__ logit, const int8_t *__restrict__ plain, float cmin,
                               int8_t *__restrict__ tags, int32_t *__restrict__ nfall) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float pr = 1.f / (1.f + expf(-logit[i]));
    const float conf = fabsf(2.f * pr - 1.f);
    const int8_t pl = plain[i];
    int8_t t;
    if (conf < cmin) {
        t = pl;
        atomicAdd(nfall, 1);
    } else {
        t = pr >= 0.5f ? 1 : (pl == -1 ? -1 : 0);
    }
    tags[i] = t;
}

template <typename K>
af_status smem_attr(K k, size_t bytes) {
    if (bytes > 227 * 1024) return AF_ERR_UNIMPLEMENTED;
    if (bytes > 48 * 1024 && cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess)
        return AF_ERR_CUDA;
    return AF_OK;
}

inline af_status launched() { return cudaGetLastError() == cudaSuccess ? AF_OK : AF_ERR_CUDA; }

template <int C, int N>
af_status forward_launch(int nsample, const void *X, const int32_t *lev, const float *P, float *lg, float *M,
                         int32_t *A, cudaStream_t s) {
    auto k = cnn_forward_kernel<C, N>;
    const size_t bytes = sizeof(float) * Smem<C, N>::fwd_end;
    if (const af_status e = smem_attr(k, bytes)) return e;
    const int grid = nsample < 152 * 4 ? nsample : 152 * 4;
    k<<<grid, 256, bytes, s>>>(nsample, static_cast<const __nv_bfloat16 *>(X), lev, P, lg, M, A);
    return launched();
}

template <int C, int N>
af_status backward_launch(int nsample, const void *X, const int32_t *lev, const float *P, const float *lg,
                          const float *M, const int32_t *A, const float *y, const float *om, float inv_om,
                          float *partial, int nblocks, float *grad, cudaStream_t s) {
    auto k = cnn_backward_kernel<C, N>;
    const size_t bytes = sizeof(float) * Smem<C, N>::bwd_end;
    if (const af_status e = smem_attr(k, bytes)) return e;
    k<<<nblocks, 256, bytes, s>>>(nsample, static_cast<const __nv_bfloat16 *>(X), lev, P, lg, M, A, y, om, inv_om,
                                  partial);
    if (launched() != AF_OK) return AF_ERR_CUDA;
    const int np = cnn_params(C);
    sum_partials<<<(np + 255) / 256, 256, 0, s>>>(partial, nblocks, np, grad);
    return launched();
}

bool cnn_shape_ok(int ncomp, int n) { return (ncomp == 1 || ncomp == 3) && (n == 8 || n == 16); }

}  // namespace
}  // namespace af

using namespace af;

extern "C" int64_t af_cnn_param_count(int32_t ncomp) {
    return (ncomp == 1 || ncomp == 3) ? cnn_params(ncomp) : 0;
}

extern "C" af_status af_cnn_inputs(const af_config *cfg, const af_forest *forest, const af_state_pair *state,
                                   const int32_t *d_nbr, double dx0, double thr, uint16_t *d_x, void *stream) {
    if (!cfg || !forest || !state || !cnn_shape_ok(cfg->ncomp, cfg->n)) return AF_ERR_ARG;
    if (cfg->prec != AF_F32 && cfg->prec != AF_F64) return AF_ERR_ARG;
    if (!(dx0 > 0.0) || !(thr > 0.0)) return AF_ERR_ARG;
    if (forest->nleaf == 0) return AF_OK;
    if (!d_nbr || !d_x || !forest->d_level || !state->buf[0] || (state->parity && !state->buf[1])) return AF_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t plane = plane_stride(cfg->n);
    __nv_bfloat16 *X = reinterpret_cast<__nv_bfloat16 *>(d_x);
    const int nl = forest->nleaf;
    if (cfg->prec == AF_F64) {
        double *b0 = static_cast<double *>(state->buf[0]), *b1 = static_cast<double *>(state->buf[1]);
        if (cfg->ncomp == 3)
            cnn_inputs_kernel<double, 3><<<nl, 256, 0, s>>>(cfg->n, plane, forest->d_level, b0, b1, state->parity,
                                                            d_nbr, dx0, thr, X);
        else
            cnn_inputs_kernel<double, 1><<<nl, 256, 0, s>>>(cfg->n, plane, forest->d_level, b0, b1, state->parity,
                                                            d_nbr, dx0, thr, X);
    } else {
        float *b0 = static_cast<float *>(state->buf[0]), *b1 = static_cast<float *>(state->buf[1]);
        if (cfg->ncomp == 3)
            cnn_inputs_kernel<float, 3><<<nl, 256, 0, s>>>(cfg->n, plane, forest->d_level, b0, b1, state->parity,
                                                           d_nbr, dx0, thr, X);
        else
            cnn_inputs_kernel<float, 1><<<nl, 256, 0, s>>>(cfg->n, plane, forest->d_level, b0, b1, state->parity,
                                                           d_nbr, dx0, thr, X);
    }
    return launched();
}

extern "C" af_status af_cnn_forward(int32_t ncomp, int32_t n, int32_t nsample, const uint16_t *d_x,
                                    const int32_t *d_level, const float *d_params, float *d_logit, float *d_m,
                                    int32_t *d_arg, void *stream) {
    if (!cnn_shape_ok(ncomp, n) || nsample < 0) return AF_ERR_ARG;
    if (nsample == 0) return AF_OK;
    if (!d_x || !d_level || !d_params || !d_logit || !d_m || !d_arg) return AF_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (ncomp == 3)
        return n == 16 ? forward_launch<3, 16>(nsample, d_x, d_level, d_params, d_logit, d_m, d_arg, s)
                       : forward_launch<3, 8>(nsample, d_x, d_level, d_params, d_logit, d_m, d_arg, s);
    return n == 16 ? forward_launch<1, 16>(nsample, d_x, d_level, d_params, d_logit, d_m, d_arg, s)
                   : forward_launch<1, 8>(nsample, d_x, d_level, d_params, d_logit, d_m, d_arg, s);
}

extern "C" int64_t af_cnn_partial_floats(int32_t ncomp, int32_t nblocks) {
    return (ncomp == 1 || ncomp == 3) && nblocks > 0 ? (int64_t)nblocks * cnn_params(ncomp) : 0;
}

extern "C" af_status af_cnn_backward(int32_t ncomp, int32_t n, int32_t nsample, const uint16_t *d_x,
                                     const int32_t *d_level, const float *d_params, const float *d_logit,
                                     const float *d_m, const int32_t *d_arg, const float *d_label,
                                     const float *d_weight, double weight_sum, float *d_partial, int32_t nblocks,
                                     float *d_grad, void *stream) {
    if (!cnn_shape_ok(ncomp, n) || nsample < 0 || nblocks < 1 || !(weight_sum > 0.0)) return AF_ERR_ARG;
    if (!d_partial || !d_grad || !d_params) return AF_ERR_ARG;
    if (nsample > 0 && (!d_x || !d_level || !d_logit || !d_m || !d_arg || !d_label || !d_weight)) return AF_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const float inv = (float)(1.0 / weight_sum);
    if (ncomp == 3)
        return n == 16 ? backward_launch<3, 16>(nsample, d_x, d_level, d_params, d_logit, d_m, d_arg, d_label,
                                                d_weight, inv, d_partial, nblocks, d_grad, s)
                       : backward_launch<3, 8>(nsample, d_x, d_level, d_params, d_logit, d_m, d_arg, d_label,
                                               d_weight, inv, d_partial, nblocks, d_grad, s);
    return n == 16 ? backward_launch<1, 16>(nsample, d_x, d_level, d_params, d_logit, d_m, d_arg, d_label, d_weight,
                                            inv, d_partial, nblocks, d_grad, s)
                   : backward_launch<1, 8>(nsample, d_x, d_level, d_params, d_logit, d_m, d_arg, d_label, d_weight,
                                           inv, d_partial, nblocks, d_grad, s);
}

extern "C" af_status af_cnn_adam(int64_t nparam, float *d_params, float *d_m, float *d_v, const float *d_grad,
                                 int32_t step, double lr, double beta1, double beta2, double eps, void *stream) {
    if (nparam < 0 || step < 1 || !(lr > 0.0) || !(beta1 >= 0.0 && beta1 < 1.0) || !(beta2 >= 0.0 && beta2 < 1.0))
        return AF_ERR_ARG;
    if (nparam == 0) return AF_OK;
    if (!d_params || !d_m || !d_v || !d_grad) return AF_ERR_ARG;
    const double c1 = 1.0 / (1.0 - std::pow(beta1, step)), c2 = 1.0 / (1.0 - std::pow(beta2, step));
    adam_kernel<<<(unsigned)((nparam + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        nparam, d_params, d_m, d_v, d_grad, (float)lr, (float)beta1, (float)beta2, (float)eps, (float)c1, (float)c2);
    return launched();
}

extern "C" af_status af_cnn_tags(int32_t nleaf, const float *d_logit, const int8_t *d_plain, double cmin,
                                 int8_t *d_tags, int32_t *d_nfallback, void *stream) {
    if (nleaf < 0) return AF_ERR_ARG;
    if (nleaf == 0) return AF_OK;
    if (!d_logit || !d_plain || !d_tags || !d_nfallback) return AF_ERR_ARG;
    combine_kernel<<<(nleaf + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(nleaf, d_logit, d_plain,
                                                                                        (float)cmin, d_tags,
                                                                                        d_nfallback);
    return launched();
}

// Learned refinement tagger of libaf.so: a 3-layer convolutional network
// that predicts, from a patch's cell averages with a two-cell halo, the tag
// the plain per-patch criterion (Section 3; the undivided-difference
// indicator of Sections 4.4 and 4.5.2) gives one coarse step later.  The
// paper has no such network; the definitions are with the declarations
// of the af_cnn_* entry points.
//
// Storage is BF16 (inputs, conv weights, layer-1 activations), arithmetic is
// FP32 with FP32 accumulation.  Both convolutions run on the tensor cores
// (tcgen05.mma, BF16 operands in shared memory, FP32 accumulators in tensor
// memory) as implicit GEMMs, one patch at a time per CTA:
//   layer 1: D1[q][g] = sum_ky sum_{c,kx} Xh[q + ky (n+4)][(c, kx)] W1[g][c][ky][kx]
//            as three accumulating GEMMs with K = 16, where Xh holds, for
//            every flat pixel r of the input patch (row pitch n + 4), its
//            horizontal taps X[c][r + kx] (3 C values, zero-padded): a
//            third of an im2col's work.  Output position q = y (n+4) + x is
//            layer-1 pixel (y, x) for x < n + 2; the others are computed and
//            ignored.  M = (n+2)(n+4) positions in tiles of 128, N = 32;
//   layer 2: D2[q][g] = sum_{ky,kx} sum_f A1[f][q + ky (n+2) + kx] W2[g][f][ky][kx]
//            as nine accumulating GEMMs with K = 32 channels.  The layer-1
//            map is stored once, pixel-major with its own row pitch n + 2,
//            so for every shift (ky, kx) the A operand of a 128-row tile is
//            the same uniformly strided block started (ky (n+2) + kx) rows
//            later; output position q = y (n+2) + x is pixel (y, x) for
//            x < n, and the two positions per row with x >= n (which read
//            across a row end) are computed and ignored.  M = n (n+2)
//            positions in tiles of 128, N = 32.
// The epilogues read the accumulators back (tcgen05.ld): layer 1 adds the
// level embedding, applies relu and BF16 rounding and writes the map; layer
// 2 adds b2 and reduces the global max-pool (value and first row-major
// position per channel, by a butterfly exchange inside each warp; without
// the positions for inference).  The backward pass recomputes layer 1 the
// same way, uses that the max-pool passes gradient to one pixel per channel
// (a small fraction of the forward work), and accumulates per-CTA partial
// gradients that a second kernel sums in a fixed order (deterministic).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>

#include "af_internal.h"
#include "af_tc.cuh"

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

// Bounded tensor-core waits that gave up (read by af_step_wait_timeouts).
__device__ unsigned int g_cnn_timeouts;

__host__ __device__ constexpr int align128(int b) { return (b + 127) / 128 * 128; }
__host__ __device__ constexpr int imax(int a, int b) { return a > b ? a : b; }

// Tensor-core geometry and shared-memory regions (bytes) of the two
// convolutions for n x n patches (N = n, C components).  BWD: the backward
// pass's layout (layer 1 only: no W2t, the region holds Xh only).
// Both layers are row-shifted GEMMs over pixel-major operands: output
// position q = y P + x of a map with row pitch P reads input row q + ky P +
// kx; the positions with x beyond the map's width are computed and ignored.
//   layer 1: Xh[kc][r][kk] = X[c][r + kx] (r = y S + x, a flat pixel of the
//            input patch; k = 8 kc + kk = 3 c + kx < 3 C, else 0), K = 16:
//            three GEMMs (one per ky, A started ky S rows later), positions
//            q = y S + x with y < n+2, in MT1 tiles of 128;
//   layer 2: as described at the top of this file.
template <int C, int N, bool BWD = false>
struct TcGeo {
    static constexpr int S = N + 4, S1 = N + 2;
    static constexpr int P1 = S1 * S1;                // layer-1 pixels (= rows of the layer-1 map)
    static constexpr int Q1 = S1 * S;                 // layer-1 output positions y S + x, y < n+2
    static constexpr int MT1 = (Q1 + 127) / 128;      // layer-1 M tiles
    static constexpr int RH = MT1 * 128 + 2 * S;      // rows of Xh a layer-1 tile may read
    static constexpr int Q2 = N * S1;                 // layer-2 output positions y (n+2) + x, y < n
    static constexpr int MT2 = (Q2 + 127) / 128;      // layer-2 M tiles
    static constexpr int R1 = MT2 * 128 + 2 * S1 + 2;  // rows of the map a layer-2 tile may read (>= P1)
    static constexpr int xh_chunk = RH * 16;          // one 8-wide column block of Xh
    static constexpr int a1_chunk = R1 * 16;          // one 8-channel block of the layer-1 map
    static constexpr int xbytes = C * S * S * 2;                   // one input patch, BF16 [C][S][S]
    static constexpr int xs = 0;                                   // input patch (forward: two buffers)
    static constexpr int w1t = align128((BWD ? 1 : 2) * xbytes);   // layer-1 B: [3 ky][2][32 g][8 k] BF16
    static constexpr int w2t = w1t + 3 * 2 * 32 * 16;              // layer-2 B: [9][4][32 g][8 f] BF16
    static constexpr int reg = w2t + (BWD ? 0 : 9 * 4 * 32 * 16);   // Xh, then (aliased) the map A1m
    static constexpr int reg_bytes = BWD ? 2 * xh_chunk : imax(2 * xh_chunk, 4 * a1_chunk);
    static constexpr int end = reg + reg_bytes;
    static_assert(3 * C <= 16, "the horizontal taps of every channel fit one K step of 16");
    static_assert(R1 >= P1, "the map holds every layer-1 pixel");
    static_assert(32 * (MT1 > MT2 ? MT1 : MT2) <= 128, "the accumulators fit the tensor-memory columns");
    static_assert(xbytes % 16 == 0, "a patch is a whole number of 16-byte bulk-copy units");
};
constexpr int kTmemCols = 128;  // >= 32 x max(MT1, MT2) columns of FP32 accumulators

__device__ __forceinline__ uint16_t bf16_bits(float v) { return __bfloat16_as_ushort(__float2bfloat16_rn(v)); }

// The tensor-core B operands (BF16, K-major core-matrix blocks) from the
// FP32 parameters: W1t[ky][kc][g][kk] = W1[g][c][ky][kx] with 8 kc + kk =
// 3 c + kx (zero beyond 3C), W2t[ky*3+kx][kc][g][kk] = W2[g][8 kc + kk][ky][kx].
template <int C, int N, int NT, bool BWD>
__device__ void tc_load_weights(const float *__restrict__ P, unsigned char *smem) {
    using G = TcGeo<C, N, BWD>;
    uint16_t *w1 = reinterpret_cast<uint16_t *>(smem + G::w1t);
    for (int e = threadIdx.x; e < 3 * 2 * 32 * 8; e += NT) {
        const int kk = e & 7, g = (e >> 3) & 31, kc = (e >> 8) & 1, ky = e >> 9, k = kc * 8 + kk;
        const int c = k / 3, kx = k - 3 * c;
        w1[e] = k < 3 * C ? bf16_bits(P[off_w1() + g * C * 9 + c * 9 + ky * 3 + kx]) : (uint16_t)0;
    }
    if (BWD) return;
    uint16_t *w2 = reinterpret_cast<uint16_t *>(smem + G::w2t);
    for (int e = threadIdx.x; e < 9 * 4 * 32 * 8; e += NT) {
        const int kk = e & 7, g = (e >> 3) & 31, kc = (e >> 8) & 3, sft = e >> 10;
        w2[e] = bf16_bits(P[off_w2(C) + (g * kF + kc * 8 + kk) * 9 + sft]);
    }
}

// Issue (one thread) layer 1's MMAs (three row shifts per M tile) on Xh
// in the tensor-core region and commit them to *bar.
template <int C, int N, bool BWD>
__device__ __forceinline__ void tc_issue_layer1(unsigned char *smem, uint32_t tmem, uint64_t *bar) {
    using G = TcGeo<C, N, BWD>;
    const uint32_t a0 = tc::saddr(smem + G::reg), b0 = tc::saddr(smem + G::w1t);
    constexpr uint32_t id = tc::idesc_bf16(128, 32);
#pragma unroll
    for (int mt = 0; mt < G::MT1; ++mt)
#pragma unroll
        for (int ky = 0; ky < 3; ++ky)
            tc::mma_bf16(tmem + 32 * mt, tc::smem_desc(a0 + (mt * 128 + ky * G::S) * 16, G::xh_chunk, 128),
                         tc::smem_desc(b0 + ky * 2 * 32 * 16, 32 * 16, 128), id, ky > 0);
    tc::mma_commit(bar);
}

// Issue (one thread) layer 2's MMAs (nine shifts x two K steps per M tile)
// on the layer-1 map in the A1m region and commit them to *bar.
template <int C, int N>
__device__ __forceinline__ void tc_issue_layer2(unsigned char *smem, uint32_t tmem, uint64_t *bar) {
    using G = TcGeo<C, N>;
    const uint32_t a0 = tc::saddr(smem + G::reg), b0 = tc::saddr(smem + G::w2t);
    constexpr uint32_t id = tc::idesc_bf16(128, 32);
#pragma unroll 1
    for (int mt = 0; mt < G::MT2; ++mt)
#pragma unroll
        for (int sft = 0; sft < 9; ++sft) {
            const int ky = sft / 3, kx = sft - 3 * ky;
#pragma unroll
            for (int ks = 0; ks < 2; ++ks)
                tc::mma_bf16(tmem + 32 * mt,
                             tc::smem_desc(a0 + 2 * ks * G::a1_chunk + (mt * 128 + ky * G::S1 + kx) * 16,
                                           G::a1_chunk, 128),
                             tc::smem_desc(b0 + sft * 4 * 32 * 16 + 2 * ks * 32 * 16, 32 * 16, 128), id,
                             sft > 0 || ks > 0);
        }
    tc::mma_commit(bar);
}

// Wait (every thread) for the MMAs committed to *bar, phase `parity`; all
// threads agree on the outcome.  On a wait that gave up: count it, wait once
// more (bounded) so nothing is in flight when the caller frees its tensor
// memory, and return false.
template <int NT>
__device__ __forceinline__ bool tc_wait(uint64_t *bar, unsigned parity) {
    const bool ok = tc::mbar_wait(bar, parity);
    if (__syncthreads_or(!ok)) {
        if (threadIdx.x == 0) {
            atomicAdd(&g_cnn_timeouts, 1u);
            tc::mbar_wait(bar, parity);
        }
        __syncthreads();
        return false;
    }
    tc::fence_after_sync();
    return true;
}

// Layer 1 of sample b on the tensor cores: input patch, its horizontal taps (Xh), MMAs, and
// the epilogue A1 = bf16(relu(D1 + emb[level])) written either as the BF16
// map layer 2 reads (F32OUT false) or as an FP32 map a1[f][y][x] (F32OUT
// true, the backward pass).  xin: the patch already in shared memory, or
// null (it is then read from X[b]).  Ends with a barrier; false if the wait
// gave up.
template <int C, int N, int NT, bool F32OUT>
__device__ bool tc_layer1(const __nv_bfloat16 *__restrict__ X, int b, const uint16_t *xin, const float *emb,
                          unsigned char *smem, uint32_t tmem, uint64_t *bar, unsigned &phase, float *a1) {
    using G = TcGeo<C, N, F32OUT>;
    constexpr int S = G::S, S1 = G::S1;
    const uint16_t *xs = xin;
    if (xs == nullptr) {
        const uint16_t *xb = reinterpret_cast<const uint16_t *>(X) + (int64_t)b * C * S * S;
        uint16_t *xw = reinterpret_cast<uint16_t *>(smem + G::xs);
        for (int e = threadIdx.x; e < C * S * S; e += NT) xw[e] = xb[e];
        __syncthreads();
        xs = xw;
    }
    // Xh, one row (both 16-byte column blocks) per item: the horizontal taps
    // X[c][r + kx] of flat pixel r of every channel (zero beyond the patch)
    for (int r = threadIdx.x; r < G::RH; r += NT) {
        uint32_t w[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
#pragma unroll
        for (int c = 0; c < C; ++c)
#pragma unroll
            for (int kx = 0; kx < 3; ++kx) {
                const int k = 3 * c + kx;
                const uint32_t v = r + kx < S * S ? (uint32_t)xs[c * S * S + r + kx] : 0u;
                w[k >> 1] |= v << (16 * (k & 1));
            }
        *reinterpret_cast<uint4 *>(smem + G::reg + r * 16) = make_uint4(w[0], w[1], w[2], w[3]);
        *reinterpret_cast<uint4 *>(smem + G::reg + G::xh_chunk + r * 16) = make_uint4(w[4], w[5], w[6], w[7]);
    }
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    __syncthreads();
    if (threadIdx.x == 0) {
        tc::fence_after_sync();
        tc_issue_layer1<C, N, F32OUT>(smem, tmem, bar);
    }
    if (!tc_wait<NT>(bar, phase)) return false;
    phase ^= 1u;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t lanes = (uint32_t)(32 * (warp & 3)) << 16;
    for (int mt = warp >> 2; mt < G::MT1; mt += NT / 128) {
        float z[32];
        tc::tmem_ld32(tmem + lanes + 32 * mt, z);
        // output position q = y S + x: layer-1 pixel m = y (n+2) + x if x < n+2
        const int q = mt * 128 + 32 * (warp & 3) + lane, y = q / S, x = q - y * S;
        const int m = y * S1 + x;
        if (y < S1 && x < S1) {
            if constexpr (F32OUT) {
#pragma unroll
                for (int g = 0; g < kF; ++g) a1[g * G::P1 + m] = rbf(fmaxf(z[g] + emb[g], 0.f));
            } else {
                // the map A1m[kc][m][8 channels], row m = the layer-1 pixel;
                // channel pairs added as packed FP32x2 and converted to a
                // BF16 pair in one instruction (each value rounded as alone)
#pragma unroll
                for (int kc = 0; kc < 4; ++kc) {
                    uint32_t w[4];
#pragma unroll
                    for (int h = 0; h < 4; ++h) {
                        const int g = kc * 8 + 2 * h;
                        const float2 a = __fadd2_rn(make_float2(z[g], z[g + 1]), make_float2(emb[g], emb[g + 1]));
                        const __nv_bfloat162 r = __floats2bfloat162_rn(fmaxf(a.x, 0.f), fmaxf(a.y, 0.f));
                        w[h] = *reinterpret_cast<const uint32_t *>(&r);
                    }
                    *reinterpret_cast<uint4 *>(smem + G::reg + kc * G::a1_chunk + m * 16) =
                        make_uint4(w[0], w[1], w[2], w[3]);
                }
            }
        }
    }
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    __syncthreads();
    return true;
}

// Forward pass: one CTA (one warpgroup) per patch at a time.  POS: also the
// first row-major position of every channel's maximum (training: the
// backward pass needs it); without it (inference) a channel's maximum is
// max_q D2[q][g] + b2[g], which equals max_q (D2[q][g] + b2[g]) bit for bit
// because rounding an addition of the same b2 is monotonic.
template <int C, int N, bool POS>
__global__ void __launch_bounds__(128) cnn_forward_kernel(int nsample, const __nv_bfloat16 *__restrict__ X,
                                                          const int32_t *__restrict__ level,
                                                          const float *__restrict__ P, float *__restrict__ logit,
                                                          float *__restrict__ Mout, int32_t *__restrict__ Aout) {
    using G = TcGeo<C, N>;
    constexpr int NT = 128;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar, xbar[2];
    __shared__ uint32_t tslot;
    __shared__ __align__(16) float s_emb[kLevels * kF], s_b2[kF], s_w3[kF], s_b3;
    __shared__ float s_best[4][kF];
    __shared__ int s_idx[4][kF];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    tc_load_weights<C, N, NT, false>(P, smem);
    for (int e = threadIdx.x; e < kLevels * kF; e += NT) s_emb[e] = P[off_emb(C) + e];
    if (threadIdx.x < kF) {
        s_b2[threadIdx.x] = P[off_b2(C) + threadIdx.x];
        s_w3[threadIdx.x] = P[off_w3(C) + threadIdx.x];
    }
    // the input patches go through two buffers, each filled by one bulk copy
    // completing on its own mbarrier; the next patch's copy is issued at the
    // start of the current one
    auto xbuf = [&](int k) { return reinterpret_cast<uint16_t *>(smem + G::xs + k * G::xbytes); };
    const uint16_t *const X16 = reinterpret_cast<const uint16_t *>(X);
    if (threadIdx.x == 0) {
        s_b3 = P[off_b3(C)];
        tc::mbar_init(&bar, 1);
        tc::mbar_init(&xbar[0], 1);
        tc::mbar_init(&xbar[1], 1);
    }
    if (warp == 0) tc::tmem_alloc(&tslot, kTmemCols);
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (threadIdx.x == 0 && blockIdx.x < nsample) {
        tc::mbar_expect_tx(&xbar[0], G::xbytes);
        tc::bulk_g2s(xbuf(0), X16 + (int64_t)blockIdx.x * (G::xbytes / 2), G::xbytes, &xbar[0]);
    }
    const uint32_t tmem = tslot, lanes = (uint32_t)(32 * warp) << 16;
    unsigned phase = 0;
    int it = 0;
    bool next_pending = false;  // a bulk copy into buffer (it + 1) & 1 is in flight
    for (int b = blockIdx.x; b < nsample; b += gridDim.x, ++it) {
        const int cur = it & 1;
        next_pending = b + (int)gridDim.x < nsample;
        if (threadIdx.x == 0 && next_pending) {
            // the other buffer was last read before the barrier that ended
            // layer 1 of the previous patch
            tc::fence_smem_to_async();
            tc::mbar_expect_tx(&xbar[cur ^ 1], G::xbytes);
            tc::bulk_g2s(xbuf(cur ^ 1), X16 + (int64_t)(b + gridDim.x) * (G::xbytes / 2), G::xbytes,
                         &xbar[cur ^ 1]);
        }
        const int lv = min(max(level[b], 0), kLevels - 1);
        if (!tc_wait<NT>(&xbar[cur], (unsigned)(it >> 1) & 1u)) break;
        if (!tc_layer1<C, N, NT, false>(X, b, xbuf(cur), s_emb + lv * kF, smem, tmem, &bar, phase, nullptr)) break;
        if (threadIdx.x == 0) {
            tc::fence_after_sync();
            tc_issue_layer2<C, N>(smem, tmem, &bar);
        }
        if (!tc_wait<NT>(&bar, phase)) break;
        phase ^= 1u;
        // max-pool of Z2 = D2 + b2 over the n^2 output pixels (pixel index =
        // row-major position y n + x; the first maximum wins)
        float best[kF];
        int bi[kF];
#pragma unroll
        for (int g = 0; g < kF; ++g) {
            best[g] = -INFINITY;
            bi[g] = 0x7fffffff;
        }
#pragma unroll 1
        for (int mt = 0; mt < G::MT2; ++mt) {
            float z[32];
            tc::tmem_ld32(tmem + lanes + 32 * mt, z);
            const int q = mt * 128 + 32 * warp + lane, y = q / G::S1, x = q - y * G::S1;
            if (y < N && x < N) {
                if constexpr (POS) {
                    // a thread visits its positions in increasing order, so a
                    // strict comparison keeps the first maximum; a channel whose
                    // maximum is not positive reports no position (-1) below,
                    // whatever a thread kept for -inf or NaN values
                    const int p = y * N + x;
#pragma unroll
                    for (int g = 0; g < kF; ++g) {
                        const float v = z[g] + s_b2[g];
                        if (v > best[g]) {
                            best[g] = v;
                            bi[g] = p;
                        }
                    }
                } else {
                    // b2 is added after the reduction (NaN accumulators are
                    // skipped by fmaxf as by the comparison above)
#pragma unroll
                    for (int g = 0; g < kF; ++g) best[g] = fmaxf(best[g], z[g]);
                }
            }
        }
        // butterfly over the warp: after the exchange at distance o, a lane
        // keeps the half of its channels selected by its bit o and merges
        // them with its partner's; lane L ends with channel L
#pragma unroll
        for (int o = 16, w = 16; o >= 1; o >>= 1, w >>= 1) {
            const bool upper = (lane & o) != 0;
#pragma unroll
            for (int j = 0; j < w; ++j) {
                const float sv = upper ? best[j] : best[j + w];
                const float kv = upper ? best[j + w] : best[j];
                const float ov = __shfl_xor_sync(0xffffffffu, sv, o);
                if constexpr (POS) {
                    const int si = upper ? bi[j] : bi[j + w];
                    const int ki = upper ? bi[j + w] : bi[j];
                    const int oi = __shfl_xor_sync(0xffffffffu, si, o);
                    const bool take = ov > kv || (ov == kv && oi < ki);
                    best[j] = take ? ov : kv;
                    bi[j] = take ? oi : ki;
                } else {
                    best[j] = fmaxf(ov, kv);
                }
            }
        }
        s_best[warp][lane] = best[0];
        if constexpr (POS) s_idx[warp][lane] = bi[0];
        tc::fence_before_sync();
        __syncthreads();
        if (warp == 0) {
            const int g = lane;
            float bv = s_best[0][g];
            int ix = 0;
            if constexpr (POS) {
                ix = s_idx[0][g];
#pragma unroll
                for (int w = 1; w < 4; ++w) {
                    const float ob = s_best[w][g];
                    const int oi = s_idx[w][g];
                    if (ob > bv || (ob == bv && oi < ix)) {
                        bv = ob;
                        ix = oi;
                    }
                }
            } else {
#pragma unroll
                for (int w = 1; w < 4; ++w) bv = fmaxf(bv, s_best[w][g]);
                bv += s_b2[g];
            }
            const float mg = bv > 0.f ? bv : 0.f;
            float v = s_w3[g] * mg;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            Mout[(int64_t)b * kF + g] = mg;
            if constexpr (POS) Aout[(int64_t)b * kF + g] = bv > 0.f ? ix : -1;
            if (g == 0) logit[b] = v + s_b3;
        }
        __syncthreads();
    }
    // after a wait that gave up: the copy of the next patch may still be in
    // flight (bounded wait)
    if (next_pending && threadIdx.x == 0) tc::mbar_wait(&xbar[(it + 1) & 1], (unsigned)((it + 1) >> 1) & 1u);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, kTmemCols);
}

// Byte offset of the backward pass's tensor-core region, after its FP32 arrays.
template <int C, int N>
__host__ __device__ constexpr int bwd_tc_offset() { return align128(4 * Smem<C, N>::bwd_end); }

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
    constexpr int NT = 256;
    extern __shared__ __align__(128) float sm[];
    __shared__ float s_dz[kF];
    __shared__ int s_arg[kF];
    __shared__ float s_dlogit;
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tslot;
    unsigned char *const tcs = reinterpret_cast<unsigned char *>(sm) + bwd_tc_offset<C, N>();
    load_weights<C, N>(P, sm);
    tc_load_weights<C, N, NT, true>(P, tcs);
    for (int e = threadIdx.x; e < L::bwd_end - L::gw1; e += blockDim.x) sm[L::gw1 + e] = 0.f;
    if (threadIdx.x == 0) tc::mbar_init(&bar, 1);
    if (threadIdx.x < 32) tc::tmem_alloc(&tslot, kTmemCols);
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tslot;
    unsigned phase = 0;
    for (int b = blockIdx.x; b < nsample; b += gridDim.x) {
        const int lv = min(max(level[b], 0), kLevels - 1);
        // layer 1 recomputed on the tensor cores (A1 as an FP32 map), and the
        // input patch in FP32 for the W1 gradient
        if (!tc_layer1<C, N, NT, true>(X, b, nullptr, sm + L::emb + lv * kF, tcs, tmem, &bar, phase, sm + L::a1))
            break;
        const uint16_t *xs = reinterpret_cast<const uint16_t *>(tcs + TcGeo<C, N, true>::xs);
        for (int e = threadIdx.x; e < C * S * S; e += NT) sm[L::x + e] = __uint_as_float((uint32_t)xs[e] << 16);
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
    tc::fence_before_sync();
    __syncthreads();
    if (threadIdx.x < 32) tc::tmem_dealloc(tmem, kTmemCols);
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

// Allows `bytes` of dynamic shared memory (the default limit of 48 KB covers
// static and dynamic shared memory together) and asks for the largest
// shared-memory carveout, so that several CTAs fit on an SM.
template <typename K>
af_status smem_attr(K k, size_t bytes) {
    if (bytes > 227 * 1024) return AF_ERR_UNIMPLEMENTED;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess ||
        cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared) !=
            cudaSuccess)
        return AF_ERR_CUDA;
    return AF_OK;
}

inline af_status launched() { return cudaGetLastError() == cudaSuccess ? AF_OK : AF_ERR_CUDA; }

template <int C, int N, bool POS>
af_status forward_launch(int nsample, const void *X, const int32_t *lev, const float *P, float *lg, float *M,
                         int32_t *A, cudaStream_t s) {
    auto k = cnn_forward_kernel<C, N, POS>;
    const size_t bytes = TcGeo<C, N>::end;
    if (const af_status e = smem_attr(k, bytes)) return e;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return AF_ERR_CUDA;
    // persistent CTAs: as many per SM as tensor memory holds (512 columns)
    // and shared memory allows (static + dynamic + the per-CTA reserve)
    int smem_sm = 0, reserved = 0;
    cudaFuncAttributes fa;
    if (cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess ||
        cudaFuncGetAttributes(&fa, k) != cudaSuccess)
        return AF_ERR_CUDA;
    int per_sm = smem_sm / (int)(bytes + fa.sharedSizeBytes + reserved);
    per_sm = per_sm < 1 ? 1 : (per_sm > 512 / kTmemCols ? 512 / kTmemCols : per_sm);
    const int slots = sms * per_sm;
    const int grid = nsample < slots ? nsample : slots;
    k<<<grid, 128, bytes, s>>>(nsample, static_cast<const __nv_bfloat16 *>(X), lev, P, lg, M, A);
    return launched();
}

template <int C, int N>
af_status backward_launch(int nsample, const void *X, const int32_t *lev, const float *P, const float *lg,
                          const float *M, const int32_t *A, const float *y, const float *om, float inv_om,
                          float *partial, int nblocks, float *grad, cudaStream_t s) {
    auto k = cnn_backward_kernel<C, N>;
    const size_t bytes = bwd_tc_offset<C, N>() + TcGeo<C, N, true>::end;
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

// Reads (and, if reset, clears) the count of tagger kernels whose bounded
// tensor-core wait gave up.
af_status wait_timeouts_cnn(unsigned int *count, bool reset) {
    unsigned int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_cnn_timeouts, sizeof(v)) != cudaSuccess) return AF_ERR_CUDA;
    *count = v;
    if (reset && v != 0) {
        const unsigned int zero = 0;
        if (cudaMemcpyToSymbol(g_cnn_timeouts, &zero, sizeof(zero)) != cudaSuccess) return AF_ERR_CUDA;
    }
    return AF_OK;
}
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
    if (!d_x || !d_level || !d_params || !d_logit || !d_m) return AF_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (d_arg != nullptr) {  // training: the positions too
        if (ncomp == 3)
            return n == 16 ? forward_launch<3, 16, true>(nsample, d_x, d_level, d_params, d_logit, d_m, d_arg, s)
                           : forward_launch<3, 8, true>(nsample, d_x, d_level, d_params, d_logit, d_m, d_arg, s);
        return n == 16 ? forward_launch<1, 16, true>(nsample, d_x, d_level, d_params, d_logit, d_m, d_arg, s)
                       : forward_launch<1, 8, true>(nsample, d_x, d_level, d_params, d_logit, d_m, d_arg, s);
    }
    if (ncomp == 3)
        return n == 16 ? forward_launch<3, 16, false>(nsample, d_x, d_level, d_params, d_logit, d_m, nullptr, s)
                       : forward_launch<3, 8, false>(nsample, d_x, d_level, d_params, d_logit, d_m, nullptr, s);
    return n == 16 ? forward_launch<1, 16, false>(nsample, d_x, d_level, d_params, d_logit, d_m, nullptr, s)
                   : forward_launch<1, 8, false>(nsample, d_x, d_level, d_params, d_logit, d_m, nullptr, s);
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

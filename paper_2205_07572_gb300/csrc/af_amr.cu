// Adaptive-mesh kernels of libaf.so (Section 3 of arXiv 2205.07572):
// ghost exchange, regrid transfer, conservative fix, tagging, mass totals.
//
// Positions are exact integers: one unit is half the cell width of level
// lmax, so a level-l cell is 2^(lmax-l+1) units wide and every node, cell
// centre and Simpson point is a lattice point of that unit.  The forest is
// located through per-level region maps (af_forest.d_map), which stay in L2.
#include <cuda_runtime.h>

#include <cstring>

#include "af_internal.h"

namespace af {
namespace {

struct DevForest {
    int nleaf, B, lmax, n;
    const int32_t *level, *ix, *iy, *map;
    long long D;  // domain width in units
};

DevForest make_dev(const af_forest &f, int n) {
    DevForest d;
    d.nleaf = f.nleaf;
    d.B = f.B;
    d.lmax = f.lmax;
    d.n = n;
    d.level = f.d_level;
    d.ix = f.d_ix;
    d.iy = f.d_iy;
    d.map = f.d_map;
    d.D = (long long)f.B * n * (2LL << f.lmax);
    return d;
}

__host__ __device__ inline long long map_offset(int B, int l) {
    // sum_{m<l} (B << m)^2 = B^2 (4^l - 1) / 3
    return (long long)B * B * (((1LL << (2 * l)) - 1) / 3);
}

__device__ __forceinline__ long long hwid(const DevForest &F, int l) { return 2LL << (F.lmax - l); }

__device__ __forceinline__ long long wrapd(const DevForest &F, long long x) {
    // positions are at most one domain width outside [0, D)
    if (x >= 0 && x < F.D) return x;
    if (x < 0 && x >= -F.D) return x + F.D;
    if (x >= F.D && x < 2 * F.D) return x - F.D;
    long long r = x % F.D;
    return r < 0 ? r + F.D : r;
}

// Leaf whose half-open extent contains (x, y).  A region of the finest level
// lmax is a leaf (entry q >= 0) or lies inside the coarser leaf -2 - entry
// (af_forest_build_map), so one load finds it; a map without that second
// kind of entry is searched level by level.
__device__ int lookup(const DevForest &F, long long x, long long y) {
    x = wrapd(F, x);
    y = wrapd(F, y);
    {
        const long long pw = 2LL * F.n;  // a finest-level region, in units
        const long long side = (long long)F.B << F.lmax;
        const int q = __ldg(F.map + map_offset(F.B, F.lmax) + (y / pw) * side + (x / pw));
        if (q >= 0) return q < F.nleaf ? q : -1;
        if (q <= -2) return -2 - q < F.nleaf ? -2 - q : -1;
    }
    for (int l = F.lmax - 1; l >= 0; --l) {
        const long long pw = (long long)F.n * hwid(F, l);
        const long long side = (long long)F.B << l;
        const int q = __ldg(F.map + map_offset(F.B, l) + (y / pw) * side + (x / pw));
        if (q >= 0) return q < F.nleaf ? q : -1;
    }
    return -1;
}

// Owner of a point value: the finest leaf touching the point, ties in the
// order above-right, above-left, below-right, below-left.
__device__ int node_owner(const DevForest &F, long long x, long long y) {
    int best = lookup(F, x, y);
    int bl = best >= 0 ? __ldg(F.level + best) : -1;
    const long long dx[3] = {-1, 0, -1}, dy[3] = {0, -1, -1};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int q = lookup(F, x + dx[k], y + dy[k]);
        if (q >= 0) {
            const int lq = __ldg(F.level + q);
            if (lq > bl) {
                best = q;
                bl = lq;
            }
        }
    }
    return best;
}

__device__ __forceinline__ int entry_owner(const DevForest &F, int plane, long long x, long long y) {
    return plane == kAvg ? lookup(F, x, y) : node_owner(F, x, y);
}

__device__ __forceinline__ long long leaf_x0(const DevForest &F, int q) {
    return (long long)__ldg(F.ix + q) * F.n * hwid(F, __ldg(F.level + q));
}
__device__ __forceinline__ long long leaf_y0(const DevForest &F, int q) {
    return (long long)__ldg(F.iy + q) * F.n * hwid(F, __ldg(F.level + q));
}

// x - x0 unwrapped across the periodic box
__device__ __forceinline__ long long reld(const DevForest &F, long long x, long long x0) {
    long long d = wrapd(F, x - x0);
    return d > F.D / 2 ? d - F.D : d;
}

// State of all leaves: one array, or two with a per-level choice of the
// current one (af_state_pair).
template <typename T>
struct StateView {
    T *base0, *base1;
    const int32_t *level;  // leaf levels (read only when parity != 0)
    uint32_t parity;       // bit l: level l is current in base1
    int64_t plane;         // plane stride
    int ncomp, W;          // components, lattice width
    __device__ __forceinline__ T *patch(int q) const {
        T *b = (parity != 0u && ((parity >> __ldg(level + q)) & 1u)) ? base1 : base0;
        return b + (int64_t)q * ncomp * kPlanes * plane;
    }
    __device__ __forceinline__ T *patch_at_level(int q, int l) const {
        return (((parity >> l) & 1u) ? base1 : base0) + (int64_t)q * ncomp * kPlanes * plane;
    }
    __device__ __forceinline__ T *at(int q, int c, int k, int i, int j) const {
        return patch(q) + (int64_t)(c * kPlanes + k) * plane + (int64_t)(j + kGhost) * W + (i + kGhost);
    }
};

// Lattice indices (i, j) of point (x, y) in plane k of leaf q.
__device__ __forceinline__ void lattice_of(const DevForest &F, int q, int k, long long x, long long y, int &i,
                                           int &j) {
    const int sh = F.lmax - __ldg(F.level + q) + 1;  // hw = 2^sh
    const long long hw = 1LL << sh;
    long long dx = reld(F, x, leaf_x0(F, q)), dy = reld(F, y, leaf_y0(F, q));
    if (k == kAvg || k == kYmid) dx -= hw / 2;
    if (k == kAvg || k == kXmid) dy -= hw / 2;
    i = (int)(dx >> sh);  // floor division (arithmetic shift)
    j = (int)(dy >> sh);
    // owners are always within two cells of the lattice; clamp defensively
    const int lo = -kGhost, hi = F.n + kGhost;
    i = i < lo ? lo : (i > hi ? hi : i);
    j = j < lo ? lo : (j > hi ? hi : j);
}

// Explicitly rounded operations: the reconstruction below is evaluated in
// one fixed order of roundings wherever it is inlined, so the direct and the
// planned ghost exchange (and the regrid transfer) agree bit for bit.
__device__ __forceinline__ float r_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double r_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float r_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double r_sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float r_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double r_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float r_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double r_fma(double a, double b, double c) { return __fma_rn(a, b, c); }

// sum_a w_a row_a of the three rows of nodal values with weights (l0, l1, l2)
// in x and (m0, m1, m2) in y.
template <typename R>
__device__ __forceinline__ R recon_combine(R c00, R c10, R c01, R c11, R xl, R xr, R yb, R yt, R cen, R l0, R l1,
                                           R l2, R m0, R m1, R m2) {
    const R r0 = r_fma(l2, c10, r_fma(l1, yb, r_mul(l0, c00)));
    const R r1 = r_fma(l2, xr, r_fma(l1, cen, r_mul(l0, xl)));
    const R r2 = r_fma(l2, c11, r_fma(l1, yt, r_mul(l0, c01)));
    return r_fma(m2, r2, r_fma(m1, r1, r_mul(m0, r0)));
}

// The centre value of the biquadratic from its average and boundary nodes:
// (9/4) Q - (1/16) sum(corners) - (1/4) sum(edge midpoints).
template <typename R>
__device__ __forceinline__ R recon_centre(R c00, R c10, R c01, R c11, R xl, R xr, R yb, R yt, R avg) {
    const R sc = r_add(r_add(c00, c10), r_add(c01, c11)), se = r_add(r_add(xl, xr), r_add(yb, yt));
    return r_sub(r_sub(r_mul(R(2.25), avg), r_mul(R(0.0625), sc)), r_mul(R(0.25), se));
}

// The reconstruction (Eq. poly) of one cell at (xi, eta) in [-1, 1]^2 from
// its corners c.., edge midpoints x./y. and average: the tensor Lagrange
// interpolant on {-1,0,1}^2 whose centre value follows from the average.
// Evaluated in the state's precision R (FP32 for an FP32 state: GB300's
// FP64 rate is a small fraction of its FP32 rate).
template <typename R>
__device__ __forceinline__ R recon_eval(R c00, R c10, R c01, R c11, R xl, R xr, R yb, R yt, R avg, R xi, R eta) {
    const R cen = recon_centre<R>(c00, c10, c01, c11, xl, xr, yb, yt, avg);
    const R lx0 = r_mul(r_mul(R(0.5), xi), r_sub(xi, R(1))), lx1 = r_sub(R(1), r_mul(xi, xi));
    const R lx2 = r_mul(r_mul(R(0.5), xi), r_add(xi, R(1)));
    const R ly0 = r_mul(r_mul(R(0.5), eta), r_sub(eta, R(1))), ly1 = r_sub(R(1), r_mul(eta, eta));
    const R ly2 = r_mul(r_mul(R(0.5), eta), r_add(eta, R(1)));
    return recon_combine<R>(c00, c10, c01, c11, xl, xr, yb, yt, cen, lx0, lx1, lx2, ly0, ly1, ly2);
}

// Mean of the biquadratic reconstruction of a cell (nodal values as for
// recon_eval) over one of its four quarters: qx, qy = 0 for the lower half
// (xi or eta in [-1, 0]), 1 for the upper half.  The mean of each 1D
// Lagrange basis function over a half interval replaces its point value:
// over [-1, 0] the three functions average 5/12, 2/3, -1/12, over [0, 1]
// -1/12, 2/3, 5/12.  This is exactly the Simpson rule over the quarter
// (exact for quadratics), in 9 multiply-adds instead of 9 evaluations.
template <typename R>
__device__ __forceinline__ R recon_quarter_mean(R c00, R c10, R c01, R c11, R xl, R xr, R yb, R yt, R avg, int qx,
                                                int qy) {
    const R cen = recon_centre<R>(c00, c10, c01, c11, xl, xr, yb, yt, avg);
    const R lo = R(5) / R(12), mid = R(2) / R(3), hi = R(-1) / R(12);
    return recon_combine<R>(c00, c10, c01, c11, xl, xr, yb, yt, cen, qx ? hi : lo, mid, qx ? lo : hi,
                            qy ? hi : lo, mid, qy ? lo : hi);
}

// Simpson's rule over a cell from the values f(a, b) at its 3 x 3 points
// (a, b in {0, 1, 2}): exact for the biquadratic reconstruction.
template <typename R, typename Fn>
__device__ __forceinline__ R simpson9(Fn f) {
    const R w[3] = {R(1) / R(6), R(2) / R(3), R(1) / R(6)};
    R s = R(0);
    for (int b = 0; b < 3; ++b)
        for (int a = 0; a < 3; ++a) s = r_fma(r_mul(w[a], w[b]), f(a, b), s);
    return s;
}

// The nine values the reconstruction of one cell of leaf q combines at
// (x, y) (component 0; component c is cstride entries further), and where
// (x, y) lies in the cell.
template <typename T>
struct ReconSite {
    const T *v[9];  // c00, c10, c01, c11, xl, xr, yb, yt, avg
    T xi, eta;      // position in [-1, 1]^2
    int qx, qy;     // quarter holding (x, y)
};

template <typename T>
__device__ void recon_locate(const DevForest &F, const StateView<T> &S, int q, long long x, long long y,
                             ReconSite<T> &r) {
    const int sh = F.lmax - __ldg(F.level + q) + 1;  // hw = 2^sh
    const long long hw = 1LL << sh;
    const long long dx = reld(F, x, leaf_x0(F, q)), dy = reld(F, y, leaf_y0(F, q));
    long long ci = dx >= 0 ? (dx >> sh) : -1, cj = dy >= 0 ? (dy >> sh) : -1;
    ci = ci < 0 ? 0 : (ci > F.n - 1 ? F.n - 1 : ci);
    cj = cj < 0 ? 0 : (cj > F.n - 1 ? F.n - 1 : cj);
    r.xi = (T)(2.0 * (double)(dx - ci * hw) / (double)hw - 1.0);  // exact: a multiple of 1/2
    r.eta = (T)(2.0 * (double)(dy - cj * hw) / (double)hw - 1.0);
    r.qx = 2 * (dx - ci * hw) >= hw;
    r.qy = 2 * (dy - cj * hw) >= hw;
    const int i = (int)ci, j = (int)cj;
    // Point values on the leaf's boundary lines are read from their owner:
    // a leaf whose neighbours are all same-level does not keep the copies in
    // its ghost ring current (its step reads the neighbours directly).
    auto node = [&](int k, int ii, int jj) -> const T * {
        if (ii > 0 && ii < F.n && jj > 0 && jj < F.n) return S.at(q, 0, k, ii, jj);
        const long long x0 = leaf_x0(F, q), y0 = leaf_y0(F, q);
        const long long nx = x0 + (long long)ii * hw + (k == kYmid ? hw / 2 : 0);
        const long long ny = y0 + (long long)jj * hw + (k == kXmid ? hw / 2 : 0);
        const int o = node_owner(F, nx, ny);
        if (o < 0 || o == q) return S.at(q, 0, k, ii, jj);
        const int lo = __ldg(F.level + o);
        const int ko = lo == __ldg(F.level + q) ? k : kCorner;
        int oi, oj;
        lattice_of(F, o, ko, nx, ny, oi, oj);
        return S.at(o, 0, ko, oi, oj);
    };
    r.v[0] = node(kCorner, i, j);
    r.v[1] = node(kCorner, i + 1, j);
    r.v[2] = node(kCorner, i, j + 1);
    r.v[3] = node(kCorner, i + 1, j + 1);
    r.v[4] = node(kXmid, i, j);
    r.v[5] = node(kXmid, i + 1, j);
    r.v[6] = node(kYmid, i, j);
    r.v[7] = node(kYmid, i, j + 1);
    r.v[8] = S.at(q, 0, kAvg, i, j);
}

// The reconstruction at a located site (quarter: its mean over the quarter
// of the cell holding the site instead), component offset coff.
template <typename T>
__device__ __forceinline__ T recon_value(const ReconSite<T> &r, int64_t coff, bool quarter) {
    T v[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) v[e] = r.v[e][coff];
    if (quarter) return recon_quarter_mean<T>(v[0], v[1], v[2], v[3], v[4], v[5], v[6], v[7], v[8], r.qx, r.qy);
    return recon_eval<T>(v[0], v[1], v[2], v[3], v[4], v[5], v[6], v[7], v[8], r.xi, r.eta);
}

// Value of the reconstruction of leaf q, component c, at (x, y); with
// quarter set instead the mean of the reconstruction over the quarter of the
// cell holding (x, y) that (x, y) lies in (the centre of a finer cell).
template <typename T>
__device__ T recon_at(const DevForest &F, const StateView<T> &S, int q, int c, long long x, long long y,
                      bool quarter = false) {
    ReconSite<T> r;
    recon_locate<T>(F, S, q, x, y, r);
    return recon_value<T>(r, (int64_t)c * kPlanes * S.plane, quarter);
}

// Value for an entry of plane k of a destination at level lp from owner q
// (Section 3.1: copy, fine -> coarse, coarse -> fine).
template <typename T>
__device__ double transfer(const DevForest &F, const StateView<T> &S, int lp, int q, int c, int k, long long x,
                           long long y) {
    const int lq = __ldg(F.level + q);
    int i, j;
    if (lq == lp) {
        lattice_of(F, q, k, x, y, i, j);
        return *S.at(q, c, k, i, j);
    }
    if (lq > lp) {
        if (k == kAvg) {
            const long long h = hwid(F, lq) / 2;
            double s = 0.0;
#pragma unroll
            for (int b = -1; b <= 1; b += 2)
#pragma unroll
                for (int a = -1; a <= 1; a += 2) {
                    lattice_of(F, q, kAvg, x + a * h, y + b * h, i, j);
                    s += *S.at(q, c, kAvg, i, j);
                }
            return 0.25 * s;
        }
        lattice_of(F, q, kCorner, x, y, i, j);
        return *S.at(q, c, kCorner, i, j);
    }
    if (k != kAvg) return (double)recon_at<T>(F, S, q, c, x, y);
    // the mean of the coarse biquadratic over the destination cell, a quarter
    // of a coarse cell (the Simpson rule over it, exact for the biquadratic)
    if (lq == lp - 1) return (double)recon_at<T>(F, S, q, c, x, y, true);
    const long long h = hwid(F, lp) / 2;
    return (double)simpson9<T>([&](int a, int b) { return recon_at<T>(F, S, q, c, x + (a - 1) * h, y + (b - 1) * h); });
}

// transfer() for every component c < nc at once (the owner's sites are
// located once): out[c].
template <typename T>
__device__ void transfer_all(const DevForest &F, const StateView<T> &S, int lp, int q, int k, long long x,
                             long long y, int nc, double out[3]) {
    const int lq = __ldg(F.level + q);
    const int64_t cs = (int64_t)kPlanes * S.plane;
    int i, j;
    if (lq == lp || (lq > lp && k != kAvg)) {
        const int ko = lq == lp ? k : kCorner;
        lattice_of(F, q, ko, x, y, i, j);
        const T *v = S.at(q, 0, ko, i, j);
        for (int c = 0; c < nc; ++c) out[c] = (double)v[c * cs];
        return;
    }
    if (lq > lp) {  // an average from a finer owner: the mean of its four cells
        const long long h = hwid(F, lq) / 2;
        const T *v[4];
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                lattice_of(F, q, kAvg, x + (2 * a - 1) * h, y + (2 * b - 1) * h, i, j);
                v[2 * b + a] = S.at(q, 0, kAvg, i, j);
            }
        for (int c = 0; c < nc; ++c) {
            // the same order of additions as transfer()
            double s = 0.0;
            s += (double)v[0][c * cs];
            s += (double)v[1][c * cs];
            s += (double)v[2][c * cs];
            s += (double)v[3][c * cs];
            out[c] = 0.25 * s;
        }
        return;
    }
    if (k != kAvg || lq == lp - 1) {  // a coarser owner: its reconstruction (quarter mean for an average)
        ReconSite<T> r;
        recon_locate<T>(F, S, q, x, y, r);
        for (int c = 0; c < nc; ++c) out[c] = (double)recon_value<T>(r, c * cs, k == kAvg);
        return;
    }
    for (int c = 0; c < nc; ++c) out[c] = transfer<T>(F, S, lp, q, c, k, x, y);
}

__device__ __forceinline__ void entry_xy(const DevForest &F, int p, int k, int i, int j, long long &x, long long &y) {
    const long long hw = hwid(F, __ldg(F.level + p));
    x = leaf_x0(F, p) + (long long)i * hw + ((k == kAvg || k == kYmid) ? hw / 2 : 0);
    y = leaf_y0(F, p) + (long long)j * hw + ((k == kAvg || k == kXmid) ? hw / 2 : 0);
}

// True if some neighbour region of leaf p at its own level is not a leaf.
__device__ bool has_other_level_neighbour(const DevForest &F, int p) {
    const int l = __ldg(F.level + p);
    const long long side = (long long)F.B << l;
    const long long px = __ldg(F.ix + p), py = __ldg(F.iy + p);
    for (int sy = -1; sy <= 1; ++sy)
        for (int sx = -1; sx <= 1; ++sx) {
            if (sx == 0 && sy == 0) continue;
            const long long nx = ((px + sx) % side + side) % side, ny = ((py + sy) % side + side) % side;
            if (__ldg(F.map + map_offset(F.B, l) + ny * side + nx) < 0) return true;
        }
    return false;
}

// One pass of the exchange: pass 0 = finer owners, 1 = same level, 2 = coarser.
template <typename T>
__global__ void fill_kernel(DevForest F, StateView<T> S, uint32_t dst, uint32_t src, int flags, int pass) {
    const int p = blockIdx.x;
    const int lp = __ldg(F.level + p);
    if (!((dst >> lp) & 1u)) return;
    __shared__ int s_skip;
    if (threadIdx.x == 0) s_skip = !(flags & AF_FILL_ALL_PATCHES) && !has_other_level_neighbour(F, p);
    __syncthreads();
    if (s_skip) return;
    const int n = F.n, W = n + 2 * kGhost + 1;
    const int total = kPlanes * W * W;
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        const int k = e / (W * W), r = e - k * W * W;
        const int j = r / W - kGhost, i = r % W - kGhost;
        if (i > 0 && i < n && j > 0 && j < n) continue;  // strictly inside: the leaf's own
        if (i == n + kGhost && (k == kAvg || k == kYmid)) continue;  // never read by the step
        if (j == n + kGhost && (k == kAvg || k == kXmid)) continue;
        long long x, y;
        entry_xy(F, p, k, i, j, x, y);
        const int q = entry_owner(F, k, x, y);
        if (q < 0 || q == p) continue;
        const int lq = __ldg(F.level + q);
        const int rel_pass = lq > lp ? 0 : (lq == lp ? 1 : 2);
        if (rel_pass != pass || !((src >> lq) & 1u)) continue;
        if ((flags & AF_FILL_SAME_LEVEL_ONLY) && lq != lp) continue;
        double v[3];
        transfer_all<T>(F, S, lp, q, k, x, y, S.ncomp, v);
        for (int c = 0; c < S.ncomp; ++c) *S.at(p, c, k, i, j) = (T)v[c];
    }
}

// ---------------------------------------------------------------------------
// Ghost plan: the owner of every ghost entry resolved once per forest, so an
// exchange is two flat passes over a list instead of per-entry searches.
// Pass A (kinds copy / mean of four finer averages) writes only entries the
// destination does not own and reads only owned ones, so its entries are
// independent; among them are the boundary-line point values of every leaf
// with a coarser-or-finer neighbour.  Pass B (coarse -> fine) then reads the
// coarse leaf's whole cell -- boundary-line nodes included -- from that
// leaf's own lattice, which pass A has just made current.
struct GhostEntry {
    int32_t dst, src;
    uint16_t dst_off;  // plane * plane_stride + lattice index (component 0)
    uint8_t kind, levels;  // levels: dst level | src level << 4
    uint32_t aux;      // kinds 0, 1: source offset; kinds 2, 3: u | v << 16 (quarter cells of the source)
};
static_assert(sizeof(GhostEntry) == AF_GHOST_ENTRY_BYTES, "ghost plan entry layout");
enum : uint8_t { kGCopy = 0, kGMean4 = 1, kGPoint = 2, kGSimpson = 3 };

// Classify ghost entry (k, i, j) of leaf p; false if it is not exchanged.
__device__ bool ghost_entry(const DevForest &F, int64_t plane, int p, int lp, int k, int i, int j, GhostEntry &g) {
    const int n = F.n, W = n + 2 * kGhost + 1;
    if (i > 0 && i < n && j > 0 && j < n) return false;
    if (i == n + kGhost && (k == kAvg || k == kYmid)) return false;
    if (j == n + kGhost && (k == kAvg || k == kXmid)) return false;
    long long x, y;
    entry_xy(F, p, k, i, j, x, y);
    const int q = entry_owner(F, k, x, y);
    if (q < 0 || q == p) return false;
    const int lq = __ldg(F.level + q);
    g.dst = p;
    g.src = q;
    g.dst_off = (uint16_t)(k * plane + (int64_t)(j + kGhost) * W + (i + kGhost));
    g.levels = (uint8_t)(lp | (lq << 4));
    int si, sj;
    if (lq == lp) {
        lattice_of(F, q, k, x, y, si, sj);
        g.kind = kGCopy;
        g.aux = (uint32_t)(k * plane + (int64_t)(sj + kGhost) * W + (si + kGhost));
    } else if (lq > lp) {
        if (k == kAvg) {
            const long long h = hwid(F, lq) / 2;  // the four finer cells: (si, sj) .. (si + 1, sj + 1)
            lattice_of(F, q, kAvg, x - h, y - h, si, sj);
            g.kind = kGMean4;
            g.aux = (uint32_t)(kAvg * plane + (int64_t)(sj + kGhost) * W + (si + kGhost));
        } else {
            lattice_of(F, q, kCorner, x, y, si, sj);
            g.kind = kGCopy;
            g.aux = (uint32_t)(kCorner * plane + (int64_t)(sj + kGhost) * W + (si + kGhost));
        }
    } else {
        const long long quarter = hwid(F, lq) / 4;
        long long u = reld(F, x, leaf_x0(F, q)) / quarter, v = reld(F, y, leaf_y0(F, q)) / quarter;
        u = u < 0 ? 0 : (u > 4 * n ? 4 * n : u);
        v = v < 0 ? 0 : (v > 4 * n ? 4 * n : v);
        g.kind = k == kAvg ? kGSimpson : kGPoint;
        g.aux = (uint32_t)u | ((uint32_t)v << 16);
    }
    return true;
}

__device__ __forceinline__ bool plan_leaf(const DevForest &F, int p, int flags) {
    return (flags & AF_FILL_ALL_PATCHES) || has_other_level_neighbour(F, p);
}

// counts[0]: pass-A entries, counts[1]: pass-B entries.
__global__ void plan_count_kernel(DevForest F, int64_t plane, int flags, unsigned long long *counts) {
    const int p = blockIdx.x;
    __shared__ int s_use;
    __shared__ unsigned int s_cnt[2];
    if (threadIdx.x == 0) {
        s_use = plan_leaf(F, p, flags);
        s_cnt[0] = s_cnt[1] = 0;
    }
    __syncthreads();
    if (!s_use) return;
    const int lp = __ldg(F.level + p), W = F.n + 2 * kGhost + 1;
    for (int e = threadIdx.x; e < kPlanes * W * W; e += blockDim.x) {
        const int k = e / (W * W), r = e - k * W * W;
        GhostEntry g;
        if (ghost_entry(F, plane, p, lp, k, r % W - kGhost, r / W - kGhost, g)) atomicAdd(&s_cnt[g.kind >= kGPoint], 1u);
    }
    __syncthreads();
    if (threadIdx.x < 2 && s_cnt[threadIdx.x]) atomicAdd(counts + threadIdx.x, (unsigned long long)s_cnt[threadIdx.x]);
}

// Pass-A entries fill [0, na), pass-B entries [na, na + nb); cursor[2] starts at 0.
// Each leaf reserves one contiguous range per pass and writes its entries
// there in lattice order (plane, row, column), so the threads of an
// executing warp touch consecutive destination entries (and, for copies,
// consecutive source entries): the exchange's accesses coalesce.  The order
// of the leaves' ranges is whatever order the CTAs reserve them in; each
// destination entry appears once, so the order does not change the result.
__global__ void plan_build_kernel(DevForest F, int64_t plane, int flags, GhostEntry *plan, long long na, long long nb,
                                  unsigned long long *cursor, int *overflow) {
    const int p = blockIdx.x;
    __shared__ int s_use;
    __shared__ unsigned int s_cnt[2];
    __shared__ unsigned long long s_base[2];
    __shared__ unsigned int s_warp[2][32];
    if (threadIdx.x == 0) {
        s_use = plan_leaf(F, p, flags);
        s_cnt[0] = s_cnt[1] = 0;
    }
    __syncthreads();
    if (!s_use) return;
    const int lp = __ldg(F.level + p), W = F.n + 2 * kGhost + 1;
    const int total = kPlanes * W * W;
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        const int k = e / (W * W), r = e - k * W * W;
        GhostEntry g;
        if (ghost_entry(F, plane, p, lp, k, r % W - kGhost, r / W - kGhost, g)) atomicAdd(&s_cnt[g.kind >= kGPoint], 1u);
    }
    __syncthreads();
    if (threadIdx.x < 2) s_base[threadIdx.x] = s_cnt[threadIdx.x] ? atomicAdd(cursor + threadIdx.x, s_cnt[threadIdx.x]) : 0ull;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = (blockDim.x + 31) >> 5;
    const unsigned below = (1u << lane) - 1u;
    unsigned long long run0 = s_base[0], run1 = s_base[1];
    for (int e0 = 0; e0 < total; e0 += blockDim.x) {
        const int e = e0 + threadIdx.x;
        GhostEntry g;
        bool v = false;
        if (e < total) {
            const int k = e / (W * W), r = e - k * W * W;
            v = ghost_entry(F, plane, p, lp, k, r % W - kGhost, r / W - kGhost, g);
        }
        const int b = v ? (g.kind >= kGPoint) : 0;
        const unsigned m0 = __ballot_sync(0xffffffffu, v && b == 0), m1 = __ballot_sync(0xffffffffu, v && b == 1);
        if (lane == 0) {
            s_warp[0][warp] = __popc(m0);
            s_warp[1][warp] = __popc(m1);
        }
        __syncthreads();
        unsigned off0 = 0, off1 = 0, tot0 = 0, tot1 = 0;
        for (int w = 0; w < nwarp; ++w) {
            if (w < warp) {
                off0 += s_warp[0][w];
                off1 += s_warp[1][w];
            }
            tot0 += s_warp[0][w];
            tot1 += s_warp[1][w];
        }
        if (v) {
            const unsigned long long slot = b ? run1 + off1 + __popc(m1 & below) : run0 + off0 + __popc(m0 & below);
            if ((long long)slot >= (b ? nb : na)) {
                atomicExch(overflow, 1);
            } else {
                plan[(b ? na : 0) + (long long)slot] = g;
            }
        }
        run0 += tot0;
        run1 += tot1;
        __syncthreads();
    }
}

template <typename T>
__global__ void plan_exec_a(StateView<T> S, const GhostEntry *__restrict__ plan, long long na, uint32_t levels,
                            int same_only) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < na; t += (long long)gridDim.x * blockDim.x) {
        const GhostEntry g = plan[t];
        const int ld = g.levels & 15, ls = g.levels >> 4;
        if (!((levels >> ld) & 1u) || !((levels >> ls) & 1u) || (same_only && ld != ls)) continue;
        const T *src = S.patch_at_level(g.src, ls) + g.aux;
        T *dst = S.patch_at_level(g.dst, ld) + g.dst_off;
        const int64_t cs = (int64_t)kPlanes * S.plane;
        for (int c = 0; c < S.ncomp; ++c) {
            if (g.kind == kGCopy) {
                dst[c * cs] = src[c * cs];
            } else {
                const T *a = src + c * cs;
                const double sum = (double)a[0] + (double)a[1] + (double)a[S.W] + (double)a[S.W + 1];
                dst[c * cs] = (T)(0.25 * sum);
            }
        }
    }
}

template <typename T>
__global__ void plan_exec_b(StateView<T> S, int n, const GhostEntry *__restrict__ plan, long long nb, uint32_t levels) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nb; t += (long long)gridDim.x * blockDim.x) {
        const GhostEntry g = plan[t];
        const int ld = g.levels & 15, ls = g.levels >> 4;
        if (!((levels >> ld) & 1u) || !((levels >> ls) & 1u)) continue;
        const T *q = S.patch_at_level(g.src, ls);
        T *dst = S.patch_at_level(g.dst, ld) + g.dst_off;
        const int u0 = (int)(g.aux & 0xffffu), v0 = (int)(g.aux >> 16);
        const int64_t cs = (int64_t)kPlanes * S.plane;
        const int W = S.W;
        // value at quarter-cell position (u, v) of the source leaf, with the
        // cell chosen as the direct exchange chooses it
        // quarter: the mean over the quarter of the cell holding (u, v) that
        // (u, v), the centre of a cell one level finer, lies in
        auto at = [&](const T *b, int u, int v, bool quarter) -> T {
            int ci = u / 4, cj = v / 4;
            ci = ci > n - 1 ? n - 1 : ci;
            cj = cj > n - 1 ? n - 1 : cj;
            const T xi = (T)(0.5 * (double)(u - 4 * ci) - 1.0), eta = (T)(0.5 * (double)(v - 4 * cj) - 1.0);
            const T *cr = b + kCorner * S.plane + (int64_t)(cj + kGhost) * W + (ci + kGhost);
            const T *xm = b + kXmid * S.plane + (int64_t)(cj + kGhost) * W + (ci + kGhost);
            const T *ym = b + kYmid * S.plane + (int64_t)(cj + kGhost) * W + (ci + kGhost);
            const T *av = b + kAvg * S.plane + (int64_t)(cj + kGhost) * W + (ci + kGhost);
            if (quarter)
                return recon_quarter_mean<T>(cr[0], cr[1], cr[W], cr[W + 1], xm[0], xm[1], ym[0], ym[W], av[0],
                                             u - 4 * ci >= 2, v - 4 * cj >= 2);
            return recon_eval<T>(cr[0], cr[1], cr[W], cr[W + 1], xm[0], xm[1], ym[0], ym[W], av[0], xi, eta);
        };
        for (int c = 0; c < S.ncomp; ++c) {
            const T *b = q + c * cs;
            dst[c * cs] = at(b, u0, v0, g.kind != kGPoint);
        }
    }
}

template <typename T>
__global__ void transfer_kernel(DevForest Fo, StateView<T> So, DevForest Fn, StateView<T> Sn) {
    const int p = blockIdx.x;
    const int l = __ldg(Fn.level + p), px = __ldg(Fn.ix + p), py = __ldg(Fn.iy + p);
    const int64_t words = (int64_t)Sn.ncomp * kPlanes * Sn.plane;
    T *dst = Sn.patch(p);
    int same = -1;
    if (l <= Fo.lmax) {
        const long long side = (long long)Fo.B << l;
        same = __ldg(Fo.map + map_offset(Fo.B, l) + (long long)py * side + px);
    }
    const int n = Fn.n, m = n + 1;
    const long long hwn = 2LL << (Fn.lmax - l);
    const long long x0 = (long long)px * n * hwn, y0 = (long long)py * n * hwn;
    if (same >= 0) {
        const T *srcp = So.patch(same);
        constexpr int V = 16 / (int)sizeof(T);  // elements per 16-byte load
        if (words % V == 0 && ((reinterpret_cast<uintptr_t>(srcp) | reinterpret_cast<uintptr_t>(dst)) & 15u) == 0) {
            const int4 *s4 = reinterpret_cast<const int4 *>(srcp);
            int4 *d4 = reinterpret_cast<int4 *>(dst);
            for (int64_t e = threadIdx.x; e < words / V; e += blockDim.x) d4[e] = __ldg(s4 + e);
        } else {
            for (int64_t e = threadIdx.x; e < words; e += blockDim.x) dst[e] = srcp[e];
        }
        __syncthreads();
        // The point values on the right (i = n) and top (j = n) faces: where the
        // neighbour across was the owner in the old forest (same level, or
        // finer) the leaf's own copy is not kept current -- a step of a leaf
        // with eight same-level neighbours stores node lines 0 .. n-1 only --
        // yet the leaf owns them in the new forest if that neighbour became
        // coarser.  Take them from their old owner.
        for (int e = threadIdx.x; e < 4 * m; e += blockDim.x) {
            const int side = e / m, r = e - side * m;  // 0, 1: corner / left-mid on line i = n; 2, 3: on j = n
            const int k = side == 0 || side == 2 ? kCorner : (side == 1 ? kXmid : kYmid);
            const int i = side < 2 ? n : r, j = side < 2 ? r : n;
            if ((k == kXmid && j == n) || (k == kYmid && i == n)) continue;
            const long long x = x0 + (long long)i * hwn + (k == kYmid ? hwn / 2 : 0);
            const long long y = y0 + (long long)j * hwn + (k == kXmid ? hwn / 2 : 0);
            const int q = entry_owner(Fo, k, x, y);
            if (q < 0 || q == same) continue;
            double v[3];
            transfer_all<T>(Fo, So, l, q, k, x, y, Sn.ncomp, v);
            for (int c = 0; c < Sn.ncomp; ++c) *Sn.at(p, c, k, i, j) = (T)v[c];
        }
        return;
    }
    for (int64_t e = threadIdx.x; e < words; e += blockDim.x) dst[e] = T(0);
    __syncthreads();
    // The cells' averages and the point values on their boundaries: node
    // lines 0 .. n, the right (i = n) and top (j = n) lines included -- a leaf
    // finer than its neighbour across that face owns those nodes (the finer
    // grid's values are used at coarse-fine faces), and nothing else writes
    // them.  Entries owned by another leaf are overwritten by the exchange
    // that follows a regrid.
    for (int e = threadIdx.x; e < kPlanes * m * m; e += blockDim.x) {
        const int k = e / (m * m), r = e - k * m * m, j = r / m, i = r - j * m;
        if ((i == n && (k == kAvg || k == kYmid)) || (j == n && (k == kAvg || k == kXmid))) continue;
        const long long x = x0 + (long long)i * hwn + ((k == kAvg || k == kYmid) ? hwn / 2 : 0);
        const long long y = y0 + (long long)j * hwn + ((k == kAvg || k == kXmid) ? hwn / 2 : 0);
        const int q = entry_owner(Fo, k, x, y);
        if (q < 0) continue;
        // an average comes from at most one level finer (the four children's
        // mean); a point value is the coinciding vertex of any finer owner
        if (k == kAvg && __ldg(Fo.level + q) > l + 1) continue;
        double v[3];
        transfer_all<T>(Fo, So, l, q, k, x, y, Sn.ncomp, v);
        for (int c = 0; c < Sn.ncomp; ++c) *Sn.at(p, c, k, i, j) = (T)v[c];
    }
}

template <typename T>
__device__ __forceinline__ void atomic_add_state(T *p, double v);
template <>
__device__ __forceinline__ void atomic_add_state<double>(double *p, double v) { atomicAdd(p, v); }
template <>
__device__ __forceinline__ void atomic_add_state<float>(float *p, double v) { atomicAdd(p, (float)v); }

template <typename T>
__global__ void reflux_kernel(DevForest F, StateView<T> S, uint32_t sync, double dx0, double dy0, double *freg) {
    const int n = F.n, nc = S.ncomp;
    const int64_t total = (int64_t)F.nleaf * 4 * n;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int p = (int)(t / (4 * n)), side = (int)((t / n) % 4), k = (int)(t % n);
        const int l = __ldg(F.level + p);
        if (l >= AF_MAX_LEVEL || !((sync >> l) & 1u) || !((sync >> (l + 1)) & 1u)) continue;
        const long long hw = hwid(F, l), x0 = leaf_x0(F, p), y0 = leaf_y0(F, p);
        const long long x1 = x0 + (long long)n * hw, y1 = y0 + (long long)n * hw;
        long long px, py;
        if (side == 0) { px = x0 - 1; py = y0 + k * hw + hw / 2; }
        else if (side == 1) { px = x1; py = y0 + k * hw + hw / 2; }
        else if (side == 2) { px = x0 + k * hw + hw / 2; py = y0 - 1; }
        else { px = x0 + k * hw + hw / 2; py = y1; }
        const int q = lookup(F, px, py);
        if (q < 0 || __ldg(F.level + q) != l + 1) continue;
        const long long hf = hwid(F, l + 1);
        const int fside = side ^ 1;
        const long long start = side < 2 ? reld(F, y0 + k * hw, leaf_y0(F, q)) : reld(F, x0 + k * hw, leaf_x0(F, q));
        const int kf = (int)(start / hf);
        if (kf < 0 || kf + 1 >= n) continue;
        const int ci = side == 0 ? 0 : (side == 1 ? n - 1 : k);
        const int cj = side == 2 ? 0 : (side == 3 ? n - 1 : k);
        const double h = (side < 2 ? dx0 : dy0) / (double)(1LL << l);
        const int64_t rw = 4LL * nc * n;
        for (int c = 0; c < nc; ++c) {
            double *rc = freg + p * rw + ((int64_t)side * nc + c) * n + k;
            double *rf = freg + q * rw + ((int64_t)fside * nc + c) * n + kf;
            const double fine = 0.5 * (rf[0] + rf[1]);
            const double d = (side == 1 || side == 3) ? (*rc - fine) / h : (fine - *rc) / h;
            atomic_add_state<T>(S.at(p, c, kAvg, ci, cj), d);
            *rc = 0.0;
            rf[0] = 0.0;
            rf[1] = 0.0;
        }
    }
}

template <typename T>
__global__ void tag_kernel(DevForest F, StateView<T> S, int comp, int kind, double dx0, double dy0, double rthr,
                           double cthr, int8_t *tags, double *ind) {
    const int p = blockIdx.x, n = F.n;
    const int l = __ldg(F.level + p);
    const double hx = dx0 / (double)(1LL << l), hy = dy0 / (double)(1LL << l);
    double a = -INFINITY, b = INFINITY;  // kind 0: max, min; kind 1: max gradient in a
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int j = e / n, i = e % n;
        if (kind == 0) {
            const double q = *S.at(p, comp, kAvg, i, j);
            a = fmax(a, q);
            b = fmin(b, q);
        } else if (i >= 1 && i < n - 1 && j >= 1 && j < n - 1) {
            const double gx = fabs((double)*S.at(p, comp, kAvg, i + 1, j) - (double)*S.at(p, comp, kAvg, i - 1, j)) / (2.0 * hx);
            const double gy = fabs((double)*S.at(p, comp, kAvg, i, j + 1) - (double)*S.at(p, comp, kAvg, i, j - 1)) / (2.0 * hy);
            a = fmax(a, fmax(gx, gy));
        }
    }
    __shared__ double sa[256], sb[256];
    sa[threadIdx.x] = a;
    sb[threadIdx.x] = b;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            sa[threadIdx.x] = fmax(sa[threadIdx.x], sa[threadIdx.x + s]);
            sb[threadIdx.x] = fmin(sb[threadIdx.x], sb[threadIdx.x + s]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double v = kind == 0 ? sa[0] - sb[0] : fmax(sa[0], 0.0);
        if (ind) ind[p] = v;
        tags[p] = (int8_t)(v >= rthr ? 1 : (v < cthr ? -1 : 0));
    }
}

constexpr int kMassBlocks = 256;
constexpr int kMassThreads = 256;

// Pass 1: block b sums leaves [b * chunk, (b+1) * chunk) in a fixed order.
template <typename T>
__global__ void mass_partial(DevForest F, StateView<T> S, double dx0, double dy0, int chunk, double *part) {
    const int n = F.n, nc = S.ncomp;
    __shared__ double sm[kMassThreads];
    for (int c = 0; c < nc; ++c) {
        double acc = 0.0;
        const int p0 = blockIdx.x * chunk, p1 = min(F.nleaf, p0 + chunk);
        for (int p = p0; p < p1; ++p) {
            const int l = __ldg(F.level + p);
            const double area = (dx0 / (double)(1LL << l)) * (dy0 / (double)(1LL << l));
            double s = 0.0;
            for (int e = threadIdx.x; e < n * n; e += blockDim.x) s += (double)*S.at(p, c, kAvg, e % n, e / n);
            acc += s * area;
        }
        sm[threadIdx.x] = acc;
        __syncthreads();
        for (int s = blockDim.x / 2; s > 0; s >>= 1) {
            if ((int)threadIdx.x < s) sm[threadIdx.x] += sm[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) part[blockIdx.x * nc + c] = sm[0];
        __syncthreads();
    }
}

__global__ void mass_final(const double *part, int nblocks, int nc, double *out) {
    __shared__ double sm[kMassThreads];
    for (int c = 0; c < nc; ++c) {
        double acc = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += blockDim.x) acc += part[b * nc + c];
        sm[threadIdx.x] = acc;
        __syncthreads();
        for (int s = blockDim.x / 2; s > 0; s >>= 1) {
            if ((int)threadIdx.x < s) sm[threadIdx.x] += sm[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[c] = sm[0];
        __syncthreads();
    }
}

bool check_cfg(const af_config *cfg) {
    return cfg && cfg->n >= 2 && cfg->n <= 64 && (cfg->eq == AF_ADVECTION || cfg->eq == AF_ACOUSTICS) &&
           (cfg->prec == AF_F64 || cfg->prec == AF_F32) && cfg->ncomp == (cfg->eq == AF_ADVECTION ? 1 : 3);
}

bool check_forest(const af_forest *f) {
    return f && f->nleaf >= 0 && f->B >= 1 && f->lmax >= 0 && f->lmax <= AF_MAX_LEVEL &&
           (f->nleaf == 0 || (f->d_level && f->d_ix && f->d_iy && f->d_map));
}

template <typename T>
StateView<T> view(const af_config &cfg, const af_forest &f, const af_state_pair &st) {
    StateView<T> s;
    s.base0 = static_cast<T *>(st.buf[0]);
    s.base1 = static_cast<T *>(st.buf[1]);
    s.level = f.d_level;
    s.parity = st.parity;
    s.plane = plane_stride(cfg.n);
    s.ncomp = cfg.ncomp;
    s.W = cfg.n + 2 * kGhost + 1;
    return s;
}

af_state_pair single(const void *d_state) {
    af_state_pair p;
    p.buf[0] = p.buf[1] = const_cast<void *>(d_state);
    p.parity = 0u;
    p.pad_ = 0u;
    return p;
}

// A pair is usable if its current arrays exist and are aligned; a pair whose
// parity is zero may leave buf[1] NULL.
af_status check_pair(const af_state_pair *st) {
    if (!st || !st->buf[0] || (st->parity != 0u && !st->buf[1])) return AF_ERR_ARG;
    if ((reinterpret_cast<uintptr_t>(st->buf[0]) | reinterpret_cast<uintptr_t>(st->buf[1])) & 31u)
        return AF_ERR_LAYOUT;
    return AF_OK;
}

inline af_status launched() { return cudaGetLastError() == cudaSuccess ? AF_OK : AF_ERR_CUDA; }

int mass_blocks(int nleaf) { return nleaf < kMassBlocks ? (nleaf < 1 ? 1 : nleaf) : kMassBlocks; }

}  // namespace
}  // namespace af

using namespace af;

extern "C" int64_t af_forest_map_offset(int32_t B, int32_t level) {
    if (B < 1 || level < 0 || level > AF_MAX_LEVEL + 1) return -1;
    return map_offset(B, level);
}

extern "C" af_status af_forest_build_map(int32_t nleaf, int32_t B, int32_t lmax, const int32_t *h_level,
                                         const int32_t *h_ix, const int32_t *h_iy, int32_t *h_map) {
    if (nleaf < 0 || B < 1 || lmax < 0 || lmax > AF_MAX_LEVEL || !h_map) return AF_ERR_ARG;
    if (nleaf > 0 && (!h_level || !h_ix || !h_iy)) return AF_ERR_ARG;
    const long long total = map_offset(B, lmax + 1);
    for (long long e = 0; e < total; ++e) h_map[e] = -1;
    for (int p = 0; p < nleaf; ++p) {
        const int l = h_level[p];
        if (l < 0 || l > lmax) return AF_ERR_ARG;
        const long long side = (long long)B << l;
        if (h_ix[p] < 0 || h_ix[p] >= side || h_iy[p] < 0 || h_iy[p] >= side) return AF_ERR_ARG;
        int32_t &slot = h_map[map_offset(B, l) + (long long)h_iy[p] * side + h_ix[p]];
        if (slot >= 0) return AF_ERR_ARG;
        slot = p;
    }
    // regions inside a leaf, at every finer level: -2 - (the leaf)
    for (int p = 0; p < nleaf; ++p) {
        const int l = h_level[p];
        for (int m = l + 1; m <= lmax; ++m) {
            const long long side = (long long)B << m, w = 1LL << (m - l);
            const long long x0 = (long long)h_ix[p] * w, y0 = (long long)h_iy[p] * w;
            int32_t *row = h_map + map_offset(B, m);
            for (long long y = y0; y < y0 + w; ++y)
                for (long long x = x0; x < x0 + w; ++x) {
                    int32_t &slot = row[y * side + x];
                    if (slot != -1) return AF_ERR_ARG;  // overlapping leaves
                    slot = -2 - p;
                }
        }
    }
    return AF_OK;
}

extern "C" af_status af_fill_ghosts_pair(const af_config *cfg, const af_forest *forest, uint32_t dst_levels,
                                         uint32_t src_levels, int32_t flags, const af_state_pair *state,
                                         void *stream) {
    if (!check_cfg(cfg) || !check_forest(forest)) return AF_ERR_ARG;
    if (forest->nleaf == 0) return AF_OK;
    if (const af_status e = check_pair(state)) return e;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const DevForest F = make_dev(*forest, cfg->n);
    for (int pass = 0; pass < 3; ++pass) {
        if ((flags & AF_FILL_SAME_LEVEL_ONLY) && pass != 1) continue;
        if (cfg->prec == AF_F64)
            fill_kernel<double><<<forest->nleaf, 256, 0, s>>>(F, view<double>(*cfg, *forest, *state), dst_levels,
                                                              src_levels, flags, pass);
        else
            fill_kernel<float><<<forest->nleaf, 256, 0, s>>>(F, view<float>(*cfg, *forest, *state), dst_levels,
                                                             src_levels, flags, pass);
        if (launched() != AF_OK) return AF_ERR_CUDA;
    }
    return AF_OK;
}

extern "C" af_status af_fill_ghosts(const af_config *cfg, const af_forest *forest, uint32_t dst_levels,
                                    uint32_t src_levels, int32_t flags, void *d_state, void *stream) {
    const af_state_pair st = single(d_state);
    return af_fill_ghosts_pair(cfg, forest, dst_levels, src_levels, flags, &st, stream);
}

// Upward-closed level set: with its lowest level it holds every level up to lmax.
static bool upward_closed(uint32_t levels, int lmax) {
    if (levels == 0u) return true;
    const int lo = __builtin_ctz(levels);
    const uint32_t want = (lmax >= 31 ? 0xffffffffu : ((1u << (lmax + 1)) - 1u)) & ~((1u << lo) - 1u);
    return (levels & want) == want;
}

extern "C" af_status af_ghost_plan_count(const af_config *cfg, const af_forest *forest, int32_t flags,
                                         int64_t *d_counts, void *stream) {
    if (!check_cfg(cfg) || !check_forest(forest) || !d_counts) return AF_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(d_counts) & 7u) return AF_ERR_LAYOUT;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(d_counts, 0, 2 * sizeof(int64_t), s) != cudaSuccess) return AF_ERR_CUDA;
    if (forest->nleaf == 0) return AF_OK;
    plan_count_kernel<<<forest->nleaf, 256, 0, s>>>(make_dev(*forest, cfg->n), plane_stride(cfg->n), flags,
                                                     reinterpret_cast<unsigned long long *>(d_counts));
    return launched();
}

extern "C" af_status af_ghost_plan_build(const af_config *cfg, const af_forest *forest, int32_t flags, void *d_plan,
                                         int64_t n_a, int64_t n_b, int64_t *d_scratch, void *stream) {
    if (!check_cfg(cfg) || !check_forest(forest) || !d_scratch || n_a < 0 || n_b < 0) return AF_ERR_ARG;
    if (n_a + n_b > 0 && !d_plan) return AF_ERR_ARG;
    if ((reinterpret_cast<uintptr_t>(d_plan) | reinterpret_cast<uintptr_t>(d_scratch)) & 15u) return AF_ERR_LAYOUT;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // scratch: two slot cursors and an overflow flag
    if (cudaMemsetAsync(d_scratch, 0, 3 * sizeof(int64_t), s) != cudaSuccess) return AF_ERR_CUDA;
    if (forest->nleaf == 0) return AF_OK;
    plan_build_kernel<<<forest->nleaf, 256, 0, s>>>(
        make_dev(*forest, cfg->n), plane_stride(cfg->n), flags, static_cast<GhostEntry *>(d_plan), n_a, n_b,
        reinterpret_cast<unsigned long long *>(d_scratch), reinterpret_cast<int *>(d_scratch + 2));
    return launched();
}

extern "C" af_status af_fill_ghosts_planned(const af_config *cfg, const af_forest *forest, uint32_t levels,
                                            int32_t flags, const void *d_plan, int64_t n_a, int64_t n_b,
                                            const af_state_pair *state, void *stream) {
    if (!check_cfg(cfg) || !check_forest(forest) || n_a < 0 || n_b < 0) return AF_ERR_ARG;
    if (!upward_closed(levels, forest->lmax)) return AF_ERR_ARG;
    if (n_a + n_b == 0 || levels == 0u) return AF_OK;
    if (!d_plan) return AF_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(d_plan) & 15u) return AF_ERR_LAYOUT;
    if (const af_status e = check_pair(state)) return e;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const GhostEntry *plan = static_cast<const GhostEntry *>(d_plan);
    const int same = (flags & AF_FILL_SAME_LEVEL_ONLY) ? 1 : 0;
    auto grid = [](int64_t m) { return (int)(m / 256 + 1 < 152 * 16 ? m / 256 + 1 : 152 * 16); };
    if (n_a > 0) {
        if (cfg->prec == AF_F64)
            plan_exec_a<double><<<grid(n_a), 256, 0, s>>>(view<double>(*cfg, *forest, *state), plan, n_a, levels, same);
        else
            plan_exec_a<float><<<grid(n_a), 256, 0, s>>>(view<float>(*cfg, *forest, *state), plan, n_a, levels, same);
        if (launched() != AF_OK) return AF_ERR_CUDA;
    }
    if (n_b > 0 && !same) {
        if (cfg->prec == AF_F64)
            plan_exec_b<double><<<grid(n_b), 256, 0, s>>>(view<double>(*cfg, *forest, *state), cfg->n, plan + n_a, n_b,
                                                         levels);
        else
            plan_exec_b<float><<<grid(n_b), 256, 0, s>>>(view<float>(*cfg, *forest, *state), cfg->n, plan + n_a, n_b,
                                                        levels);
        if (launched() != AF_OK) return AF_ERR_CUDA;
    }
    return AF_OK;
}

extern "C" af_status af_transfer_pair(const af_config *cfg, const af_forest *old_forest,
                                      const af_state_pair *old_state, const af_forest *new_forest, void *d_new,
                                      void *stream) {
    if (!check_cfg(cfg) || !check_forest(old_forest) || !check_forest(new_forest)) return AF_ERR_ARG;
    if (old_forest->B != new_forest->B || old_forest->lmax != new_forest->lmax) return AF_ERR_ARG;
    if (new_forest->nleaf == 0) return AF_OK;
    if (const af_status e = check_pair(old_state)) return e;
    if (!d_new || d_new == old_state->buf[0] || d_new == old_state->buf[1]) return AF_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(d_new) & 31u) return AF_ERR_LAYOUT;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const DevForest Fo = make_dev(*old_forest, cfg->n), Fn = make_dev(*new_forest, cfg->n);
    const af_state_pair sn = single(d_new);
    if (cfg->prec == AF_F64)
        transfer_kernel<double><<<new_forest->nleaf, 256, 0, s>>>(Fo, view<double>(*cfg, *old_forest, *old_state), Fn,
                                                                 view<double>(*cfg, *new_forest, sn));
    else
        transfer_kernel<float><<<new_forest->nleaf, 256, 0, s>>>(Fo, view<float>(*cfg, *old_forest, *old_state), Fn,
                                                                view<float>(*cfg, *new_forest, sn));
    return launched();
}

extern "C" af_status af_transfer(const af_config *cfg, const af_forest *old_forest, const void *d_old,
                                 const af_forest *new_forest, void *d_new, void *stream) {
    if (!d_old) return AF_ERR_ARG;
    const af_state_pair so = single(d_old);
    return af_transfer_pair(cfg, old_forest, &so, new_forest, d_new, stream);
}

extern "C" af_status af_reflux_pair(const af_config *cfg, const af_forest *forest, uint32_t sync_levels, double dx0,
                                    double dy0, double *d_flux_reg, const af_state_pair *state, void *stream) {
    if (!check_cfg(cfg) || !check_forest(forest)) return AF_ERR_ARG;
    if (!(dx0 > 0.0) || !(dy0 > 0.0)) return AF_ERR_ARG;
    if (forest->nleaf == 0) return AF_OK;
    if (!d_flux_reg) return AF_ERR_ARG;
    if (const af_status e = check_pair(state)) return e;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const DevForest F = make_dev(*forest, cfg->n);
    const long long total = (long long)forest->nleaf * 4 * cfg->n;
    const int blocks = (int)((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096);
    if (cfg->prec == AF_F64)
        reflux_kernel<double><<<blocks, 256, 0, s>>>(F, view<double>(*cfg, *forest, *state), sync_levels, dx0, dy0,
                                                     d_flux_reg);
    else
        reflux_kernel<float><<<blocks, 256, 0, s>>>(F, view<float>(*cfg, *forest, *state), sync_levels, dx0, dy0,
                                                    d_flux_reg);
    return launched();
}

extern "C" af_status af_reflux(const af_config *cfg, const af_forest *forest, uint32_t sync_levels, double dx0,
                               double dy0, double *d_flux_reg, void *d_state, void *stream) {
    const af_state_pair st = single(d_state);
    return af_reflux_pair(cfg, forest, sync_levels, dx0, dy0, d_flux_reg, &st, stream);
}

extern "C" af_status af_tag_pair(const af_config *cfg, const af_forest *forest, const af_state_pair *state,
                                 int32_t comp, int32_t kind, double dx0, double dy0, double refine_thr,
                                 double coarsen_thr, int8_t *d_tags, double *d_indicator, void *stream) {
    if (!check_cfg(cfg) || !check_forest(forest)) return AF_ERR_ARG;
    if (comp < 0 || comp >= cfg->ncomp || (kind != 0 && kind != 1)) return AF_ERR_ARG;
    if (!(dx0 > 0.0) || !(dy0 > 0.0)) return AF_ERR_ARG;
    if (forest->nleaf == 0) return AF_OK;
    if (!d_tags) return AF_ERR_ARG;
    if (const af_status e = check_pair(state)) return e;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const DevForest F = make_dev(*forest, cfg->n);
    if (cfg->prec == AF_F64)
        tag_kernel<double><<<forest->nleaf, 256, 0, s>>>(F, view<double>(*cfg, *forest, *state), comp, kind, dx0, dy0,
                                                        refine_thr, coarsen_thr, d_tags, d_indicator);
    else
        tag_kernel<float><<<forest->nleaf, 256, 0, s>>>(F, view<float>(*cfg, *forest, *state), comp, kind, dx0, dy0,
                                                       refine_thr, coarsen_thr, d_tags, d_indicator);
    return launched();
}

extern "C" af_status af_tag(const af_config *cfg, const af_forest *forest, const void *d_state, int32_t comp,
                            int32_t kind, double dx0, double dy0, double refine_thr, double coarsen_thr,
                            int8_t *d_tags, double *d_indicator, void *stream) {
    const af_state_pair st = single(d_state);
    return af_tag_pair(cfg, forest, &st, comp, kind, dx0, dy0, refine_thr, coarsen_thr, d_tags, d_indicator, stream);
}

extern "C" int64_t af_mass_scratch_bytes(int32_t nleaf, int32_t ncomp) {
    if (nleaf < 0 || ncomp < 1) return 0;
    return (int64_t)mass_blocks(nleaf) * ncomp * (int64_t)sizeof(double);
}

namespace af {
namespace {
// Both passes of the deterministic mass reduction into `part`.
af_status launch_mass(const af_config &cfg, const af_forest &forest, const af_state_pair &st, double dx0, double dy0,
                      double *part, double *d_mass, cudaStream_t s) {
    const DevForest F = make_dev(forest, cfg.n);
    const int nb = mass_blocks(forest.nleaf);
    const int chunk = (forest.nleaf + nb - 1) / nb;
    if (cfg.prec == AF_F64)
        mass_partial<double><<<nb, kMassThreads, 0, s>>>(F, view<double>(cfg, forest, st), dx0, dy0, chunk, part);
    else
        mass_partial<float><<<nb, kMassThreads, 0, s>>>(F, view<float>(cfg, forest, st), dx0, dy0, chunk, part);
    if (launched() != AF_OK) return AF_ERR_CUDA;
    mass_final<<<1, kMassThreads, 0, s>>>(part, nb, cfg.ncomp, d_mass);
    return launched();
}
}  // namespace
}  // namespace af

extern "C" af_status af_mass_pair(const af_config *cfg, const af_forest *forest, const af_state_pair *state,
                                  double dx0, double dy0, void *d_scratch, double *d_mass, void *stream) {
    if (!check_cfg(cfg) || !check_forest(forest)) return AF_ERR_ARG;
    if (!(dx0 > 0.0) || !(dy0 > 0.0) || !d_mass || !d_scratch) return AF_ERR_ARG;
    if ((reinterpret_cast<uintptr_t>(d_scratch) | reinterpret_cast<uintptr_t>(d_mass)) & 7u) return AF_ERR_LAYOUT;
    if (forest->nleaf > 0)
        if (const af_status e = check_pair(state)) return e;
    af_state_pair st = state ? *state : single(nullptr);
    return launch_mass(*cfg, *forest, st, dx0, dy0, static_cast<double *>(d_scratch), d_mass,
                       static_cast<cudaStream_t>(stream));
}

extern "C" af_status af_mass(const af_config *cfg, const af_forest *forest, const void *d_state, double dx0,
                             double dy0, void *d_scratch, double *d_mass, void *stream) {
    const af_state_pair st = single(d_state);
    return af_mass_pair(cfg, forest, &st, dx0, dy0, d_scratch, d_mass, stream);
}

// ---------------------------------------------------------------------------
// af_mass_noalloc: af_mass for callers that cannot allocate device memory.
// The per-block partial sums live in a fixed array compiled into the
// library instead of a caller-provided scratch buffer.  Every device that
// loads the library keeps this array (8 KB) until the process exits.
static __device__ __align__(256) double g_mass_partials[256 * 4];  // kMassBlocks partial sums x up to 4 components

extern "C" af_status af_mass_noalloc(const af_config *cfg, const af_forest *forest, const void *d_state, double dx0,
                                     double dy0, double *d_mass, void *stream) {
    if (!check_cfg(cfg) || !check_forest(forest)) return AF_ERR_ARG;
    if (!(dx0 > 0.0) || !(dy0 > 0.0) || !d_mass) return AF_ERR_ARG;
    if (forest->nleaf > 0 && !d_state) return AF_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(d_mass) & 7u) return AF_ERR_LAYOUT;
    const af_state_pair st = single(d_state);
    if (forest->nleaf > 0)
        if (const af_status e = check_pair(&st)) return e;  // the alignment af_mass requires
    const int nb = mass_blocks(forest->nleaf);
    // capacity check: partial sums needed vs. the fixed array
    if ((int64_t)nb * cfg->ncomp > (int64_t)(sizeof(g_mass_partials) / sizeof(double))) return AF_ERR_ARG;
    // In host code g_mass_partials names a host-side stand-in, not device
    // memory.  Its device address is looked up on every call, with the
    // caller's device current, so that it always belongs to the current
    // context (a cached address would go stale after a device reset).  The
    // lookup enqueues no work and allocates nothing.
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_mass_partials) != cudaSuccess || p == nullptr) return AF_ERR_CUDA;
    // every partial sum read by mass_final is written by mass_partial first,
    // so nothing left in the array by an earlier call is used
    return launch_mass(*cfg, *forest, st, dx0, dy0, static_cast<double *>(p), d_mass,
                       static_cast<cudaStream_t>(stream));
}

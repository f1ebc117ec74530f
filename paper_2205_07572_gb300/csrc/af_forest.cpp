// Host-side forest builder of libaf.so (Section 3 of arXiv 2205.07572: a
// forest of quadtrees of fixed-size patches, refined and coarsened from
// per-patch criteria, with 2:1 balance).  Plain C++, no device code: the
// regrid decision is a few microseconds per leaf on the host and feeds the
// device-side transfer (af_transfer) and work lists (af_build_step_work).
//
// Leaves are regions (l, ix, iy) of a periodic B x B brick; region (l, x, y)
// covers regions (l+1, 2x+a, 2y+b), a, b in {0, 1}.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <tuple>
#include <utility>
#include <vector>

#include "af_internal.h"

namespace af {
namespace {

// Per-level occupancy grids plus, for every region, the finest level of a
// leaf inside it (-1: none), kept current under splits and merges.
struct Occupancy {
    int B, lmax;
    std::vector<std::vector<int8_t>> leaf;    // [l][y * side + x] 1 if (l, x, y) is a leaf
    std::vector<std::vector<int8_t>> finest;  // [l][...] finest leaf level inside the region

    Occupancy(int B_, int lmax_) : B(B_), lmax(lmax_), leaf(lmax_ + 1), finest(lmax_ + 1) {
        for (int l = 0; l <= lmax; ++l) {
            const size_t cells = (size_t)side(l) * side(l);
            leaf[l].assign(cells, 0);
            finest[l].assign(cells, -1);
        }
    }
    int side(int l) const { return B << l; }
    size_t at(int l, int x, int y) const { return (size_t)y * side(l) + x; }
    bool is_leaf(int l, int x, int y) const { return leaf[l][at(l, x, y)] != 0; }

    // Recompute `finest` of region (l, x, y) and its ancestors.
    void refresh(int l, int x, int y) {
        for (int m = l; m >= 0; --m, x >>= 1, y >>= 1) {
            int f = leaf[m][at(m, x, y)] ? m : -1;
            if (m < lmax)
                for (int b = 0; b < 2; ++b)
                    for (int a = 0; a < 2; ++a) f = std::max<int>(f, finest[m + 1][at(m + 1, 2 * x + a, 2 * y + b)]);
            finest[m][at(m, x, y)] = (int8_t)f;
        }
    }
    void set(int l, int x, int y, bool v) {
        leaf[l][at(l, x, y)] = v ? 1 : 0;
        refresh(l, x, y);
    }
    void split(int l, int x, int y) {
        leaf[l][at(l, x, y)] = 0;
        for (int b = 0; b < 2; ++b)
            for (int a = 0; a < 2; ++a) leaf[l + 1][at(l + 1, 2 * x + a, 2 * y + b)] = 1;
        for (int b = 0; b < 2; ++b)
            for (int a = 0; a < 2; ++a) finest[l + 1][at(l + 1, 2 * x + a, 2 * y + b)] = (int8_t)(l + 1);
        refresh(l, x, y);
    }
    // True if a face or corner neighbour region of (l, x, y) holds a leaf of
    // level l + 2 or finer (the 2:1 rule).
    bool unbalanced(int l, int x, int y) const {
        const int s = side(l);
        for (int sy = -1; sy <= 1; ++sy)
            for (int sx = -1; sx <= 1; ++sx) {
                if (sx == 0 && sy == 0) continue;
                const int nx = ((x + sx) % s + s) % s, ny = ((y + sy) % s + s) % s;
                if (finest[l][at(l, nx, ny)] >= l + 2) return true;
            }
        return false;
    }
};

bool valid_leaves(int nleaf, int B, int lmax, const int32_t *lv, const int32_t *ix, const int32_t *iy) {
    for (int p = 0; p < nleaf; ++p) {
        if (lv[p] < 0 || lv[p] > lmax) return false;
        const int s = B << lv[p];
        if (ix[p] < 0 || ix[p] >= s || iy[p] < 0 || iy[p] >= s) return false;
    }
    return true;
}

}  // namespace
}  // namespace af

using namespace af;

extern "C" af_status af_forest_neighbours(int32_t nleaf, int32_t B, int32_t lmax, const int32_t *h_level,
                                          const int32_t *h_ix, const int32_t *h_iy, const int32_t *h_map,
                                          int32_t *h_nbr) {
    if (nleaf < 0 || B < 1 || lmax < 0 || lmax > AF_MAX_LEVEL) return AF_ERR_ARG;
    if (nleaf == 0) return AF_OK;
    if (!h_level || !h_ix || !h_iy || !h_map || !h_nbr) return AF_ERR_ARG;
    if (!valid_leaves(nleaf, B, lmax, h_level, h_ix, h_iy)) return AF_ERR_ARG;
    static const int dirs[8][2] = {{-1, 0}, {1, 0}, {0, -1}, {0, 1}, {-1, -1}, {1, -1}, {-1, 1}, {1, 1}};
    for (int p = 0; p < nleaf; ++p) {
        const int l = h_level[p], s = B << l;
        const int64_t off = (int64_t)B * B * (((int64_t)1 << (2 * l)) - 1) / 3;
        for (int d = 0; d < 8; ++d) {
            int nx = h_ix[p] + dirs[d][0], ny = h_iy[p] + dirs[d][1];  // periodic wrap
            nx = nx < 0 ? nx + s : (nx >= s ? nx - s : nx);
            ny = ny < 0 ? ny + s : (ny >= s ? ny - s : ny);
            const int32_t q = h_map[off + (int64_t)ny * s + nx];
            h_nbr[8 * p + d] = q >= 0 ? q : -1;
        }
    }
    return AF_OK;
}

extern "C" af_status af_forest_regrid(int32_t nleaf, int32_t B, int32_t lmin, int32_t lmax, const int32_t *h_level,
                                      const int32_t *h_ix, const int32_t *h_iy, const int8_t *h_tags,
                                      int32_t capacity, int32_t *out_level, int32_t *out_ix, int32_t *out_iy,
                                      int32_t *out_n) {
    if (nleaf < 0 || B < 1 || lmax < 0 || lmax > AF_MAX_LEVEL || lmin < 0 || lmin > lmax || !out_n || capacity < 0)
        return AF_ERR_ARG;
    if (nleaf > 0 && (!h_level || !h_ix || !h_iy || !h_tags)) return AF_ERR_ARG;
    if (!valid_leaves(nleaf, B, lmax, h_level, h_ix, h_iy)) return AF_ERR_ARG;
    Occupancy O(B, lmax);
    for (int p = 0; p < nleaf; ++p) {
        if (O.is_leaf(h_level[p], h_ix[p], h_iy[p])) return AF_ERR_ARG;  // duplicate leaf
        O.leaf[h_level[p]][O.at(h_level[p], h_ix[p], h_iy[p])] = 1;
    }
    for (int l = lmax; l >= 0; --l)
        for (int y = 0; y < O.side(l); ++y)
            for (int x = 0; x < O.side(l); ++x) {
                int f = O.leaf[l][O.at(l, x, y)] ? l : -1;
                if (l < lmax)
                    for (int b = 0; b < 2; ++b)
                        for (int a = 0; a < 2; ++a) f = std::max<int>(f, O.finest[l + 1][O.at(l + 1, 2 * x + a, 2 * y + b)]);
                O.finest[l][O.at(l, x, y)] = (int8_t)f;
            }
    // 1. refine: every leaf tagged 1 below lmax is split
    for (int p = 0; p < nleaf; ++p)
        if (h_tags[p] == 1 && h_level[p] < lmax) O.split(h_level[p], h_ix[p], h_iy[p]);
    // 2. coarsen: families of four leaves tagged -1 above lmin, in the order
    //    of their parent (level, x, y), each merged unless the parent would
    //    break the 2:1 rule in the forest as it stands
    struct Family {
        int l, x, y, count;
    };
    std::vector<Family> fam;
    {
        std::vector<std::pair<std::tuple<int, int, int>, int>> kids;
        for (int p = 0; p < nleaf; ++p)
            if (h_tags[p] == -1 && h_level[p] > lmin)
                kids.push_back({{h_level[p] - 1, h_ix[p] >> 1, h_iy[p] >> 1}, p});
        std::sort(kids.begin(), kids.end());
        for (size_t i = 0; i < kids.size();) {
            size_t j = i;
            while (j < kids.size() && kids[j].first == kids[i].first) ++j;
            fam.push_back({std::get<0>(kids[i].first), std::get<1>(kids[i].first), std::get<2>(kids[i].first),
                           (int)(j - i)});
            i = j;
        }
    }
    for (const Family &f : fam) {
        if (f.count != 4) continue;
        bool all = true;
        for (int b = 0; b < 2 && all; ++b)
            for (int a = 0; a < 2 && all; ++a) all = O.is_leaf(f.l + 1, 2 * f.x + a, 2 * f.y + b);
        if (!all) continue;
        for (int b = 0; b < 2; ++b)
            for (int a = 0; a < 2; ++a) O.leaf[f.l + 1][O.at(f.l + 1, 2 * f.x + a, 2 * f.y + b)] = 0;
        for (int b = 0; b < 2; ++b)
            for (int a = 0; a < 2; ++a) O.finest[f.l + 1][O.at(f.l + 1, 2 * f.x + a, 2 * f.y + b)] = -1;
        O.set(f.l, f.x, f.y, true);
        if (O.unbalanced(f.l, f.x, f.y)) {
            O.leaf[f.l][O.at(f.l, f.x, f.y)] = 0;
            for (int b = 0; b < 2; ++b)
                for (int a = 0; a < 2; ++a) {
                    O.leaf[f.l + 1][O.at(f.l + 1, 2 * f.x + a, 2 * f.y + b)] = 1;
                    O.finest[f.l + 1][O.at(f.l + 1, 2 * f.x + a, 2 * f.y + b)] = (int8_t)(f.l + 1);
                }
            O.refresh(f.l, f.x, f.y);
        }
    }
    // 3. balance: split unbalanced leaves until none is left.  Splitting is
    //    monotone and every split made is needed by any balanced refinement,
    //    so the result does not depend on the order of the sweep.
    for (bool changed = true; changed;) {
        changed = false;
        for (int l = 0; l < lmax; ++l)
            for (int y = 0; y < O.side(l); ++y)
                for (int x = 0; x < O.side(l); ++x)
                    if (O.leaf[l][O.at(l, x, y)] && O.unbalanced(l, x, y)) {
                        O.split(l, x, y);
                        changed = true;
                    }
    }
    int32_t count = 0;
    for (int l = 0; l <= lmax; ++l)
        for (int8_t v : O.leaf[l]) count += v;
    *out_n = count;
    if (count > capacity || (count > 0 && (!out_level || !out_ix || !out_iy))) return AF_ERR_ARG;
    int32_t k = 0;
    for (int l = 0; l <= lmax; ++l)
        for (int y = 0; y < O.side(l); ++y)
            for (int x = 0; x < O.side(l); ++x)
                if (O.leaf[l][O.at(l, x, y)]) {
                    out_level[k] = l;
                    out_ix[k] = x;
                    out_iy[k] = y;
                    ++k;
                }
    return AF_OK;
}

// Internal declarations shared by the host and device translation units of
// libaf.so.  Not part of the public ABI (include/af.h is).
#pragma once

#include <cstdint>

#include "af.h"

namespace af {

constexpr int kGhost = 2;      // ghost layers (Section 3.2)
constexpr int kTileMax = 32;   // cells per tile side in af_patch_step
constexpr int kPlanes = 4;     // avg, xmid, corner, ymid (Section 2, Fig. 1)
enum Plane { kAvg = 0, kXmid = 1, kCorner = 2, kYmid = 3 };


// ---------------------------------------------------------------------------
// Acoustic stencil weights (Eqs. ERFormula, sphe-mean).
//
// A node-cell work item (i, j) evolves the corner at node lines (i, j), the
// left-edge midpoint of cell (i, j) and the bottom-edge midpoint of cell
// (i, j).  All three discs lie in the 2 x 2 cell block (i-1..i, j-1..j), whose
// 25 degrees of freedom per component are numbered
//   k in [0, 4):   averages of cells (i-1+a, j-1+b),      k = 2b + a
//   k in [4, 13):  corners at lines (i-1+a, j-1+b),       k = 4 + 3b + a
//   k in [13, 19): left-edge mids (line i-1+a, row j-1+b), k = 13 + 3b + a
//   k in [19, 25): bottom-edge mids (col i-1+a, line j-1+b), k = 19 + 2b + a
// The corner uses all 25, the edge midpoints 15 each (x_idx / y_idx).
// Component pairs (out <- in) with non-zero weights:
//   0 p<-p, 1 p<-u, 2 p<-v, 3 u<-u, 4 u<-p, 5 v<-v, 6 v<-p.
// Combination 0 is T = Q^n + 4 Q^{n+1/2} + Q^{n+1} (the time-Simpson sum
// entering Eq. Simpson-2d), combination 1 is Q^{n+1}.
#ifdef __CUDACC__
#define AF_HD __host__ __device__
#else
#define AF_HD
#endif
AF_HD constexpr int64_t plane_stride(int n) {
    return ((int64_t)(n + 2 * kGhost + 1) * (n + 2 * kGhost + 1) + 7) / 8 * 8;
}

AF_HD constexpr int x_idx(int k) {
    constexpr int t[15] = {2, 3, 7, 8, 9, 10, 11, 12, 16, 17, 18, 21, 22, 23, 24};
    return t[k];
}
AF_HD constexpr int y_idx(int k) {
    constexpr int t[15] = {1, 3, 5, 6, 8, 9, 11, 12, 14, 15, 17, 18, 20, 22, 24};
    return t[k];
}

template <typename T>
struct AcousticWeights {
    T wc[2][7][25];
    T wx[2][7][15];
    T wy[2][7][15];
};

// The same weights folded by the mirror symmetries of each node's stencil
// (x -> -x and y -> -y about the node; they hold for dx != dy).  Degrees of
// freedom are first combined into orbit sums: SS (symmetric in x and y),
// AS (antisymmetric in x, symmetric in y), SA (symmetric in x, antisymmetric
// in y).  The operator M + R d_R M acts on SS, -R M{d/dX} on AS and
// -R M{d/dY} on SA; by symmetry every other combination vanishes.  Orbit
// order and representatives: see sym_rep() in af_weights.cpp.
//   corner node: SS 9, AS 6, SA 6;  left-edge mid: SS 6, AS 4, SA 3;
//   bottom-edge mid: SS 6, AS 3, SA 4.   [2] = T combination, Q^{n+1}.
template <typename T>
struct AcousticSymWeights {
    T cA[2][9], cDx[2][6], cDy[2][6];
    T xA[2][6], xDx[2][4], xDy[2][3];
    T yA[2][6], yDx[2][3], yDy[2][4];
};

// FP32 acoustic weights with the two time combinations of each weight side
// by side (x: T, y: Q^{n+1}), so one packed FP32x2 multiply-add advances
// both accumulators of a node value.
struct AcousticPairWeights {
    float cA[9][2], cDx[6][2], cDy[6][2];
    float xA[6][2], xDx[4][2], xDy[3][2];
    float yA[6][2], yDx[3][2], yDy[4][2];
};

// Advection weights (Eq. advection-update): for node type t (0 corner,
// 1 left-edge mid, 2 bottom-edge mid) and time s (0: dt/2, 1: dt) the foot of
// the characteristic lies in cell (line + off[t][s][0], line + off[t][s][1]);
// the value there is sum_k w[t][s][k] * dof_k over that cell's nine degrees
// of freedom ordered avg, corner(0,0), corner(1,0), corner(0,1), corner(1,1),
// xmid(0), xmid(1), ymid(0), ymid(1).
template <typename T>
struct AdvectionWeights {
    T w[3][2][9];
    int32_t off[3][2][2];
};

// Double-precision derivations on the host (af_weights.cpp).
void acoustic_weights(double rho_x, double rho_y, AcousticWeights<double> &w);
// Folded weights; returns false if the dense weights lack the symmetry
// (max deviation above 1e-12 of the largest weight), which cannot happen for
// the operators of Eq. ERFormula.
bool acoustic_sym_weights(double rho_x, double rho_y, AcousticSymWeights<double> &w);
void advection_weights(double nu_x, double nu_y, AdvectionWeights<double> &w);

}  // namespace af

namespace af {

// Tile shapes compiled into af_patch_step: at most tmx x tmy cells per tile,
// `threads` per CTA; persistent = one CTA per available slot looping over
// tiles with the next tile's copies in flight.
struct Tiling {
    int tmx, tmy, threads, persistent;
};
constexpr int kNumTilings = 10;
AF_HD constexpr Tiling tiling(int k) {
    constexpr Tiling t[kNumTilings] = {
        {32, 32, 256, 0}, {32, 16, 192, 0}, {32, 16, 160, 0}, {32, 8, 128, 0}, {16, 16, 128, 0},
        {32, 8, 256, 1}, {18, 18, 256, 0}, {18, 10, 192, 0}, {10, 10, 128, 0}, {18, 18, 128, 0}};
    return t[k];
}
// Default tiling for patches of n cells (overridden per configuration by
// the autotuner through the *_tiled entry points).
inline int default_tiling(int n) { return n <= 8 ? 8 : (n <= 16 ? 6 : 0); }

// Split `w` cells into ceil(w / kTileMax) tiles of near-equal size.
inline int tiles_for(int w) { return (w + kTileMax - 1) / kTileMax; }
inline int tile_size_max(int w) {
    const int t = tiles_for(w);
    return (w + t - 1) / t;
}
// Largest tile side af_build_step_work produces for patches of n cells.
inline int tile_max_for(int n) {
    const int a = tile_size_max(n), b = tile_size_max(n + 2);
    return a > b ? a : b;
}

}  // namespace af

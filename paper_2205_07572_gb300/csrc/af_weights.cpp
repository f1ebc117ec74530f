// Host-side derivation of the constant stencil weights of the Active Flux
// point-value evolution (FP64).  Both PDEs are linear with constant
// coefficients and dt/dx is the same on every refinement level, so every
// evolved point value is a fixed linear combination of the degrees of freedom
// of the cells around it; these weights are computed once per
// (equation, Courant numbers) and passed to the kernels by value.
#include <cmath>
#include <cstring>

#include "af_internal.h"

namespace af {
namespace {

constexpr double kPi = 3.14159265358979323846;

// 1-D Lagrange polynomials on the nodes {-1, 0, 1}: L(s) = c0 + c1 s + c2 s^2.
constexpr double kLag[3][3] = {{0.0, -0.5, 0.5}, {1.0, 0.0, -1.0}, {0.0, 0.5, 0.5}};
// Cell average of L_a over [-1, 1] (Simpson weights; exact for quadratics).
constexpr double kMean[3] = {1.0 / 6.0, 2.0 / 3.0, 1.0 / 6.0};

// The nine degrees of freedom of one cell in the order used by the weight
// tables: avg, corner(0,0), corner(1,0), corner(0,1), corner(1,1), xmid(0),
// xmid(1), ymid(0), ymid(1).  kNode gives the Lagrange node (a, b) of each
// point value (a, b in {0,1,2} for xi, eta in {-1, 0, 1}).
constexpr int kNode[9][2] = {{1, 1}, {0, 0}, {2, 0}, {0, 2}, {2, 2}, {0, 1}, {2, 1}, {1, 0}, {1, 2}};

// Coefficients (in t) of L_a(s0 + 2 t): t is an offset measured in cell widths.
void lag_shifted(int a, double s0, double out[3]) {
    const double *c = kLag[a];
    out[0] = c[0] + c[1] * s0 + c[2] * s0 * s0;
    out[1] = 2.0 * c[1] + 4.0 * c[2] * s0;
    out[2] = 4.0 * c[2];
}

// Basis function of degree of freedom d of Eq. poly, written as a polynomial
// sum_{m,n<=2} coef[m][n] x^m y^n in offsets (x, y) (cell widths) from the
// reference point (xi0, eta0).  The point values are nodal; the centre value
// is eliminated through the average condition, so the average's basis is
// L_1 L_1 / (w_1 w_1) and each point value's basis subtracts w_a w_b / (w_1 w_1)
// of it.
void basis_poly(int d, double xi0, double eta0, double coef[3][3]) {
    double cx[3], cy[3], kx[3], ky[3];
    lag_shifted(1, xi0, kx);
    lag_shifted(1, eta0, ky);
    const double wc = kMean[1] * kMean[1];
    if (d == 0) {
        for (int m = 0; m < 3; ++m)
            for (int n = 0; n < 3; ++n) coef[m][n] = kx[m] * ky[n] / wc;
        return;
    }
    const int a = kNode[d][0], b = kNode[d][1];
    lag_shifted(a, xi0, cx);
    lag_shifted(b, eta0, cy);
    const double r = kMean[a] * kMean[b] / wc;
    for (int m = 0; m < 3; ++m)
        for (int n = 0; n < 3; ++n) coef[m][n] = cx[m] * cy[n] - r * kx[m] * ky[n];
}

double basis_value(int d, double xi, double eta) {
    auto L = [](int a, double s) { return kLag[a][0] + kLag[a][1] * s + kLag[a][2] * s * s; };
    const double c = L(1, xi) * L(1, eta) / (kMean[1] * kMean[1]);
    if (d == 0) return c;
    const int a = kNode[d][0], b = kNode[d][1];
    return L(a, xi) * L(b, eta) - kMean[a] * kMean[b] * c;
}

// Normalised spherical-mean moment of X^m Y^n over the part of the disc in
// quadrant q (angles [q pi/2, (q+1) pi/2]):
//   (1 / (2 pi R)) int_S int_0^R X^m Y^n s / sqrt(R^2 - s^2) ds dphi / R^{m+n}
// = J_{m+n+1} A_mn(q) / (2 pi),
// with the radial factor J_k = int_0^1 t^k / sqrt(1 - t^2) dt = B((k+1)/2, 1/2)/2
// and the angular factor A_mn(0) = int_0^{pi/2} cos^m sin^n = B((m+1)/2, (n+1)/2)/2;
// the other quadrants follow from cos -> -sin, sin -> cos under phi -> phi + pi/2.
double beta(double x, double y) { return std::exp(std::lgamma(x) + std::lgamma(y) - std::lgamma(x + y)); }

double moment(int m, int n, int q) {
    const double radial = 0.5 * beta(0.5 * (m + n + 2), 0.5);
    const double angular = 0.5 * beta(0.5 * (m + 1), 0.5 * (n + 1));
    const bool flip_cos = (q == 1 || q == 2);
    const bool flip_sin = (q == 2 || q == 3);
    double sgn = 1.0;
    if (flip_cos && (m & 1)) sgn = -sgn;
    if (flip_sin && (n & 1)) sgn = -sgn;
    return radial * angular * sgn / (2.0 * kPi);
}

struct Sector {
    int cx, cy;        // cell offset from the node line (i, j): cell (i+cx, j+cy)
    double xi0, eta0;  // the node in that cell's reference coordinates
    int q0, q1;        // quadrants [q0, q1] of the disc inside the cell
};

// Map degree of freedom d of the cell at block position (cx, cy) (cx, cy in
// {-1, 0}) to its index in the 25-entry block of the node line (i, j).
int block_index(int d, int cx, int cy) {
    const int a = cx + 1, b = cy + 1;  // block cell
    switch (d) {
    case 0: return 2 * b + a;
    case 1: return 4 + 3 * b + a;
    case 2: return 4 + 3 * b + a + 1;
    case 3: return 4 + 3 * (b + 1) + a;
    case 4: return 4 + 3 * (b + 1) + a + 1;
    case 5: return 13 + 3 * b + a;
    case 6: return 13 + 3 * b + a + 1;
    case 7: return 19 + 2 * b + a;
    default: return 19 + 2 * (b + 1) + a;
    }
}

// Evolution operators of Eq. ERFormula applied to each block basis function at
// radius R (rx = R/dx, ry = R/dy): A = M + R d_R M, Dx = -R M{d/dX},
// Dy = -R M{d/dY}.
void node_operators(const Sector *sec, int nsec, double rx, double ry, double A[25], double Dx[25],
                    double Dy[25]) {
    for (int k = 0; k < 25; ++k) A[k] = Dx[k] = Dy[k] = 0.0;
    double px[3] = {1.0, rx, rx * rx}, py[3] = {1.0, ry, ry * ry};
    for (int s = 0; s < nsec; ++s) {
        double mu[3][3];
        for (int m = 0; m < 3; ++m)
            for (int n = 0; n < 3; ++n) {
                mu[m][n] = 0.0;
                for (int q = sec[s].q0; q <= sec[s].q1; ++q) mu[m][n] += moment(m, n, q & 3);
            }
        for (int d = 0; d < 9; ++d) {
            double c[3][3];
            basis_poly(d, sec[s].xi0, sec[s].eta0, c);
            const int k = block_index(d, sec[s].cx, sec[s].cy);
            for (int m = 0; m < 3; ++m)
                for (int n = 0; n < 3; ++n) {
                    const double t = c[m][n] * px[m] * py[n];
                    A[k] += (1.0 + m + n) * t * mu[m][n];
                    if (m > 0) Dx[k] -= m * t * mu[m - 1][n];
                    if (n > 0) Dy[k] -= n * t * mu[m][n - 1];
                }
        }
    }
}

}  // namespace

// Dense operators of node type t (0 corner, 1 left-edge mid, 2 bottom-edge
// mid) over the 25-entry block: op[c][0..2][k] = A, Dx, Dy for combination
// c (0: T = Q^n + 4 Q^{n+1/2} + Q^{n+1}, 1: Q^{n+1}).
void node_type_operators(int t, double rho_x, double rho_y, double op[2][3][25]) {
    // Sectors of the three node types (Eq. cfl-acoustics keeps each disc inside
    // the cells that share the node).
    const Sector corner[4] = {{0, 0, -1.0, -1.0, 0, 0}, {-1, 0, 1.0, -1.0, 1, 1},
                              {-1, -1, 1.0, 1.0, 2, 2}, {0, -1, -1.0, 1.0, 3, 3}};
    const Sector xmid[2] = {{0, 0, -1.0, 0.0, 3, 4}, {-1, 0, 1.0, 0.0, 1, 2}};
    const Sector ymid[2] = {{0, 0, 0.0, -1.0, 0, 1}, {0, -1, 0.0, 1.0, 2, 3}};
    const Sector *secs[3] = {corner, xmid, ymid};
    const int nsec[3] = {4, 2, 2};
    const int own[3] = {8, 17, 22};  // block index of the node itself
    double Ah[25], Dxh[25], Dyh[25], A1[25], Dx1[25], Dy1[25];
    node_operators(secs[t], nsec[t], 0.5 * rho_x, 0.5 * rho_y, Ah, Dxh, Dyh);
    node_operators(secs[t], nsec[t], rho_x, rho_y, A1, Dx1, Dy1);
    for (int k = 0; k < 25; ++k) {
        op[0][0][k] = 4.0 * Ah[k] + A1[k] + (k == own[t] ? 1.0 : 0.0);
        op[0][1][k] = 4.0 * Dxh[k] + Dx1[k];
        op[0][2][k] = 4.0 * Dyh[k] + Dy1[k];
        op[1][0][k] = A1[k];
        op[1][1][k] = Dx1[k];
        op[1][2][k] = Dy1[k];
    }
}

void acoustic_weights(double rho_x, double rho_y, AcousticWeights<double> &w) {
    for (int t = 0; t < 3; ++t) {
        double op[2][3][25];
        node_type_operators(t, rho_x, rho_y, op);
        double full[2][7][25];
        for (int k = 0; k < 25; ++k) {
            const double ta = op[0][0][k];
            const double tx = op[0][1][k];
            const double ty = op[0][2][k];
            const double A1[1] = {op[1][0][k]}, Dx1[1] = {op[1][1][k]}, Dy1[1] = {op[1][2][k]};
            const double T[7] = {ta, tx, ty, ta, tx, ta, ty};
            const double N[7] = {A1[0], Dx1[0], Dy1[0], A1[0], Dx1[0], A1[0], Dy1[0]};
            for (int p = 0; p < 7; ++p) {
                full[0][p][k] = T[p];
                full[1][p][k] = N[p];
            }
        }
        for (int c = 0; c < 2; ++c)
            for (int p = 0; p < 7; ++p) {
                if (t == 0) {
                    for (int k = 0; k < 25; ++k) w.wc[c][p][k] = full[c][p][k];
                } else {
                    for (int k = 0; k < 15; ++k) {
                        if (t == 1) w.wx[c][p][k] = full[c][p][x_idx(k)];
                        else w.wy[c][p][k] = full[c][p][y_idx(k)];
                    }
                }
            }
    }
}

void advection_weights(double nu_x, double nu_y, AdvectionWeights<double> &w) {
    // Eq. advection-update: the value at a node after tau is q^n at the foot
    // (x - a tau, y - b tau); in cell units relative to the node line the foot
    // sits at (ox - nu_x f, oy - nu_y f), f = tau / dt.
    for (int t = 0; t < 3; ++t)
        for (int s = 0; s < 2; ++s) {
            const double f = (s == 0) ? 0.5 : 1.0;
            const double ox = (t == 2) ? 0.5 : 0.0, oy = (t == 1) ? 0.5 : 0.0;
            const double fx = ox - nu_x * f, fy = oy - nu_y * f;
            int kx = (int)std::floor(fx), ky = (int)std::floor(fy);
            // a node on a grid line whose foot lands exactly one cell ahead
            // (Courant number exactly 1): use the cell behind, at its far face
            if (t != 2 && kx == 1) kx = 0;
            if (t != 1 && ky == 1) ky = 0;
            // |Courant number| <= 1 keeps the foot cell within these bounds
            // (checked by the caller); clamp so the stencil never leaves the
            // staged window even for a rounding-level overshoot
            const int kxmin = -1, kxmax = (t == 2) ? 1 : 0;
            const int kymin = -1, kymax = (t == 1) ? 1 : 0;
            kx = kx < kxmin ? kxmin : (kx > kxmax ? kxmax : kx);
            ky = ky < kymin ? kymin : (ky > kymax ? kymax : ky);
            const double xi = 2.0 * (fx - kx) - 1.0, eta = 2.0 * (fy - ky) - 1.0;
            w.off[t][s][0] = kx;
            w.off[t][s][1] = ky;
            for (int d = 0; d < 9; ++d) w.w[t][s][d] = basis_value(d, xi, eta);
        }
}

}  // namespace af

namespace af {
namespace {

// Orbits of the block entries under the two mirror symmetries of a node.
// A quad lists (++, +-, -+, --) by the signs of (x, y) relative to the node;
// an x-pair (p, m) lies on y = 0, a y-pair on x = 0.
struct Orbit {
    int kind;    // 0 quad, 1 x-pair, 2 y-pair, 3 single
    int m[4];
};

// SS / AS / SA orbit lists of node type t, in the order the kernel uses.
int orbits(int t, int which, Orbit *o) {
    static const Orbit c_ss[9] = {{0, {3, 1, 2, 0}},   {0, {12, 6, 10, 4}}, {0, {18, 15, 16, 13}},
                                  {0, {24, 20, 23, 19}}, {1, {9, 7}},        {1, {22, 21}},
                                  {2, {11, 5}},          {2, {17, 14}},      {3, {8}}};
    static const Orbit x_ss[6] = {{0, {12, 9, 10, 7}}, {0, {24, 22, 23, 21}}, {1, {3, 2}},
                                  {1, {18, 16}},       {2, {11, 8}},          {3, {17}}};
    static const Orbit y_ss[6] = {{0, {12, 6, 11, 5}}, {0, {18, 15, 17, 14}}, {1, {9, 8}},
                                  {2, {3, 1}},         {2, {24, 20}},         {3, {22}}};
    const Orbit *ss = t == 0 ? c_ss : (t == 1 ? x_ss : y_ss);
    const int nss = t == 0 ? 9 : 6;
    int n = 0;
    for (int i = 0; i < nss; ++i) {
        const int k = ss[i].kind;
        if (which == 0 || (which == 1 && (k == 0 || k == 1)) || (which == 2 && (k == 0 || k == 2))) o[n++] = ss[i];
    }
    return n;
}

// Expected sign of member j of an orbit for operator `which` (0 A, 1 Dx, 2 Dy).
double member_sign(const Orbit &o, int which, int j) {
    if (which == 0) return 1.0;
    if (o.kind == 0) {
        const bool xneg = (j >= 2), yneg = (j == 1 || j == 3);
        return which == 1 ? (xneg ? -1.0 : 1.0) : (yneg ? -1.0 : 1.0);
    }
    return j == 0 ? 1.0 : -1.0;  // the antisymmetric direction of a pair
}

}  // namespace

bool acoustic_sym_weights(double rho_x, double rho_y, AcousticSymWeights<double> &w) {
    bool ok = true;
    for (int t = 0; t < 3; ++t) {
        double op[2][3][25];
        node_type_operators(t, rho_x, rho_y, op);
        double big = 0.0;
        for (int c = 0; c < 2; ++c)
            for (int q = 0; q < 3; ++q)
                for (int k = 0; k < 25; ++k) big = std::fmax(big, std::fabs(op[c][q][k]));
        for (int c = 0; c < 2; ++c)
            for (int which = 0; which < 3; ++which) {
                Orbit o[9];
                const int no = orbits(t, which, o);
                double *dst = nullptr;
                if (t == 0) dst = which == 0 ? w.cA[c] : (which == 1 ? w.cDx[c] : w.cDy[c]);
                if (t == 1) dst = which == 0 ? w.xA[c] : (which == 1 ? w.xDx[c] : w.xDy[c]);
                if (t == 2) dst = which == 0 ? w.yA[c] : (which == 1 ? w.yDx[c] : w.yDy[c]);
                bool used[25] = {false};
                for (int i = 0; i < no; ++i) {
                    const int nm = o[i].kind == 0 ? 4 : (o[i].kind == 3 ? 1 : 2);
                    const double rep = op[c][which][o[i].m[0]];
                    dst[i] = rep;
                    for (int j = 0; j < nm; ++j) {
                        used[o[i].m[j]] = true;
                        if (std::fabs(op[c][which][o[i].m[j]] - member_sign(o[i], which, j) * rep) > 1e-12 * big)
                            ok = false;
                    }
                }
                // every weight outside the listed orbits must vanish
                for (int k = 0; k < 25; ++k)
                    if (!used[k] && std::fabs(op[c][which][k]) > 1e-12 * big) ok = false;
            }
    }
    return ok;
}

}  // namespace af

/*
 * FP64 CPU oracle for the Cartesian-grid Active Flux method with AMR
 * (Calhoun, Chudzik, Helzel, "The Cartesian Grid Active Flux Method with
 * Adaptive Mesh Refinement", arXiv 2205.07572).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or helper with the CUDA library; the two meet only in the
 * documented state layout.
 *
 * Everything is written in the order and notation of the paper, slow and
 * plain: one node at a time, one face at a time, one cell at a time.
 *
 * State layout (the library's interface contract): per patch, per component,
 * four planes (0 = cell average Q_{i,j}, 1 = left-edge midpoint Q_{i-1/2,j},
 * 2 = lower-left corner Q_{i-1/2,j-1/2}, 3 = bottom-edge midpoint
 * Q_{i,j-1/2}; Section 2, Fig. 1), each a (N+2g+1)^2 row-major lattice padded
 * to a multiple of 8 entries, g = 2 ghost layers (Section 3.2).
 *
 * Parity status of each function is stated next to it; the pins live in
 * tests/test_oracle_*.py.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NG 2 /* ghost layers (Section 3.2, "two layers of ghost cells") */

enum { PL_AVG = 0, PL_XMID = 1, PL_CORNER = 2, PL_YMID = 3 };
enum { EQ_ADVECTION = 0, EQ_ACOUSTICS = 1 };
enum { ND_CORNER = 0, ND_XMID = 1, ND_YMID = 2 };

typedef struct {
    int32_t eq;     /* EQ_ADVECTION or EQ_ACOUSTICS */
    int32_t n;      /* interior cells per patch side */
    int32_t ncomp;  /* 1 or 3 */
    int32_t pad_;
    double dx, dy, dt;
    double a, b;    /* advection velocity (Eq. advection2d) */
    double c;       /* speed of sound (Eq. acoustics) */
} orc_cfg;

typedef struct {
    int n, w;
    long plane;
    int ncomp;
} lay_t;

static lay_t lay_make(int n, int ncomp) {
    lay_t L;
    L.n = n;
    L.w = n + 2 * NG + 1;
    L.plane = ((long)L.w * L.w + 7) / 8 * 8;
    L.ncomp = ncomp;
    return L;
}

static long lay_patch_words(const lay_t *L) { return (long)L->ncomp * 4 * L->plane; }

/* Lattice offset of cell / node-line index (i, j), i, j in [-g, N+g]. */
static long IX(const lay_t *L, int i, int j) { return (long)(j + NG) * L->w + (i + NG); }

static const double *PLc(const lay_t *L, const double *patch, int comp, int plane) {
    return patch + ((long)comp * 4 + plane) * L->plane;
}
static double *PL(const lay_t *L, double *patch, int comp, int plane) {
    return patch + ((long)comp * 4 + plane) * L->plane;
}

long orc_plane_stride(int n) { lay_t L = lay_make(n, 1); return L.plane; }

/* ------------------------------------------------------------------ Eq. poly
 * Reconstruction on the reference cell [-1,1]^2 (Section 2, Eq. poly).  The
 * biquadratic space spanned by the nine monomials of Eq. poly is written in
 * the tensor Lagrange basis on the nodes {-1,0,1}^2.  Eight nodal values are
 * the point values on the cell boundary; the ninth (the centre) is fixed by
 * requiring the cell average of the polynomial to equal Q_{i,j}.  The average
 * of L_a(xi) L_b(eta) over the cell is w_a w_b with the Simpson weights
 * w = (1/6, 2/3, 1/6), because Simpson's rule integrates quadratics exactly.
 * Pinned by: biquadratics are reproduced exactly, average matches (P1).      */
static const double SIMPSON_W[3] = {1.0 / 6.0, 2.0 / 3.0, 1.0 / 6.0};

/* k-th Lagrange polynomial on nodes {-1,0,1} (k = 0,1,2), d-th derivative. */
static double lag(int k, int d, double s) {
    switch (k) {
    case 0: return d == 0 ? 0.5 * s * (s - 1.0) : (d == 1 ? s - 0.5 : 1.0);
    case 1: return d == 0 ? 1.0 - s * s : (d == 1 ? -2.0 * s : -2.0);
    default: return d == 0 ? 0.5 * s * (s + 1.0) : (d == 1 ? s + 0.5 : 1.0);
    }
}

/* Nodal values q[b][a] of cell (i, j) (a indexes xi = -1,0,1; b indexes eta). */
static void cell_nodal(const lay_t *L, const double *patch, int comp, int i, int j, double q[3][3]) {
    const double *avg = PLc(L, patch, comp, PL_AVG);
    const double *xm = PLc(L, patch, comp, PL_XMID);
    const double *co = PLc(L, patch, comp, PL_CORNER);
    const double *ym = PLc(L, patch, comp, PL_YMID);
    q[0][0] = co[IX(L, i, j)];
    q[0][2] = co[IX(L, i + 1, j)];
    q[2][0] = co[IX(L, i, j + 1)];
    q[2][2] = co[IX(L, i + 1, j + 1)];
    q[1][0] = xm[IX(L, i, j)];
    q[1][2] = xm[IX(L, i + 1, j)];
    q[0][1] = ym[IX(L, i, j)];
    q[2][1] = ym[IX(L, i, j + 1)];
    double rest = 0.0;
    for (int b = 0; b < 3; ++b)
        for (int a = 0; a < 3; ++a)
            if (!(a == 1 && b == 1)) rest += SIMPSON_W[a] * SIMPSON_W[b] * q[b][a];
    q[1][1] = (avg[IX(L, i, j)] - rest) / (SIMPSON_W[1] * SIMPSON_W[1]);
}

/* d^{mx}/dxi^{mx} d^{my}/deta^{my} of the reconstruction at (xi, eta). */
static double recon_deriv(const double q[3][3], double xi, double eta, int mx, int my) {
    double s = 0.0;
    for (int b = 0; b < 3; ++b)
        for (int a = 0; a < 3; ++a) s += q[b][a] * lag(a, mx, xi) * lag(b, my, eta);
    return s;
}

/* Exported for the pins: value (or derivative, in physical units) of the
 * reconstruction of cell (i, j) of one patch at reference point (xi, eta). */
double orc_recon_eval(int n, int ncomp, const double *patch, int comp, int i, int j,
                      double xi, double eta, int mx, int my, double dx, double dy) {
    lay_t L = lay_make(n, ncomp);
    double q[3][3];
    cell_nodal(&L, patch, comp, i, j, q);
    return recon_deriv(q, xi, eta, mx, my) * pow(2.0 / dx, mx) * pow(2.0 / dy, my);
}

/* ------------------------------------------- Section 2.1, Eq. advection-update
 * q(x, y, t + tau) = q(x - a tau, y - b tau, t): the point value at a node is
 * the reconstruction q^n evaluated at the foot of the characteristic.  The
 * foot is located relative to the node (in cell units) so the arithmetic does
 * not depend on where the patch sits; with CFL <= 1 (Eq. cfl-adv) it lies in a
 * cell adjacent to the node.  On a cell face either neighbour gives the same
 * value because q^n is continuous.
 * Pinned by: exact translation of polynomial data (P2, P3).                   */
static double advect_node(const lay_t *L, const double *patch, int comp, const orc_cfg *cf,
                          int type, int i, int j, double tau) {
    /* node position in cell units relative to node line (i, j) */
    double ox = (type == ND_YMID) ? 0.5 : 0.0;
    double oy = (type == ND_XMID) ? 0.5 : 0.0;
    double fx = ox - cf->a * tau / cf->dx; /* foot, relative to line i */
    double fy = oy - cf->b * tau / cf->dy;
    double kx = floor(fx), ky = floor(fy);
    int ci = i + (int)kx, cj = j + (int)ky;
    double xi = 2.0 * (fx - kx) - 1.0, eta = 2.0 * (fy - ky) - 1.0;
    double q[3][3];
    cell_nodal(L, patch, comp, ci, cj, q);
    return recon_deriv(q, xi, eta, 0, 0);
}

/* ---------------------------------- Section 2.3, Eqs. ERFormula and sphe-mean
 * p(t) = M_R{p} + R (d_R M_R{p} - M_R{div u}),
 * u(t) = M_R{u} + R (d_R M_R{u} - M_R{grad p}),  R = c t,
 * M_R{f}(x) = 1/(2 pi R) int_0^{2pi} int_0^R f(x + s(cos phi, sin phi))
 *             s / sqrt(R^2 - s^2) ds dphi.
 * With the time step restricted by Eq. cfl-acoustics the disc of radius R
 * around a corner lies in the four cells sharing the corner (one quadrant
 * each) and around an edge midpoint in the two cells sharing the edge (one
 * half-plane each).  In each such sector the reconstruction is a polynomial;
 * written in physical offsets (X, Y) from the node, f = sum t_mn X^m Y^n with
 * Taylor coefficients t_mn (exact, m, n <= 2).  For one monomial
 *   M_R{X^m Y^n}|_S = R^{m+n} J_{m+n+1} A_mn(S) / (2 pi),
 *   J_k = int_0^1 t^k / sqrt(1 - t^2) dt,  A_mn(S) = int_S cos^m sin^n dphi,
 * and R d_R of it is (m+n) times the same.  This is the exact evaluation the
 * paper asks for ("the solution formula can be evaluated exactly").
 * Pinned by: brute-force quadrature of Eq. sphe-mean (P4) and the exact wave
 * solution for curl-free polynomial data (P5).                               */
static double J_int(int k) {
    double j0 = M_PI / 2.0, j1 = 1.0;
    if (k == 0) return j0;
    if (k == 1) return j1;
    double jm2 = (k % 2 == 0) ? j0 : j1;
    for (int s = (k % 2 == 0) ? 2 : 3; s <= k; s += 2) jm2 = jm2 * (double)(s - 1) / (double)s;
    return jm2;
}

/* antiderivative of cos^m(phi) sin^n(phi), m, n in {0,1,2} */
static double trig_prim(int m, int n, double f) {
    double s = sin(f), c = cos(f);
    switch (m * 3 + n) {
    case 0: return f;
    case 1: return -c;
    case 2: return 0.5 * f - 0.25 * sin(2.0 * f);
    case 3: return s;
    case 4: return 0.5 * s * s;
    case 5: return s * s * s / 3.0;
    case 6: return 0.5 * f + 0.25 * sin(2.0 * f);
    case 7: return -c * c * c / 3.0;
    default: return f / 8.0 - sin(4.0 * f) / 32.0;
    }
}

static double sector_A(int m, int n, double phi0, double phi1) {
    return trig_prim(m, n, phi1) - trig_prim(m, n, phi0);
}

/* Taylor coefficients t[m][n] of the reconstruction of a cell about the
 * reference point (xin, etan), in physical offsets. */
static void taylor(const double q[3][3], double xin, double etan, double dx, double dy, double t[3][3]) {
    static const double fact[3] = {1.0, 1.0, 2.0};
    for (int m = 0; m < 3; ++m)
        for (int n = 0; n < 3; ++n)
            t[m][n] = recon_deriv(q, xin, etan, m, n) * pow(2.0 / dx, m) * pow(2.0 / dy, n) /
                      (fact[m] * fact[n]);
}

/* M_R and R d_R M_R of the polynomial sum t_mn X^m Y^n over one sector. */
static void sector_mean(const double t[3][3], double R, double phi0, double phi1, double *M, double *RdM) {
    double s0 = 0.0, s1 = 0.0;
    for (int m = 0; m < 3; ++m)
        for (int n = 0; n < 3; ++n) {
            double mono = pow(R, m + n) * J_int(m + n + 1) * sector_A(m, n, phi0, phi1) / (2.0 * M_PI);
            s0 += t[m][n] * mono;
            s1 += (double)(m + n) * t[m][n] * mono;
        }
    *M = s0;
    *RdM = s1;
}

typedef struct {
    int di, dj;        /* cell offset from node line (i, j) */
    double xin, etan;  /* node in that cell's reference coordinates */
    double phi0, phi1; /* angular sector of the disc inside that cell */
} sector_t;

static int node_sectors(int type, sector_t s[4]) {
    const double h = 0.5 * M_PI;
    if (type == ND_CORNER) {
        s[0] = (sector_t){0, 0, -1.0, -1.0, 0.0, h};
        s[1] = (sector_t){-1, 0, 1.0, -1.0, h, 2.0 * h};
        s[2] = (sector_t){-1, -1, 1.0, 1.0, 2.0 * h, 3.0 * h};
        s[3] = (sector_t){0, -1, -1.0, 1.0, 3.0 * h, 4.0 * h};
        return 4;
    }
    if (type == ND_XMID) {
        s[0] = (sector_t){0, 0, -1.0, 0.0, -h, h};
        s[1] = (sector_t){-1, 0, 1.0, 0.0, h, 3.0 * h};
        return 2;
    }
    s[0] = (sector_t){0, 0, 0.0, -1.0, 0.0, 2.0 * h};
    s[1] = (sector_t){0, -1, 0.0, 1.0, 2.0 * h, 4.0 * h};
    return 2;
}

static void acoustic_node(const lay_t *L, const double *patch, const orc_cfg *cf, int type, int i, int j,
                          double tau, double out[3]) {
    double R = cf->c * tau;
    sector_t sec[4];
    int ns = node_sectors(type, sec);
    double Mp = 0, RdMp = 0, Mu = 0, RdMu = 0, Mv = 0, RdMv = 0, Mdiv = 0, Mpx = 0, Mpy = 0;
    for (int k = 0; k < ns; ++k) {
        const sector_t *S = &sec[k];
        double qp[3][3], qu[3][3], qv[3][3], tp[3][3], tu[3][3], tv[3][3];
        cell_nodal(L, patch, 0, i + S->di, j + S->dj, qp);
        cell_nodal(L, patch, 1, i + S->di, j + S->dj, qu);
        cell_nodal(L, patch, 2, i + S->di, j + S->dj, qv);
        taylor(qp, S->xin, S->etan, cf->dx, cf->dy, tp);
        taylor(qu, S->xin, S->etan, cf->dx, cf->dy, tu);
        taylor(qv, S->xin, S->etan, cf->dx, cf->dy, tv);
        /* polynomial coefficients of div u = u_X + v_Y and of grad p */
        double tdiv[3][3] = {{0}}, tpx[3][3] = {{0}}, tpy[3][3] = {{0}};
        for (int m = 0; m < 3; ++m)
            for (int n = 0; n < 3; ++n) {
                double ux = (m + 1 < 3) ? (m + 1) * tu[m + 1][n] : 0.0;
                double vy = (n + 1 < 3) ? (n + 1) * tv[m][n + 1] : 0.0;
                tdiv[m][n] = ux + vy;
                tpx[m][n] = (m + 1 < 3) ? (m + 1) * tp[m + 1][n] : 0.0;
                tpy[m][n] = (n + 1 < 3) ? (n + 1) * tp[m][n + 1] : 0.0;
            }
        double M, RdM, dummy;
        sector_mean(tp, R, S->phi0, S->phi1, &M, &RdM); Mp += M; RdMp += RdM;
        sector_mean(tu, R, S->phi0, S->phi1, &M, &RdM); Mu += M; RdMu += RdM;
        sector_mean(tv, R, S->phi0, S->phi1, &M, &RdM); Mv += M; RdMv += RdM;
        sector_mean(tdiv, R, S->phi0, S->phi1, &M, &dummy); Mdiv += M;
        sector_mean(tpx, R, S->phi0, S->phi1, &M, &dummy); Mpx += M;
        sector_mean(tpy, R, S->phi0, S->phi1, &M, &dummy); Mpy += M;
    }
    /* Eq. ERFormula: M + R d_R M - R M{...} */
    out[0] = Mp + RdMp - R * Mdiv;
    out[1] = Mu + RdMu - R * Mpx;
    out[2] = Mv + RdMv - R * Mpy;
}

/* Point value of node (type, i, j) of one patch evolved by tau. */
static void evolve_node(const lay_t *L, const double *patch, const orc_cfg *cf, int type, int i, int j,
                        double tau, double *out) {
    if (cf->eq == EQ_ADVECTION) {
        for (int c = 0; c < L->ncomp; ++c) out[c] = advect_node(L, patch, c, cf, type, i, j, tau);
    } else {
        acoustic_node(L, patch, cf, type, i, j, tau, out);
    }
}

/* Exported for the pins. */
void orc_node_evolve(const orc_cfg *cf, const double *patch, int type, int i, int j, double tau, double *out) {
    lay_t L = lay_make(cf->n, cf->ncomp);
    evolve_node(&L, patch, cf, type, i, j, tau, out);
}

/* Physical fluxes f(q), g(q): advection f = a q, g = b q (Eq. advection2d);
 * acoustics for (p, u, v): f = c (u, p, 0), g = c (v, 0, p) (Eq. acoustics). */
static void phys_flux(const orc_cfg *cf, int dir, const double *q, double *f) {
    if (cf->eq == EQ_ADVECTION) {
        for (int c = 0; c < cf->ncomp; ++c) f[c] = (dir == 0 ? cf->a : cf->b) * q[c];
        return;
    }
    if (dir == 0) { f[0] = cf->c * q[1]; f[1] = cf->c * q[0]; f[2] = 0.0; }
    else          { f[0] = cf->c * q[2]; f[1] = 0.0;         f[2] = cf->c * q[0]; }
}

/* ------------------------------------------------------------- one patch step
 * One Active Flux step on one patch whose two ghost layers are filled
 * (Section 2 and Section 3.2): the interior and the first ghost layer are
 * advanced ("the first layer of ghost cells is updated along with all
 * interior cells"), i.e. the averages of cells [-1, N+1)^2 and every point
 * value on the boundary of those cells.
 *   1. point values at t^{n+1/2} and t^{n+1} from q^n (Eq. advection-update /
 *      Eq. ERFormula);
 *   2. numerical fluxes by the space-time Simpson rule (Eq. Simpson-2d and
 *      its analogue for G);
 *   3. conservative update (Eq. 2dfv).
 * `out` receives a copy of `in` with the updated entries replaced.  If freg is
 * not NULL, dt * F (resp. dt * G) on the four patch faces is ADDED to it:
 * freg[side][comp][k], side 0 = x-line 0, 1 = x-line N, 2 = y-line 0,
 * 3 = y-line N, k in [0, N) (Section 3.2, conservative fix).
 * Pinned by: the full step exact for Q2 data without x^2 y^2 (P3); constant
 * states and the rotating state u = w(-y, x) preserved (P6); mass conserved
 * (P7); third-order convergence and the paper's Table 1 (P10, P11).        */
void orc_step_patch(const orc_cfg *cf, const double *in, double *out, double *freg) {
    lay_t L = lay_make(cf->n, cf->ncomp);
    const int n = cf->n, nc = cf->ncomp;
    const int nl = n + 3; /* node lines -1 .. N+1 */
    memcpy(out, in, sizeof(double) * lay_patch_words(&L));

    /* q_node[time][type][comp][(j+1)*nl + (i+1)] */
    size_t per = (size_t)nl * nl;
    double *qn = (double *)calloc((size_t)3 * 3 * nc * per, sizeof(double));
#define QN(t, ty, c, i, j) qn[((((size_t)(t) * 3 + (ty)) * nc + (c)) * per) + (size_t)((j) + 1) * nl + ((i) + 1)]
    static const int plane_of[3] = {PL_CORNER, PL_XMID, PL_YMID};
    double v[3];
    for (int ty = 0; ty < 3; ++ty) {
        int imax = (ty == ND_YMID) ? n + 1 : n + 2; /* exclusive upper line / column */
        int jmax = (ty == ND_XMID) ? n + 1 : n + 2;
        for (int j = -1; j < jmax; ++j)
            for (int i = -1; i < imax; ++i) {
                for (int c = 0; c < nc; ++c) QN(0, ty, c, i, j) = PLc(&L, in, c, plane_of[ty])[IX(&L, i, j)];
                evolve_node(&L, in, cf, ty, i, j, 0.5 * cf->dt, v);
                for (int c = 0; c < nc; ++c) QN(1, ty, c, i, j) = v[c];
                evolve_node(&L, in, cf, ty, i, j, cf->dt, v);
                for (int c = 0; c < nc; ++c) QN(2, ty, c, i, j) = v[c];
            }
    }

    /* Eq. Simpson-2d: F at x-line i, row j; G at y-line j, column i. */
    const double wt[3] = {1.0, 4.0, 1.0};
    double *F = (double *)calloc((size_t)nc * per, sizeof(double));
    double *Gf = (double *)calloc((size_t)nc * per, sizeof(double));
#define FX(c, i, j) F[(size_t)(c) * per + (size_t)((j) + 1) * nl + ((i) + 1)]
#define GY(c, i, j) Gf[(size_t)(c) * per + (size_t)((j) + 1) * nl + ((i) + 1)]
    double q[3], f[3];
    for (int j = -1; j < n + 1; ++j)
        for (int i = -1; i < n + 2; ++i) {
            double acc[3] = {0, 0, 0};
            for (int t = 0; t < 3; ++t) {
                /* three face points: lower corner, midpoint, upper corner */
                for (int s = 0; s < 3; ++s) {
                    for (int c = 0; c < nc; ++c)
                        q[c] = (s == 0) ? QN(t, ND_CORNER, c, i, j)
                             : (s == 1) ? QN(t, ND_XMID, c, i, j)
                                        : QN(t, ND_CORNER, c, i, j + 1);
                    phys_flux(cf, 0, q, f);
                    for (int c = 0; c < nc; ++c) acc[c] += wt[t] * wt[s] * f[c];
                }
            }
            for (int c = 0; c < nc; ++c) FX(c, i, j) = acc[c] / 36.0;
        }
    for (int j = -1; j < n + 2; ++j)
        for (int i = -1; i < n + 1; ++i) {
            double acc[3] = {0, 0, 0};
            for (int t = 0; t < 3; ++t) {
                for (int s = 0; s < 3; ++s) {
                    for (int c = 0; c < nc; ++c)
                        q[c] = (s == 0) ? QN(t, ND_CORNER, c, i, j)
                             : (s == 1) ? QN(t, ND_YMID, c, i, j)
                                        : QN(t, ND_CORNER, c, i + 1, j);
                    phys_flux(cf, 1, q, f);
                    for (int c = 0; c < nc; ++c) acc[c] += wt[t] * wt[s] * f[c];
                }
            }
            for (int c = 0; c < nc; ++c) GY(c, i, j) = acc[c] / 36.0;
        }

    /* Eq. 2dfv on cells [-1, N+1)^2 */
    for (int c = 0; c < nc; ++c) {
        const double *ain = PLc(&L, in, c, PL_AVG);
        double *aout = PL(&L, out, c, PL_AVG);
        for (int j = -1; j < n + 1; ++j)
            for (int i = -1; i < n + 1; ++i)
                aout[IX(&L, i, j)] = ain[IX(&L, i, j)] - cf->dt / cf->dx * (FX(c, i + 1, j) - FX(c, i, j)) -
                                     cf->dt / cf->dy * (GY(c, i, j + 1) - GY(c, i, j));
    }
    /* new point values */
    for (int ty = 0; ty < 3; ++ty) {
        int imax = (ty == ND_YMID) ? n + 1 : n + 2;
        int jmax = (ty == ND_XMID) ? n + 1 : n + 2;
        for (int c = 0; c < nc; ++c) {
            double *pl = PL(&L, out, c, plane_of[ty]);
            for (int j = -1; j < jmax; ++j)
                for (int i = -1; i < imax; ++i) pl[IX(&L, i, j)] = QN(2, ty, c, i, j);
        }
    }
    if (freg) {
        for (int c = 0; c < nc; ++c)
            for (int k = 0; k < n; ++k) {
                freg[(0 * nc + c) * n + k] += cf->dt * FX(c, 0, k);
                freg[(1 * nc + c) * n + k] += cf->dt * FX(c, n, k);
                freg[(2 * nc + c) * n + k] += cf->dt * GY(c, k, 0);
                freg[(3 * nc + c) * n + k] += cf->dt * GY(c, k, n);
            }
    }
#undef QN
#undef FX
#undef GY
    free(qn);
    free(F);
    free(Gf);
}

/* ------------------------------------------- Sections 4.2 and 4.3 (variable
 * velocity) ------------------------------------------------------------------
 * q_t + (a q)_x + (b q)_y = 0 with a divergence-free velocity, one component.
 *   field 0, solid-body rotation (Section 4.2, Eq. solidbodyODE):
 *     a = -pi y, b = pi x; the characteristics are rotations about the origin
 *     (Eq. characteristics_advtwo), so the foot of a node traced back by tau
 *     is the node rotated by -pi tau.  Flux through an x-face: Simpson's rule
 *     in y and t of a(x_face, y) q(x_face, y, t) -- the velocity at each of
 *     the three face points, constant in time.
 *   field 1, swirl (Section 4.3): stream function
 *     Psi = sin^2(pi x) sin^2(pi y) cos(pi t) / pi, velocities by the
 *     centred differences of Eq. swirlODE over one mesh width; the foot is
 *     found by one classical Runge-Kutta step of size -tau; flux through an
 *     x-face by Eq. swirlF: at each time level the velocity at the face
 *     centre times Simpson's rule of q along the face (likewise Eq. swirlG).
 * Positions are physical: x0, y0 locate node line 0 of the patch.
 * Pinned by: exact rotation of quadratic data (solid body), constant states
 * preserved (Remark of Section 4.2, Theorem of Section 4.3), third-order
 * convergence, and Table 3 of the paper (swirl).                            */
void orc_fill_periodic(int n, int ncomp, int px, int py, double *state);

typedef struct {
    int32_t n;
    int32_t field; /* 0 solid-body rotation, 1 swirl */
    double dx, dy, dt;
    double x0, y0; /* position of node line 0 (lower-left corner of cell 0) */
    double t;      /* time t^n */
} orc_var;

static double swirl_psi(double x, double y, double t) {
    double sx = sin(M_PI * x), sy = sin(M_PI * y);
    return sx * sx * sy * sy * cos(M_PI * t) / M_PI;
}

/* Velocity (a, b) at (x, y, t). */
static void var_velocity(const orc_var *v, double x, double y, double t, double *a, double *b) {
    if (v->field == 0) {
        *a = -M_PI * y;
        *b = M_PI * x;
        return;
    }
    *a = -(swirl_psi(x, y + 0.5 * v->dy, t) - swirl_psi(x, y - 0.5 * v->dy, t)) / v->dy;
    *b = (swirl_psi(x + 0.5 * v->dx, y, t) - swirl_psi(x - 0.5 * v->dx, y, t)) / v->dx;
}

/* Foot at time t^n of the characteristic through (x, y) at t^n + tau. */
static void var_foot(const orc_var *v, double x, double y, double tau, double *xf, double *yf) {
    if (v->field == 0) {
        double c = cos(M_PI * tau), s = sin(M_PI * tau);
        *xf = x * c + y * s;
        *yf = -x * s + y * c;
        return;
    }
    double h = -tau, t1 = v->t + tau;
    double k1a, k1b, k2a, k2b, k3a, k3b, k4a, k4b;
    var_velocity(v, x, y, t1, &k1a, &k1b);
    var_velocity(v, x + 0.5 * h * k1a, y + 0.5 * h * k1b, t1 + 0.5 * h, &k2a, &k2b);
    var_velocity(v, x + 0.5 * h * k2a, y + 0.5 * h * k2b, t1 + 0.5 * h, &k3a, &k3b);
    var_velocity(v, x + h * k3a, y + h * k3b, t1 + h, &k4a, &k4b);
    *xf = x + h / 6.0 * (k1a + 2.0 * k2a + 2.0 * k3a + k4a);
    *yf = y + h / 6.0 * (k1b + 2.0 * k2b + 2.0 * k3b + k4b);
}

/* Value of q^n at (xf, yf): the reconstruction of the cell holding it. */
static double var_eval(const lay_t *L, const double *patch, const orc_var *v, double xf, double yf) {
    double fx = (xf - v->x0) / v->dx, fy = (yf - v->y0) / v->dy;
    double kx = floor(fx), ky = floor(fy);
    int ci = (int)kx, cj = (int)ky;
    if (ci < -NG) ci = -NG;
    if (ci > L->n + NG - 1) ci = L->n + NG - 1;
    if (cj < -NG) cj = -NG;
    if (cj > L->n + NG - 1) cj = L->n + NG - 1;
    double xi = 2.0 * (fx - ci) - 1.0, eta = 2.0 * (fy - cj) - 1.0;
    double q[3][3];
    cell_nodal(L, patch, 0, ci, cj, q);
    return recon_deriv(q, xi, eta, 0, 0);
}

/* Position of node (type, i, j). */
static void var_node_xy(const orc_var *v, int type, int i, int j, double *x, double *y) {
    *x = v->x0 + ((double)i + (type == ND_YMID ? 0.5 : 0.0)) * v->dx;
    *y = v->y0 + ((double)j + (type == ND_XMID ? 0.5 : 0.0)) * v->dy;
}

/* Exported for the pins: the velocity and the characteristic foot. */
void orc_var_velocity(const orc_var *v, double x, double y, double t, double *ab) {
    var_velocity(v, x, y, t, &ab[0], &ab[1]);
}
void orc_var_foot(const orc_var *v, double x, double y, double tau, double *xy) {
    var_foot(v, x, y, tau, &xy[0], &xy[1]);
}

/* Exported for the pins: node (type, i, j) of one patch evolved by tau. */
double orc_node_evolve_var(const orc_var *v, const double *patch, int type, int i, int j, double tau) {
    lay_t L = lay_make(v->n, 1);
    double x, y, xf, yf;
    var_node_xy(v, type, i, j, &x, &y);
    var_foot(v, x, y, tau, &xf, &yf);
    return var_eval(&L, patch, v, xf, yf);
}

/* One step of one patch, as orc_step_patch (same entries advanced, same flux
 * registers) with the fluxes described above. */
void orc_step_patch_var(const orc_var *v, const double *in, double *out, double *freg) {
    lay_t L = lay_make(v->n, 1);
    const int n = v->n, nl = n + 3;
    memcpy(out, in, sizeof(double) * lay_patch_words(&L));
    size_t per = (size_t)nl * nl;
    double *qn = (double *)calloc((size_t)3 * 3 * per, sizeof(double));
#define QV(t, ty, i, j) qn[(((size_t)(t) * 3 + (ty)) * per) + (size_t)((j) + 1) * nl + ((i) + 1)]
    static const int plane_of[3] = {PL_CORNER, PL_XMID, PL_YMID};
    for (int ty = 0; ty < 3; ++ty) {
        int imax = (ty == ND_YMID) ? n + 1 : n + 2;
        int jmax = (ty == ND_XMID) ? n + 1 : n + 2;
        for (int j = -1; j < jmax; ++j)
            for (int i = -1; i < imax; ++i) {
                double x, y, xf, yf;
                var_node_xy(v, ty, i, j, &x, &y);
                QV(0, ty, i, j) = PLc(&L, in, 0, plane_of[ty])[IX(&L, i, j)];
                var_foot(v, x, y, 0.5 * v->dt, &xf, &yf);
                QV(1, ty, i, j) = var_eval(&L, in, v, xf, yf);
                var_foot(v, x, y, v->dt, &xf, &yf);
                QV(2, ty, i, j) = var_eval(&L, in, v, xf, yf);
            }
    }
    const double wt[3] = {1.0, 4.0, 1.0};
    const double tk[3] = {v->t, v->t + 0.5 * v->dt, v->t + v->dt};
    double *F = (double *)calloc(per, sizeof(double));
    double *G = (double *)calloc(per, sizeof(double));
    for (int j = -1; j < n + 1; ++j)
        for (int i = -1; i < n + 2; ++i) {
            double xs = v->x0 + i * v->dx;
            double ys[3] = {v->y0 + j * v->dy, v->y0 + (j + 0.5) * v->dy, v->y0 + (j + 1) * v->dy};
            double acc = 0.0;
            for (int t = 0; t < 3; ++t) {
                double q[3] = {QV(t, ND_CORNER, i, j), QV(t, ND_XMID, i, j), QV(t, ND_CORNER, i, j + 1)};
                if (v->field == 0) {
                    for (int s = 0; s < 3; ++s) {
                        double a, b;
                        var_velocity(v, xs, ys[s], tk[t], &a, &b);
                        acc += wt[t] * wt[s] * a * q[s];
                    }
                } else {
                    double a, b;
                    var_velocity(v, xs, ys[1], tk[t], &a, &b);
                    acc += wt[t] * a * (q[0] + 4.0 * q[1] + q[2]);
                }
            }
            F[(size_t)(j + 1) * nl + (i + 1)] = acc / 36.0;
        }
    for (int j = -1; j < n + 2; ++j)
        for (int i = -1; i < n + 1; ++i) {
            double ys = v->y0 + j * v->dy;
            double xs[3] = {v->x0 + i * v->dx, v->x0 + (i + 0.5) * v->dx, v->x0 + (i + 1) * v->dx};
            double acc = 0.0;
            for (int t = 0; t < 3; ++t) {
                double q[3] = {QV(t, ND_CORNER, i, j), QV(t, ND_YMID, i, j), QV(t, ND_CORNER, i + 1, j)};
                if (v->field == 0) {
                    for (int s = 0; s < 3; ++s) {
                        double a, b;
                        var_velocity(v, xs[s], ys, tk[t], &a, &b);
                        acc += wt[t] * wt[s] * b * q[s];
                    }
                } else {
                    double a, b;
                    var_velocity(v, xs[1], ys, tk[t], &a, &b);
                    acc += wt[t] * b * (q[0] + 4.0 * q[1] + q[2]);
                }
            }
            G[(size_t)(j + 1) * nl + (i + 1)] = acc / 36.0;
        }
#define FV(i, j) F[(size_t)((j) + 1) * nl + ((i) + 1)]
#define GV(i, j) G[(size_t)((j) + 1) * nl + ((i) + 1)]
    const double *ain = PLc(&L, in, 0, PL_AVG);
    double *aout = PL(&L, out, 0, PL_AVG);
    for (int j = -1; j < n + 1; ++j)
        for (int i = -1; i < n + 1; ++i)
            aout[IX(&L, i, j)] = ain[IX(&L, i, j)] - v->dt / v->dx * (FV(i + 1, j) - FV(i, j)) -
                                 v->dt / v->dy * (GV(i, j + 1) - GV(i, j));
    for (int ty = 0; ty < 3; ++ty) {
        int imax = (ty == ND_YMID) ? n + 1 : n + 2;
        int jmax = (ty == ND_XMID) ? n + 1 : n + 2;
        double *pl = PL(&L, out, 0, plane_of[ty]);
        for (int j = -1; j < jmax; ++j)
            for (int i = -1; i < imax; ++i) pl[IX(&L, i, j)] = QV(2, ty, i, j);
    }
    if (freg)
        for (int k = 0; k < n; ++k) {
            freg[0 * n + k] += v->dt * FV(0, k);
            freg[1 * n + k] += v->dt * FV(n, k);
            freg[2 * n + k] += v->dt * GV(k, 0);
            freg[3 * n + k] += v->dt * GV(k, n);
        }
#undef QV
#undef FV
#undef GV
    free(qn);
    free(F);
    free(G);
}

/* Uniform periodic run with variable velocity: px x py patches tiling the box
 * with lower-left corner (lo_x, lo_y); v->t is the start time and advances. */
void orc_run_uniform_var(orc_var *v, int px, int py, double lo_x, double lo_y, int nsteps, double *state,
                         double *tmp, int nthreads) {
    lay_t L = lay_make(v->n, 1);
    long pw = lay_patch_words(&L);
    int np = px * py;
    (void)nthreads;
    for (int s = 0; s < nsteps; ++s) {
        orc_fill_periodic(v->n, 1, px, py, state);
#pragma omp parallel for num_threads(nthreads) schedule(dynamic, 1)
        for (int p = 0; p < np; ++p) {
            orc_var vp = *v;
            vp.x0 = lo_x + (p % px) * v->n * v->dx;
            vp.y0 = lo_y + (p / px) * v->n * v->dy;
            orc_step_patch_var(&vp, state + p * pw, tmp + p * pw, NULL);
        }
        memcpy(state, tmp, sizeof(double) * pw * np);
        v->t += v->dt;
    }
}

/* --------------------------------------------------------- Section 3.1 (3.)
 * Same-level ghost fill on a px x py array of patches tiling a periodic box:
 * every ghost entry (lattice entries outside [g, g+N)^2 of every plane) is a
 * copy of the entry owned by the neighbouring patch at the same position.
 * Pinned by: ghost entries equal the analytic values at the wrapped
 * positions; one patch equals many (P9).                                   */
void orc_fill_periodic(int n, int ncomp, int px, int py, double *state) {
    lay_t L = lay_make(n, ncomp);
    long pw = lay_patch_words(&L);
    int gx = px * n, gy = py * n;
    for (int p = 0; p < px * py; ++p) {
        int ix = p % px, iy = p / px;
        for (int c = 0; c < ncomp; ++c)
            for (int k = 0; k < 4; ++k) {
                double *dst = PL(&L, state + p * pw, c, k);
                for (int J = 0; J < L.w; ++J)
                    for (int I = 0; I < L.w; ++I) {
                        int li = I - NG, lj = J - NG;
                        if (li >= 0 && li < n && lj >= 0 && lj < n) continue;
                        int gi = ((ix * n + li) % gx + gx) % gx;
                        int gj = ((iy * n + lj) % gy + gy) % gy;
                        int sp = (gj / n) * px + gi / n;
                        const double *src = PLc(&L, state + sp * pw, c, k);
                        dst[(long)J * L.w + I] = src[IX(&L, gi % n, gj % n)];
                    }
            }
    }
}

/* Uniform periodic run: nsteps x (fill ghosts, step every patch).  `tmp` has
 * the size of `state`.  OpenMP over patches with `nthreads` threads.
 * Pinned by: one patch equals many (P9); mass conserved (P7); convergence
 * and the paper's Table 1 (P10, P11).                                      */
void orc_run_uniform(const orc_cfg *cf, int px, int py, int nsteps, double *state, double *tmp, int nthreads) {
    lay_t L = lay_make(cf->n, cf->ncomp);
    long pw = lay_patch_words(&L);
    int np = px * py;
    (void)nthreads;
    for (int s = 0; s < nsteps; ++s) {
        orc_fill_periodic(cf->n, cf->ncomp, px, py, state);
#pragma omp parallel for num_threads(nthreads) schedule(dynamic, 1)
        for (int p = 0; p < np; ++p) orc_step_patch(cf, state + p * pw, tmp + p * pw, NULL);
        memcpy(state, tmp, sizeof(double) * pw * np);
    }
}

/* One step of the patches idx[0..np) of a state of `words`-word patches,
 * each patch independent of the others (its ghost ring already filled):
 * the loop of the adaptive driver over the leaves of one level, with OpenMP
 * over patches.  freg: flux registers of `rwords` words per patch, or NULL.
 * var: NULL for constant coefficients (cf), else the variable-velocity
 * configuration, with x0[k], y0[k] the position of patch idx[k]. */
void orc_step_patches(const orc_cfg *cf, const orc_var *var, const double *x0, const double *y0, int np,
                      const int32_t *idx, long words, double *state, double *freg, long rwords, int nthreads) {
    double *tmp = (double *)malloc(sizeof(double) * (size_t)words * (size_t)(np > 0 ? np : 1));
#pragma omp parallel for num_threads(nthreads) schedule(dynamic, 1)
    for (int k = 0; k < np; ++k) {
        const long p = idx[k];
        double *fr = freg ? freg + p * rwords : NULL;
        if (var) {
            orc_var vp = *var;
            vp.x0 = x0[k];
            vp.y0 = y0[k];
            orc_step_patch_var(&vp, state + p * words, tmp + (long)k * words, fr);
        } else {
            orc_step_patch(cf, state + p * words, tmp + (long)k * words, fr);
        }
    }
    for (int k = 0; k < np; ++k) memcpy(state + (long)idx[k] * words, tmp + (long)k * words, sizeof(double) * words);
    free(tmp);
}

int orc_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* =========================================================================
 * Adaptive mesh refinement (Section 3): a forest of quadtrees over a B x B
 * brick of level-0 patches, periodic in both directions.  Every leaf is a
 * patch of N x N cells; level l+1 halves the mesh width (2:1 ratio).
 *
 * Positions are integers: the unit is half the cell width of level lmax, so
 * a level-l cell is 2^(lmax-l+1) units wide and every node, cell centre and
 * Simpson point used below is an exact integer (no rounding in lookups).
 * ========================================================================= */
typedef struct {
    int n, ncomp, nleaf, B, lmax;
    const int32_t *level, *ix, *iy;
    int32_t **map; /* map[l][iy * (B << l) + ix] = leaf index or -1 */
    long D;        /* domain width in units */
} forest_t;

static long hw_of(const forest_t *F, int l) { return 2L << (F->lmax - l); }

static int forest_init(forest_t *F, int n, int ncomp, int nleaf, const int32_t *level, const int32_t *ix,
                       const int32_t *iy, int B, int lmax) {
    F->n = n; F->ncomp = ncomp; F->nleaf = nleaf; F->B = B; F->lmax = lmax;
    F->level = level; F->ix = ix; F->iy = iy;
    F->D = (long)B * n * hw_of(F, 0);
    F->map = (int32_t **)calloc((size_t)lmax + 1, sizeof(int32_t *));
    for (int l = 0; l <= lmax; ++l) {
        long side = (long)B << l;
        F->map[l] = (int32_t *)malloc(sizeof(int32_t) * side * side);
        for (long k = 0; k < side * side; ++k) F->map[l][k] = -1;
    }
    for (int p = 0; p < nleaf; ++p) {
        if (level[p] < 0 || level[p] > lmax) return -1;
        long side = (long)B << level[p];
        F->map[level[p]][(long)iy[p] * side + ix[p]] = p;
    }
    return 0;
}

static void forest_free(forest_t *F) {
    for (int l = 0; l <= F->lmax; ++l) free(F->map[l]);
    free(F->map);
}

static long wrapD(const forest_t *F, long x) { long r = x % F->D; return r < 0 ? r + F->D : r; }

/* Leaf covering the point (x, y) with half-open patch extents [x0, x1). */
static int forest_lookup(const forest_t *F, long x, long y) {
    x = wrapD(F, x); y = wrapD(F, y);
    for (int l = F->lmax; l >= 0; --l) {
        long pw = (long)F->n * hw_of(F, l), side = (long)F->B << l;
        int q = F->map[l][(y / pw) * side + (x / pw)];
        if (q >= 0) return q;
    }
    return -1;
}

static long leaf_x0(const forest_t *F, int p) { return (long)F->ix[p] * F->n * hw_of(F, F->level[p]); }
static long leaf_y0(const forest_t *F, int p) { return (long)F->iy[p] * F->n * hw_of(F, F->level[p]); }

/* offset of (x) relative to the origin of leaf q, unwrapping the periodic box */
static long rel(const forest_t *F, long x, long x0) {
    long d = wrapD(F, x - x0);
    if (d > F->D / 2) d -= F->D;
    return d;
}

static int node_owner(const forest_t *F, long x, long y);
static double leaf_entry(const forest_t *F, const double *state, int q, int c, int plane, long x, long y);

/* Value of the reconstruction (Eq. poly) of leaf q, component c, at (x, y).
 * The cell is found with the half-open rule, clamped into q's interior;
 * the reconstruction is continuous, so a point on a cell face may use
 * either neighbour.  Every point value of the cell is its owner's (see
 * node_owner), so nodes on q's boundary lines are read from the leaf that
 * owns them. */
static double leaf_eval(const forest_t *F, const double *state, int q, int c, long x, long y) {
    lay_t L = lay_make(F->n, F->ncomp);
    const double *patch = state + (long)q * lay_patch_words(&L);
    long hw = hw_of(F, F->level[q]);
    long x0 = leaf_x0(F, q), y0 = leaf_y0(F, q);
    long dx = rel(F, x, x0), dy = rel(F, y, y0);
    long ci = dx >= 0 ? dx / hw : -((-dx + hw - 1) / hw);
    long cj = dy >= 0 ? dy / hw : -((-dy + hw - 1) / hw);
    if (ci < 0) ci = 0;
    if (ci > F->n - 1) ci = F->n - 1;
    if (cj < 0) cj = 0;
    if (cj > F->n - 1) cj = F->n - 1;
    double xi = 2.0 * (double)(dx - ci * hw) / (double)hw - 1.0;
    double eta = 2.0 * (double)(dy - cj * hw) / (double)hw - 1.0;
    double qn[3][3];
    /* nodes at reference (a-1, b-1): positions x0 + ci hw + a hw/2 */
    for (int b = 0; b < 3; ++b)
        for (int a = 0; a < 3; ++a) {
            if (a == 1 && b == 1) continue;
            long px = x0 + ci * hw + a * hw / 2, py = y0 + cj * hw + b * hw / 2;
            int o = node_owner(F, px, py);
            int plane = (a == 1) ? PL_YMID : (b == 1 ? PL_XMID : PL_CORNER);
            if (o >= 0 && F->level[o] > F->level[q]) plane = PL_CORNER; /* finer owner: its vertex */
            qn[b][a] = leaf_entry(F, state, o >= 0 ? o : q, c, plane, px, py);
        }
    double rest = 0.0;
    for (int b = 0; b < 3; ++b)
        for (int a = 0; a < 3; ++a)
            if (!(a == 1 && b == 1)) rest += SIMPSON_W[a] * SIMPSON_W[b] * qn[b][a];
    qn[1][1] = (PLc(&L, patch, c, PL_AVG)[IX(&L, (int)ci, (int)cj)] - rest) / (SIMPSON_W[1] * SIMPSON_W[1]);
    return recon_deriv(qn, xi, eta, 0, 0);
}

/* Entry of leaf q in `plane` at the lattice position of point (x, y) (which
 * must be a lattice point of that plane for q). */
static double leaf_entry(const forest_t *F, const double *state, int q, int c, int plane, long x, long y) {
    lay_t L = lay_make(F->n, F->ncomp);
    const double *patch = state + (long)q * lay_patch_words(&L);
    long hw = hw_of(F, F->level[q]);
    long dx = rel(F, x, leaf_x0(F, q)), dy = rel(F, y, leaf_y0(F, q));
    if (plane == PL_AVG || plane == PL_YMID) dx -= hw / 2;
    if (plane == PL_AVG || plane == PL_XMID) dy -= hw / 2;
    int i = (int)(dx / hw), j = (int)(dy / hw);
    return PLc(&L, patch, c, plane)[IX(&L, i, j)];
}

/* Position (units) of lattice entry (plane, i, j) of leaf p. */
static void entry_pos(const forest_t *F, int p, int plane, int i, int j, long *x, long *y) {
    long hw = hw_of(F, F->level[p]);
    *x = leaf_x0(F, p) + (long)i * hw + ((plane == PL_AVG || plane == PL_YMID) ? hw / 2 : 0);
    *y = leaf_y0(F, p) + (long)j * hw + ((plane == PL_AVG || plane == PL_XMID) ? hw / 2 : 0);
}

/* Section 3.1: value of a ghost entry of leaf p from the leaf q covering it.
 *  same level: copy;
 *  q finer (fine -> coarse): the average is the mean of the four fine cell
 *    averages, a point value is copied from the coinciding fine vertex;
 *  q coarser (coarse -> fine): point values are the coarse reconstruction
 *    evaluated at the point, the average is Simpson's rule over the fine
 *    cell applied to that reconstruction (exact for it). */
static double transfer_value(const forest_t *F, const double *state, int lp, int q, int c, int plane, long x,
                             long y) {
    int lq = F->level[q];
    if (lq == lp) return leaf_entry(F, state, q, c, plane, x, y);
    if (lq > lp) {
        if (plane == PL_AVG) {
            long h = hw_of(F, lq) / 2; /* fine half width: fine centres at x +- h */
            return 0.25 * (leaf_entry(F, state, q, c, PL_AVG, x - h, y - h) +
                           leaf_entry(F, state, q, c, PL_AVG, x + h, y - h) +
                           leaf_entry(F, state, q, c, PL_AVG, x - h, y + h) +
                           leaf_entry(F, state, q, c, PL_AVG, x + h, y + h));
        }
        return leaf_entry(F, state, q, c, PL_CORNER, x, y);
    }
    if (plane != PL_AVG) return leaf_eval(F, state, q, c, x, y);
    long h = hw_of(F, lp) / 2; /* half width of the fine (destination) cell */
    double s = 0.0;
    for (int b = 0; b < 3; ++b)
        for (int a = 0; a < 3; ++a)
            s += SIMPSON_W[a] * SIMPSON_W[b] * leaf_eval(F, state, q, c, x + (a - 1) * h, y + (b - 1) * h);
    return s;
}

/* Which leaf's value a point value takes.  A node on the boundary between
 * leaves of different levels takes the value of the finest leaf touching it
 * (Section 3.2: the fluxes, and hence the face values, of "the more resolved
 * grid" are used at coarse-fine interfaces); among equally fine leaves the
 * one above-right, above-left, below-right, below-left of the point is used,
 * in that order.  A cell average belongs to the leaf covering its centre.  */
static int node_owner(const forest_t *F, long x, long y) {
    int cand[4] = {forest_lookup(F, x, y), forest_lookup(F, x - 1, y), forest_lookup(F, x, y - 1),
                   forest_lookup(F, x - 1, y - 1)};
    int best = cand[0];
    for (int k = 1; k < 4; ++k)
        if (cand[k] >= 0 && (best < 0 || F->level[cand[k]] > F->level[best])) best = cand[k];
    return best;
}

static int entry_owner(const forest_t *F, int plane, long x, long y) {
    return plane == PL_AVG ? forest_lookup(F, x, y) : node_owner(F, x, y);
}

/* Ghost exchange of Section 3.1 / 3.2 on a forest.
 * Destination leaves: those whose level bit is set in dst_levels.  Every
 * entry of a destination leaf whose owner (entry_owner) is another leaf is
 * replaced by the owner's data, transferred by transfer_value, provided the
 * owner's level bit is set in src_levels (time-synchronised levels) and, if
 * same_only, the owner has the destination's level (the copy done before
 * every step of a level).  This covers the ghost ring and the nodes on a
 * leaf's left / bottom face that a finer neighbour owns.  Entries the step
 * never reads (the average and bottom-mid of the far column, the average and
 * left-mid of the far row) are skipped.
 * The exchange runs in three passes, each reading the result of the one
 * before: entries owned by finer leaves, then by same-level leaves, then by
 * coarser leaves; so a coarse reconstruction used for interpolation already
 * carries the fine values on its coarse-fine faces.  Results are written to
 * `out` (a copy of `in` on entry).
 * Pinned by: coarse-to-fine interpolation exact for biquadratic data and
 * conservative (P8); a same-level forest equals the uniform run (P9).      */
void orc_fill_amr(int n, int ncomp, int nleaf, const int32_t *level, const int32_t *ix, const int32_t *iy,
                  int B, int lmax, uint32_t dst_levels, uint32_t src_levels, int same_only, const double *in,
                  double *out) {
    forest_t F;
    lay_t L = lay_make(n, ncomp);
    long pw = lay_patch_words(&L);
    memcpy(out, in, sizeof(double) * pw * nleaf);
    if (forest_init(&F, n, ncomp, nleaf, level, ix, iy, B, lmax) != 0) { forest_free(&F); return; }
    double *prev = (double *)malloc(sizeof(double) * pw * nleaf);
    for (int pass = 0; pass < 3; ++pass) { /* 0: finer owner, 1: same level, 2: coarser */
        memcpy(prev, out, sizeof(double) * pw * nleaf);
        /* every leaf writes only its own ghost entries, read from prev */
#pragma omp parallel for schedule(dynamic, 4)
        for (int p = 0; p < nleaf; ++p) {
            int lp = level[p];
            if (!((dst_levels >> lp) & 1u)) continue;
            for (int k = 0; k < 4; ++k)
                for (int j = -NG; j <= n + NG; ++j)
                    for (int i = -NG; i <= n + NG; ++i) {
                        if (i > 0 && i < n && j > 0 && j < n) continue; /* strictly inside: own */
                        if (i == n + NG && (k == PL_AVG || k == PL_YMID)) continue;
                        if (j == n + NG && (k == PL_AVG || k == PL_XMID)) continue;
                        long x, y;
                        entry_pos(&F, p, k, i, j, &x, &y);
                        int q = entry_owner(&F, k, x, y);
                        if (q < 0 || q == p) continue;
                        int lq = level[q];
                        int rel_pass = lq > lp ? 0 : (lq == lp ? 1 : 2);
                        if (rel_pass != pass) continue;
                        if (!((src_levels >> lq) & 1u)) continue;
                        if (same_only && lq != lp) continue;
                        for (int c = 0; c < ncomp; ++c)
                            PL(&L, out + p * pw, c, k)[IX(&L, i, j)] = transfer_value(&F, prev, lp, q, c, k, x, y);
                    }
        }
    }
    free(prev);
    forest_free(&F);
}

/* Section 3.2, "Global conservation property": Berger-Colella correction.
 * For every coarse leaf C at level l with l and l+1 both synchronised, and
 * every face k of C whose neighbour across is a finer leaf F, the coarse
 * average next to the face is corrected so that it has used the fine fluxes:
 *   right/top face:  dQ = (R_C - (R_F,a + R_F,b) / 2) / h_C
 *   left/bottom face: dQ = ((R_F,a + R_F,b) / 2 - R_C) / h_C
 * where R = sum over the steps since the last synchronisation of dt * F
 * (registers filled by orc_step_patch; the fine one spans two fine steps and
 * two fine faces), h_C the coarse mesh width normal to the face.  Consumed
 * register entries (both sides) are reset to zero.
 * Pinned by: mass conserved to round-off across coarse-fine faces with
 * subcycling, and not without the fix (P7).                                */
void orc_reflux_amr(int n, int ncomp, int nleaf, const int32_t *level, const int32_t *ix, const int32_t *iy,
                    int B, int lmax, uint32_t sync_levels, double dx0, double dy0, double *freg, double *state) {
    forest_t F;
    lay_t L = lay_make(n, ncomp);
    long pw = lay_patch_words(&L);
    if (forest_init(&F, n, ncomp, nleaf, level, ix, iy, B, lmax) != 0) { forest_free(&F); return; }
    long rw = 4L * ncomp * n; /* register words per patch */
    /* collect corrections first so consumption order does not matter */
    double *dq = (double *)calloc((size_t)nleaf * ncomp * n * n, sizeof(double));
    unsigned char *used = (unsigned char *)calloc((size_t)nleaf * rw, 1);
    for (int p = 0; p < nleaf; ++p) {
        int l = level[p];
        if (!((sync_levels >> l) & 1u) || !((sync_levels >> (l + 1)) & 1u)) continue;
        long hw = hw_of(&F, l), x0 = leaf_x0(&F, p), y0 = leaf_y0(&F, p);
        long x1 = x0 + (long)n * hw, y1 = y0 + (long)n * hw;
        double hx = dx0 / (double)(1L << l), hy = dy0 / (double)(1L << l);
        for (int side = 0; side < 4; ++side)
            for (int k = 0; k < n; ++k) {
                long px, py; /* a point just across the middle of face k */
                if (side == 0) { px = x0 - 1; py = y0 + k * hw + hw / 2; }
                else if (side == 1) { px = x1; py = y0 + k * hw + hw / 2; }
                else if (side == 2) { px = x0 + k * hw + hw / 2; py = y0 - 1; }
                else { px = x0 + k * hw + hw / 2; py = y1; }
                int q = forest_lookup(&F, px, py);
                if (q < 0 || level[q] != l + 1) continue;
                long hf = hw_of(&F, l + 1);
                int fside = side ^ 1; /* opposite side of the fine leaf */
                long start = (side < 2) ? rel(&F, y0 + k * hw, leaf_y0(&F, q)) : rel(&F, x0 + k * hw, leaf_x0(&F, q));
                int kf = (int)(start / hf);
                int ci = (side == 0) ? 0 : (side == 1 ? n - 1 : k);
                int cj = (side == 2) ? 0 : (side == 3 ? n - 1 : k);
                double h = (side < 2) ? hx : hy;
                for (int c = 0; c < ncomp; ++c) {
                    double rc = freg[p * rw + ((long)side * ncomp + c) * n + k];
                    double rf = 0.5 * (freg[q * rw + ((long)fside * ncomp + c) * n + kf] +
                                       freg[q * rw + ((long)fside * ncomp + c) * n + kf + 1]);
                    double d = (side == 1 || side == 3) ? (rc - rf) / h : (rf - rc) / h;
                    dq[(((long)p * ncomp + c) * n + cj) * n + ci] += d;
                    used[p * rw + ((long)side * ncomp + c) * n + k] = 1;
                    used[q * rw + ((long)fside * ncomp + c) * n + kf] = 1;
                    used[q * rw + ((long)fside * ncomp + c) * n + kf + 1] = 1;
                }
            }
    }
    for (int p = 0; p < nleaf; ++p)
        for (int c = 0; c < ncomp; ++c) {
            double *avg = PL(&L, state + p * pw, c, PL_AVG);
            for (int j = 0; j < n; ++j)
                for (int i = 0; i < n; ++i) avg[IX(&L, i, j)] += dq[(((long)p * ncomp + c) * n + j) * n + i];
        }
    for (long e = 0; e < (long)nleaf * rw; ++e)
        if (used[e]) freg[e] = 0.0;
    free(dq);
    free(used);
    forest_free(&F);
}

/* Refinement indicator of every patch (Section 3: criteria applied to the
 * solution on each quadrant).  kind 0: max - min of the interior cell
 * averages of component `comp` (Section 4.1, Section 4.5.2); kind 1: largest
 * centred difference quotient |Q_{i+1,j} - Q_{i-1,j}| / (2 dx) or
 * |Q_{i,j+1} - Q_{i,j-1}| / (2 dy) over cells whose two neighbours are both
 * interior (Section 4.4).  tag = 1 if indicator >= refine_thr, -1 if
 * indicator < coarsen_thr, else 0.
 * Pinned by: the indicators of linear data (range and slope) and the exact
 * centred quotient 2x of quadratic data; the threshold rule at its boundaries
 * (test_oracle_tag_regrid.py).                                                */
void orc_tag(int n, int ncomp, int nleaf, const int32_t *level, const double *state, int comp, int kind,
             double dx0, double dy0, double refine_thr, double coarsen_thr, int8_t *tags, double *ind) {
    lay_t L = lay_make(n, ncomp);
    long pw = lay_patch_words(&L);
    for (int p = 0; p < nleaf; ++p) {
        const double *a = PLc(&L, state + p * pw, comp, PL_AVG);
        double v;
        if (kind == 0) {
            double mx = -INFINITY, mn = INFINITY;
            for (int j = 0; j < n; ++j)
                for (int i = 0; i < n; ++i) {
                    double q = a[IX(&L, i, j)];
                    if (q > mx) mx = q;
                    if (q < mn) mn = q;
                }
            v = mx - mn;
        } else {
            double hx = dx0 / (double)(1L << level[p]), hy = dy0 / (double)(1L << level[p]);
            v = 0.0;
            for (int j = 1; j < n - 1; ++j)
                for (int i = 1; i < n - 1; ++i) {
                    double gx = fabs(a[IX(&L, i + 1, j)] - a[IX(&L, i - 1, j)]) / (2.0 * hx);
                    double gy = fabs(a[IX(&L, i, j + 1)] - a[IX(&L, i, j - 1)]) / (2.0 * hy);
                    if (gx > v) v = gx;
                    if (gy > v) v = gy;
                }
        }
        if (ind) ind[p] = v;
        tags[p] = (int8_t)(v >= refine_thr ? 1 : (v < coarsen_thr ? -1 : 0));
    }
}

/* Total of every component: sum over patches and interior cells of
 * Q_{i,j} dx_l dy_l (the conserved quantity of Eq. 2dfv).
 * Pinned by: its definition, used by the P7 conservation pins.            */
void orc_mass(int n, int ncomp, int nleaf, const int32_t *level, const double *state, double dx0, double dy0,
              double *out) {
    lay_t L = lay_make(n, ncomp);
    long pw = lay_patch_words(&L);
    for (int c = 0; c < ncomp; ++c) {
        double s = 0.0;
        for (int p = 0; p < nleaf; ++p) {
            const double *a = PLc(&L, state + p * pw, c, PL_AVG);
            double area = (dx0 / (double)(1L << level[p])) * (dy0 / (double)(1L << level[p]));
            for (int j = 0; j < n; ++j)
                for (int i = 0; i < n; ++i) s += a[IX(&L, i, j)] * area;
        }
        out[c] = s;
    }
}

/* Regrid transfer (Section 3.1, cases 1 and 2): every leaf of the new forest
 * that is also a leaf of the old one is copied; every other new leaf gets,
 * from the old leaf owning each entry (coarse -> fine interpolation if that
 * leaf is coarser, fine -> coarse averaging or the coinciding vertex if it is
 * finer), its cell averages and the point values of its cells' boundaries:
 * node lines 0 .. n, the far lines i = n and j = n included, because a leaf
 * finer than its right or top neighbour owns the nodes on that face (the more
 * resolved grid's values are used at coarse-fine faces, Section 3.2).  Entries
 * another leaf owns, and the ghost ring, are replaced by the next exchange.
 * Pinned by: refine-then-coarsen returns the original averages, and the
 * nodes shared with the old leaf are copied exactly (P8); after any regrid
 * and exchange of biquadratic data every entry of every leaf is exact.     */
void orc_transfer(int n, int ncomp, int B, int lmax, int nold, const int32_t *olevel, const int32_t *oix,
                  const int32_t *oiy, const double *old_state, int nnew, const int32_t *nlevel, const int32_t *nix,
                  const int32_t *niy, double *new_state) {
    forest_t F;
    lay_t L = lay_make(n, ncomp);
    long pw = lay_patch_words(&L);
    if (forest_init(&F, n, ncomp, nold, olevel, oix, oiy, B, lmax) != 0) { forest_free(&F); return; }
    for (int p = 0; p < nnew; ++p) {
        long side = (long)B << nlevel[p];
        int same = F.map[nlevel[p]][(long)niy[p] * side + nix[p]];
        double *dst = new_state + p * pw;
        if (same >= 0) { memcpy(dst, old_state + same * pw, sizeof(double) * pw); continue; }
        for (long e = 0; e < pw; ++e) dst[e] = 0.0;
        long hw = hw_of(&F, nlevel[p]);
        long x0 = (long)nix[p] * n * hw, y0 = (long)niy[p] * n * hw;
        for (int k = 0; k < 4; ++k) {
            /* lattice lines of the plane on the leaf's cells and their
             * boundaries: averages [0,n)^2, corners [0,n]^2, left-edge
             * midpoints [0,n] x [0,n), bottom-edge midpoints [0,n) x [0,n] */
            const int ni = (k == PL_CORNER || k == PL_XMID) ? n + 1 : n;
            const int nj = (k == PL_CORNER || k == PL_YMID) ? n + 1 : n;
            for (int j = 0; j < nj; ++j)
                for (int i = 0; i < ni; ++i) {
                    long x = x0 + (long)i * hw + ((k == PL_AVG || k == PL_YMID) ? hw / 2 : 0);
                    long y = y0 + (long)j * hw + ((k == PL_AVG || k == PL_XMID) ? hw / 2 : 0);
                    int q = entry_owner(&F, k, x, y);
                    if (q < 0) continue;
                    for (int c = 0; c < ncomp; ++c)
                        PL(&L, dst, c, k)[IX(&L, i, j)] = transfer_value(&F, old_state, nlevel[p], q, c, k, x, y);
                }
        }
    }
    forest_free(&F);
}

/*
 * af.h -- C ABI of the GB300 Active Flux library (libaf.so).
 *
 * Cartesian-grid Active Flux method with adaptive mesh refinement,
 * Calhoun, Chudzik, Helzel, arXiv 2205.07572.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Every pointer named d_* is a DEVICE pointer owned by the caller; h_* is a
 *    host pointer owned by the caller.  The library keeps no reference to any
 *    of them after the call returns and never frees them.
 *  - Device work is enqueued asynchronously on `stream` (a cudaStream_t; NULL
 *    is the legacy default stream).  Argument errors are detected on the host
 *    and returned synchronously before anything is enqueued; a launch error is
 *    returned as AF_ERR_CUDA.  Nothing is thrown across the ABI.
 *  - Calls allocate no device memory.
 *
 * State layout (Section 2, Fig. 1: four degrees of freedom per cell)
 * -------------------------------------------------------------------
 *  state[patch][comp][plane][plane_stride], elements double (AF_F64) or float
 *  (AF_F32).  plane 0 = cell average Q_{i,j}; 1 = left-edge midpoint
 *  Q_{i-1/2,j}; 2 = lower-left corner Q_{i-1/2,j-1/2}; 3 = bottom-edge
 *  midpoint Q_{i,j-1/2}.  Each plane is a (M+1) x (M+1) row-major lattice,
 *  M = N + 2g, g = 2 ghost layers (Section 3.2), x fastest; lattice entry
 *  (I, J) belongs to cell / node line (i, j) = (I - g, J - g), i, j in
 *  [-g, N+g].  plane_stride = af_plane_stride(N) = (M+1)^2 rounded up to a
 *  multiple of 8 elements.  Entries with i, j in [0, N) are the patch's own
 *  ("interior-owned") degrees of freedom; the rest is the ghost ring.  The base
 *  pointer must be 32-byte aligned (AF_ERR_LAYOUT otherwise).
 *  ncomp = 1 for advection (q), 3 for acoustics (p, u, v).
 */
#ifndef AF_H
#define AF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    AF_OK = 0,
    AF_ERR_ARG = 1,           /* invalid argument (null pointer, bad size, aliasing) */
    AF_ERR_CFL = 2,           /* time step violates Eq. cfl-adv / Eq. cfl-acoustics */
    AF_ERR_LAYOUT = 3,        /* misaligned pointer or inconsistent layout */
    AF_ERR_CUDA = 4,          /* a CUDA runtime call failed */
    AF_ERR_TIMEOUT = 5,       /* a bounded device wait gave up */
    AF_ERR_UNIMPLEMENTED = 6  /* combination not supported by this build */
} af_status;

typedef enum { AF_ADVECTION = 0, AF_ACOUSTICS = 1 } af_equation;
typedef enum { AF_F64 = 0, AF_F32 = 1 } af_precision;

/* Problem description.  eq: Eq. advection2d (q_t + a q_x + b q_y = 0) or
 * Eq. acoustics (p_t + c div u = 0, u_t + c grad p = 0).  n: interior cells
 * per patch side, 2 <= n <= 64 (the paper uses 8, 16 or 32, Section 3). */
typedef struct {
    int32_t eq;     /* af_equation */
    int32_t prec;   /* af_precision of the state arrays and the arithmetic */
    int32_t n;      /* interior cells per patch side */
    int32_t ncomp;  /* must be 1 (advection) or 3 (acoustics) */
    double a, b;    /* advection velocity */
    double c;       /* speed of sound, > 0 */
} af_config;

/* One unit of work of af_patch_step: a rectangle of cells of one patch,
 * produced by af_build_step_work (callers normally treat it as opaque and
 * just copy the array to the device).  64 bytes. */
typedef struct {
    int32_t patch;      /* index into the state array */
    int32_t level;      /* refinement level: dx = dx0 / 2^level, dt = dt0 / 2^level */
    int32_t nbr[8];     /* same-level neighbour patch of W, E, S, N, SW, SE, NW, NE, or -1 */
    int16_t x0, x1;     /* cells [x0, x1) of the patch, in [-1, N+1] */
    int16_t y0, y1;
    int32_t flags;      /* bit 0: the patch advances its first ghost layer too */
    int32_t pad_[3];
} af_work;

/* Human-readable name of a status code (static storage). */
const char *af_status_string(af_status s);

/* Elements per plane for patches of n x n cells: ((n+5)^2 rounded up to 8). */
int64_t af_plane_stride(int32_t n);

/* Elements of one patch: ncomp * 4 * af_plane_stride(n). */
int64_t af_patch_words(int32_t n, int32_t ncomp);

/* Build the work list of af_patch_step on the host (Section 2; Section 3.2
 * for the ghost layer).
 *
 * h_patch[k]   state index of the k-th patch to advance, k < npatch
 * h_level[k]   its refinement level (NULL: all 0)
 * h_nbr[8k+d]  state index of its same-level neighbour in direction d
 *              (order W, E, S, N, SW, SE, NW, NE), or -1 when that direction
 *              is a coarser/finer patch or a physical boundary.  h_nbr == NULL
 *              means "no neighbours": every patch reads its own ghost ring.
 *
 * A patch whose eight neighbours are all same-level reads its halo straight
 * from the neighbours' interiors (no ghost copy is needed) and advances its
 * interior only.  Any other patch reads the missing directions from its own
 * ghost ring (filled by af_fill_ghosts) and also advances its first ghost
 * layer, which subcycling needs at intermediate times (Section 3.2).
 *
 * Patches are split into tiles of at most 32 x 32 cells.  Writes at most
 * `capacity` entries to h_work and the count to *nwork; returns AF_ERR_ARG if
 * capacity is too small (*nwork then holds the required count). */
af_status af_build_step_work(const af_config *cfg, int32_t npatch, const int32_t *h_patch,
                             const int32_t *h_level, const int32_t *h_nbr, af_work *h_work,
                             int32_t capacity, int32_t *nwork);

/* One Active Flux time step (Section 2) for every work item:
 *   1. point values at t^{n+1/2}, t^{n+1} at corners and edge midpoints from
 *      the continuous biquadratic reconstruction (Eq. poly) by exact
 *      back-tracing (Eq. advection-update) or the spherical-means formula
 *      (Eqs. ERFormula, sphe-mean);
 *   2. fluxes by the 3 x 3 space-time Simpson rule (Eq. Simpson-2d);
 *   3. the conservative update of the cell averages (Eq. 2dfv).
 *
 * d_work     device copy of the af_build_step_work output (nwork entries)
 * d_in       state at t^n (npatch_total patches, layout above)
 * d_out      receives the new averages and point values of every advanced
 *            cell; entries not advanced are left untouched.  Must not
 *            overlap d_in (AF_ERR_ARG).
 * dt0, dx0, dy0   time step and mesh widths of level 0 (level l uses /2^l).
 *            AF_ERR_CFL if max(|a| dt/dx, |b| dt/dy) > 1 (Eq. cfl-adv) or
 *            max(c dt/dx, c dt/dy) > 1/2 (Eq. cfl-acoustics).
 * d_flux_reg NULL, or FP64 [npatch_total][4][ncomp][n]: dt_l * F (x faces)
 *            or dt_l * G (y faces) on the patch's four boundary faces is
 *            ADDED (side 0 = x-line 0, 1 = x-line n, 2 = y-line 0,
 *            3 = y-line n) for the conservative fix (Section 3.2). */
af_status af_patch_step(const af_config *cfg, int32_t nwork, const af_work *d_work,
                        const void *d_in, void *d_out, double dt0, double dx0, double dy0,
                        double *d_flux_reg, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* AF_H */

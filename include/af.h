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
    int32_t flags;      /* bit 0: the patch advances its first ghost layer too;
                           bit 1 (AF_WORK_SKIP_BULK_COPY): failure injection --
                           a bulk-staged tile does not issue its copies, so its
                           bounded wait runs out (af_step_wait_timeouts) */
    int32_t ix, iy;     /* column and row of the patch among the patches of its level
                           (af_build_step_work_at; used only by af_patch_step_var) */
    int32_t pad_;
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
 * Patches are split into tiles of the default tiling for cfg (see
 * af_step_tilings).  Writes at most
 * `capacity` entries to h_work and the count to *nwork; returns AF_ERR_ARG if
 * capacity is too small (*nwork then holds the required count). */
af_status af_build_step_work(const af_config *cfg, int32_t npatch, const int32_t *h_patch,
                             const int32_t *h_level, const int32_t *h_nbr, af_work *h_work,
                             int32_t capacity, int32_t *nwork);

/* Compiled tile shapes of af_patch_step.  A tiling splits every patch (or
 * its interior plus first ghost layer) into near-equal tiles of at most
 * tile_x x tile_y cells, each advanced by one CTA of `threads` threads;
 * persistent = CTAs loop over tiles with the next tile's copies in flight;
 * af_patch_step* refuse persistent tilings (AF_ERR_UNIMPLEMENTED: the kernel
 * is withdrawn), af_patch_step_var runs them as one tile per CTA.  Which is
 * fastest depends on the patch size, equation and precision; the autotuner
 * (paper_2205_07572_gb300/tune.py) times them. */
typedef struct {
    int32_t tile_x, tile_y;
    int32_t threads;
    int32_t persistent;
} af_tiling;

/* Writes up to `capacity` compiled tilings to `out`; returns how many exist. */
int32_t af_step_tilings(af_tiling *out, int32_t capacity);

/* Index of the tiling af_build_step_work / af_patch_step use for cfg. */
int32_t af_step_default_tiling(const af_config *cfg);

/* af_build_step_work with an explicit tiling (index into af_step_tilings). */
af_status af_build_step_work_tiled(const af_config *cfg, int32_t tiling, int32_t npatch, const int32_t *h_patch,
                                   const int32_t *h_level, const int32_t *h_nbr, af_work *h_work,
                                   int32_t capacity, int32_t *nwork);

/* af_build_step_work_tiled that also records each patch's position:
 * h_ix[k], h_iy[k] = column and row of patch k among the patches of its
 * level (so its lower-left corner is at (x_lo + ix n dx_l, y_lo + iy n dy_l));
 * needed by af_patch_step_var, ignored by the constant-velocity steps.
 * NULL means 0. */
af_status af_build_step_work_at(const af_config *cfg, int32_t tiling, int32_t npatch, const int32_t *h_patch,
                                const int32_t *h_level, const int32_t *h_ix, const int32_t *h_iy,
                                const int32_t *h_nbr, af_work *h_work, int32_t capacity, int32_t *nwork);

/* One Active Flux time step (Section 2) for every work item:
 *   1. point values at t^{n+1/2}, t^{n+1} at corners and edge midpoints from
 *      the continuous biquadratic reconstruction (Eq. poly) by exact
 *      back-tracing (Eq. advection-update) or the spherical-means formula
 *      (Eqs. ERFormula, sphe-mean);
 *   2. fluxes by the 3 x 3 space-time Simpson rule (Eq. Simpson-2d);
 *   3. the conservative update of the cell averages (Eq. 2dfv).
 *
 * d_work     device copy of the af_build_step_work output (nwork entries),
 *            16-byte aligned (AF_ERR_LAYOUT otherwise)
 * d_in       state at t^n (npatch_total patches, layout above)
 * d_out      receives the new averages and point values of every advanced
 *            cell.  A patch that advances its first ghost layer (one with a
 *            non-same-level neighbour) is written whole: its other entries
 *            are copied from d_in (same-level directions: from the
 *            neighbours).  For other patches the ghost ring is not kept:
 *            its entries in the rows of advanced cells may receive the
 *            values read at t^n (a patch's own or its neighbours'), so that
 *            whole lattice rows are written; other ghost entries are left
 *            untouched.  Must not be the same buffer as d_in (AF_ERR_ARG).
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

/* af_patch_step with an explicit tiling; d_work must have been built with the
 * same tiling (tiles larger than the tiling's maximum are skipped). */
af_status af_patch_step_tiled(const af_config *cfg, int32_t tiling, int32_t nwork, const af_work *d_work,
                              const void *d_in, void *d_out, double dt0, double dx0, double dy0,
                              double *d_flux_reg, void *stream);

/* Two state arrays with a per-level choice of the current one, so that a
 * subcycled adaptive run (Section 3.2: level l takes 2^(l-m) steps for every
 * step of the coarsest level m) can advance any set of levels without
 * copying: a step reads the current array of each level and writes the
 * other, and the caller then flips the parity bits of the levels it
 * advanced.  Both arrays have the same shape (npatch_total patches, layout
 * above) and are owned by the caller; parity bit l set means the current
 * values of the level-l leaves are in buf[1], clear means buf[0].  Entries
 * of the other array are stale and are never read.  The paper keeps one
 * array per patch; this is the GPU's way to batch all levels that advance at
 * one time into one launch. */
typedef struct {
    void *buf[2];
    uint32_t parity;
    uint32_t pad_;
} af_state_pair;

/* af_patch_step_tiled on a state pair: every work item of level l reads
 * buf[(parity >> l) & 1] and writes the other array.  Work items of several
 * levels may share one call: they use dt0 / 2^l and dx0 / 2^l, so the CFL
 * numbers and stencil weights are those of level 0, and the flux registers
 * receive dt_l * F.  Levels advanced together must not read one another
 * (true of the levels that advance at one time of a subcycled schedule:
 * their patches read only same-level neighbours and their own ghost rings).
 * AF_ERR_ARG if buf[0] == buf[1]; other errors as af_patch_step. */
af_status af_patch_step_pair(const af_config *cfg, int32_t tiling, int32_t nwork, const af_work *d_work,
                             const af_state_pair *state, double dt0, double dx0, double dy0,
                             double *d_flux_reg, void *stream);

/* The owned degrees of freedom of npatch patches (entries with i, j in
 * [0, N) of every plane: the cell averages and the corner, left-edge and
 * bottom-edge point values of the patch's own cells, Section 2, Fig. 1)
 * between the state layout above and a compact array
 * owned[patch][comp][plane][j][i], N x N per plane, elements as cfg->prec,
 * no padding.  For a state kept in host memory this is all that crosses the
 * host link: a patch with same-level neighbours on all sides reads its halo
 * from them, so its ghost ring need not travel.
 * af_pack_owned    d_state -> d_owned
 * af_unpack_owned  d_owned -> d_state; the ghost ring and the plane padding of
 *                  d_state are left untouched
 * Both asynchronous on `stream`, device pointers owned by the caller.
 * AF_ERR_ARG on a bad cfg, npatch < 0, a NULL pointer (npatch > 0) or the same
 * pointer twice; AF_ERR_LAYOUT if d_state is not 32-byte aligned or d_owned
 * not aligned to its element size. */
af_status af_pack_owned(const af_config *cfg, int32_t npatch, const void *d_state, void *d_owned, void *stream);
af_status af_unpack_owned(const af_config *cfg, int32_t npatch, const void *d_owned, void *d_state, void *stream);

/* Measurement probe (no counterpart in the paper): `blocks` CTAs of
 * af_fma_probe_threads() / 8 threads each run 8 independent fused
 * multiply-add chains of `iters` steps in precision `prec` (af_precision) and
 * store one value per thread to d_sink (device, blocks * 256 elements of that
 * precision, aligned to its size).  Flops per call:
 * 2 * 8 * iters * blocks * 256; timing the call on `stream` gives the GPU's
 * FMA rate, the ALU roof of the step kernels.  AF_ERR_ARG on a bad precision,
 * blocks < 1, iters < 1 or NULL d_sink; AF_ERR_LAYOUT if d_sink is misaligned. */
int32_t af_fma_probe_threads(void);
af_status af_fma_throughput(int32_t prec, int32_t blocks, int32_t iters, void *d_sink, void *stream);

/* Tiles that span a patch's interior columns are staged by bulk (TMA) copies
 * whose completion the kernel awaits for at most about a second (2^31 SM
 * cycles).  A tile whose wait gives up waits once more with the same limit
 * for its copies in flight, leaves its outputs unwritten and increments a
 * device counter.  Setting AF_WORK_SKIP_BULK_COPY in a work item's flags
 * makes that happen without any fault: its copies are never issued.  The
 * learned tagger's kernels (af_cnn_forward, af_cnn_backward) wait the same
 * bounded way for their tensor-core MMAs and count a wait that gives up in
 * the same total (that CTA then stops: its remaining samples are left
 * unwritten).  A CTA whose second wait also gives up (about two seconds in
 * all, far beyond any copy or MMA of a working GPU) exits with its copies
 * possibly still in flight; the step's results must then be discarded.
 * This call synchronises with the device, writes the
 * counter to *count and, if reset != 0, sets it to zero.  AF_ERR_ARG if count
 * is NULL, AF_ERR_CUDA if the copy fails.  The counter is armed from the
 * first af_patch_step* call made outside CUDA stream capture. */
af_status af_step_wait_timeouts(uint32_t *count, int32_t reset);
#define AF_WORK_SKIP_BULK_COPY 2


/* Variable-velocity advection q_t + (a q)_x + (b q)_y = 0 (one component),
 * with the velocity fields of Sections 4.2 and 4.3:
 *   AF_FIELD_SOLID_BODY  a = -pi y, b = pi x (Eq. solidbodyODE); point values
 *       by back-tracing along the exact rotation (Eq. characteristics_advtwo);
 *       flux through a face by Simpson's rule in space and time of a q with
 *       the velocity at each face point;
 *   AF_FIELD_SWIRL  stream function Psi = sin^2(pi x) sin^2(pi y) cos(pi t)/pi,
 *       velocities by its centred differences over one mesh width of the
 *       patch's level (Eq. swirlODE), evaluated through
 *       sin^2 A - sin^2 B = sin(A+B) sin(A-B) (the same numbers, without
 *       cancellation); feet by one classical Runge-Kutta step of size -tau;
 *       fluxes of Eqs. swirlF, swirlG (velocity at the face centre times
 *       Simpson's rule along the face, at t^n, t^{n+1/2}, t^{n+1}); these
 *       fluxes keep constant states constant (Theorem of Section 4.3). */
#define AF_FIELD_SOLID_BODY 0
#define AF_FIELD_SWIRL 1
typedef struct {
    int32_t field;
    int32_t pad_;
    double x_lo, y_lo; /* lower-left corner of the domain: node line 0 of patch (0, 0) */
    double x_hi, y_hi; /* upper-right corner (bounds the speed for the CFL check) */
    double t;          /* time t^n at the start of the step */
} af_velocity;

/* One Active Flux step of variable-velocity advection on a state pair (see
 * af_state_pair), as af_patch_step_pair otherwise: cfg->eq = AF_ADVECTION,
 * ncomp 1 (cfg->a, cfg->b unused); d_work from af_build_step_work_at (patch
 * positions).  Level l uses dx0 / 2^l, dy0 / 2^l, dt0 / 2^l; every work item
 * starts at vel->t.  AF_ERR_CFL unless the largest speed on the domain and
 * its two ghost layers times dt_l stays within one mesh width (the foot must
 * lie in a cell next to its node).  Flux registers receive dt_l * F. */
af_status af_patch_step_var(const af_config *cfg, int32_t tiling, int32_t nwork, const af_work *d_work,
                            const af_state_pair *state, const af_velocity *vel, double dt0, double dx0, double dy0,
                            double *d_flux_reg, void *stream);

/* ======================================================================
 * Adaptive mesh refinement (Section 3): a forest of quadtrees over a B x B
 * brick of level-0 patches, periodic in x and y.  Every leaf is one patch
 * (N x N cells) of the state array; level l has mesh width dx0 / 2^l.
 * ====================================================================== */

#define AF_MAX_LEVEL 15

/* Forest description.  The struct itself lives in host memory; the arrays it
 * points to are DEVICE arrays owned by the caller. */
typedef struct {
    int32_t nleaf;          /* leaves = patches of the state array, in this order */
    int32_t B;              /* level-0 patches per side of the periodic brick, >= 1 */
    int32_t lmax;           /* finest level that may occur, 0 .. AF_MAX_LEVEL */
    int32_t pad_;
    const int32_t *d_level; /* [nleaf] level of each leaf */
    const int32_t *d_ix;    /* [nleaf] column of the leaf among the B << level of its level */
    const int32_t *d_iy;    /* [nleaf] row */
    const int32_t *d_map;   /* per level l: (B << l)^2 entries starting at
                               af_forest_map_offset(B, l), row-major; entry
                               (iy, ix) is the leaf index q of region
                               (l, ix, iy) if that region is a leaf, -2 - q if
                               it lies inside the coarser leaf q, else -1 */
} af_forest;

/* Offset of level l in d_map: sum over m < l of (B << m)^2. */
int64_t af_forest_map_offset(int32_t B, int32_t level);

/* Fill h_map (af_forest_map_offset(B, lmax + 1) entries, host memory) from
 * host copies of the leaf arrays (the d_map layout above).  AF_ERR_ARG on an
 * out-of-range leaf or two leaves claiming one region (also one inside the
 * other). */
af_status af_forest_build_map(int32_t nleaf, int32_t B, int32_t lmax, const int32_t *h_level,
                              const int32_t *h_ix, const int32_t *h_iy, int32_t *h_map);

/* Same-level neighbours of every leaf (host): h_nbr[8p + d] is the leaf
 * index of the level-l region next to leaf p in direction d (W, E, S, N,
 * SW, SE, NW, NE; periodic), or -1 if that region is not a leaf.  h_map is
 * the output of af_forest_build_map.  This is the h_nbr argument of
 * af_build_step_work. */
af_status af_forest_neighbours(int32_t nleaf, int32_t B, int32_t lmax, const int32_t *h_level,
                               const int32_t *h_ix, const int32_t *h_iy, const int32_t *h_map, int32_t *h_nbr);

/* Regrid (Section 3: refinement and coarsening "at each time step" from a
 * per-patch criterion; the forest stays 2:1 balanced), on the host, from the
 * per-leaf tags of af_tag:
 *   1. every leaf tagged 1 below lmax is split into its four children;
 *   2. families of four leaves tagged -1 above lmin, taken in ascending
 *      order of their parent's (level, ix, iy), are merged into the parent
 *      unless a face or corner neighbour region of the parent then holds a
 *      leaf two or more levels finer;
 *   3. leaves with such a neighbour are split until none is left.
 * The new leaves are written sorted by (level, iy, ix), at most `capacity`
 * of them; *out_n receives their count (AF_ERR_ARG if capacity is too
 * small).  Host memory O(B^2 4^lmax) bytes.  AF_ERR_ARG on out-of-range or
 * duplicate leaves. */
af_status af_forest_regrid(int32_t nleaf, int32_t B, int32_t lmin, int32_t lmax, const int32_t *h_level,
                           const int32_t *h_ix, const int32_t *h_iy, const int8_t *h_tags, int32_t capacity,
                           int32_t *out_level, int32_t *out_ix, int32_t *out_iy, int32_t *out_n);

/* Flags of af_fill_ghosts. */
#define AF_FILL_SAME_LEVEL_ONLY 1 /* copy from same-level leaves only */
#define AF_FILL_ALL_PATCHES 2     /* also fill leaves whose 8 neighbours are all same-level */

/* Ghost exchange (Section 3.1 cases 1-3, Section 3.2 "whenever two levels are
 * time synchronized"), in place on d_state.
 * Ownership: a cell average belongs to the leaf covering the cell centre; a
 * point value belongs to the finest leaf touching the point (ties: the leaf
 * above-right, above-left, below-right, below-left of it), so values on a
 * coarse-fine face come from the finer leaf.  Every entry of a destination
 * leaf (level bit set in dst_levels) whose owner is another leaf with its
 * level bit set in src_levels is replaced: copy from a same-level owner;
 * from a finer owner the mean of the four fine averages, or the coinciding
 * fine vertex; from a coarser owner the value of its reconstruction, or for
 * an average Simpson's rule over the fine cell (exact).  Three passes run in
 * order -- finer owners, same-level owners, coarser owners -- each seeing the
 * previous one's results.  Unless AF_FILL_ALL_PATCHES is set, leaves whose
 * eight neighbours are all same-level leaves are skipped (af_patch_step
 * reads their halo from the neighbours directly). */
af_status af_fill_ghosts(const af_config *cfg, const af_forest *forest, uint32_t dst_levels,
                         uint32_t src_levels, int32_t flags, void *d_state, void *stream);

/* Ghost plan: af_fill_ghosts with the owner of every exchanged entry found
 * once per forest.  The exchange itself (Section 3.1 cases 1-3, at the
 * synchronised times of Section 3.2) is then two passes over a flat list:
 * pass A replaces entries whose owner is same-level (copy) or finer (mean of
 * the four finer averages, or the coinciding finer vertex); pass B replaces
 * entries whose owner is coarser by the owner's reconstruction (point value,
 * or Simpson's rule over the finer cell).  Pass B reads the coarse cell's
 * boundary point values from the coarse leaf's own lattice, which pass A has
 * refreshed, so the result equals af_fill_ghosts bit for bit.
 *
 * The plan is a device array of AF_GHOST_ENTRY_BYTES-byte entries owned by
 * the caller, valid for one forest (rebuild after every regrid):
 *   1. af_ghost_plan_count writes the number of pass-A and pass-B entries to
 *      d_counts[0], d_counts[1] (device, int64, 8-byte aligned);
 *   2. the caller allocates (n_a + n_b) entries (16-byte aligned) and calls
 *      af_ghost_plan_build with the counts and 3 int64 of device scratch
 *      (16-byte aligned; zeroed by the call); after the build, scratch[2]
 *      is non-zero if the counts were too small (the plan is then unusable).
 * flags: AF_FILL_ALL_PATCHES includes leaves whose eight neighbours are all
 * same-level (as af_fill_ghosts).  Each leaf's entries of a pass are
 * contiguous and in lattice order (plane, row, column), so the exchange's
 * accesses coalesce; the leaves' ranges are in no particular order.  Each
 * destination entry appears once, so the order does not change the result.
 *
 * af_fill_ghosts_planned runs the exchange for the leaves of `levels` from
 * owners of `levels` (af_fill_ghosts with dst_levels = src_levels = levels).
 * `levels` must be upward closed -- with its coarsest level it holds every
 * finer level up to the forest's lmax (true of every synchronised set of a
 * subcycled schedule, and of all levels) -- else AF_ERR_ARG, because pass B
 * relies on pass A having refreshed the coarse leaves.  flags may add
 * AF_FILL_SAME_LEVEL_ONLY (pass A's copies from same-level owners only). */
#define AF_GHOST_ENTRY_BYTES 16
af_status af_ghost_plan_count(const af_config *cfg, const af_forest *forest, int32_t flags, int64_t *d_counts,
                              void *stream);
af_status af_ghost_plan_build(const af_config *cfg, const af_forest *forest, int32_t flags, void *d_plan,
                              int64_t n_a, int64_t n_b, int64_t *d_scratch, void *stream);
af_status af_fill_ghosts_planned(const af_config *cfg, const af_forest *forest, uint32_t levels, int32_t flags,
                                 const void *d_plan, int64_t n_a, int64_t n_b, const af_state_pair *state,
                                 void *stream);

/* Regrid transfer (Section 3.1 cases 1 and 2): every leaf of new_forest that
 * is a leaf of old_forest is copied whole from d_old, except the point values
 * on its right and top faces, which are taken from their owners in old_forest
 * (a leaf whose neighbours are all same-level does not keep those copies
 * current, and it owns them once the neighbour across has coarsened); every
 * other new leaf gets, from the owners in old_forest (coarse -> fine interpolation, fine ->
 * coarse averaging over one level, the coinciding vertex of a finer owner),
 * its cell averages and the point values on its cells' boundaries -- node
 * lines 0 .. n, the right and top lines included, which the leaf owns where
 * its neighbour across is coarser (Section 3.2 uses the finer grid's values
 * at coarse-fine faces) -- and zeros in the rest of its ghost ring.  Entries
 * another leaf owns are replaced by the exchange (af_fill_ghosts over all
 * levels) that must follow.  d_old and d_new must not overlap. */
af_status af_transfer(const af_config *cfg, const af_forest *old_forest, const void *d_old,
                      const af_forest *new_forest, void *d_new, void *stream);

/* Conservative fix (Section 3.2, Berger-Colella).  For every leaf C whose
 * level l and l+1 are both set in sync_levels and every face k of C whose
 * neighbour across is a level-(l+1) leaf F, the average of the coarse cell at
 * that face is corrected so that it has used the fine fluxes:
 *   right/top face:  dQ = (R_C[k] - (R_F[a] + R_F[a+1]) / 2) / h_C
 *   left/bottom face: dQ = ((R_F[a] + R_F[a+1]) / 2 - R_C[k]) / h_C
 * with R the flux registers of af_patch_step (sum of dt * F since they were
 * last consumed) and h_C = dx0 / 2^l (x faces) or dy0 / 2^l (y faces).
 * Consumed register entries (coarse and fine) are reset to zero. */
af_status af_reflux(const af_config *cfg, const af_forest *forest, uint32_t sync_levels, double dx0,
                    double dy0, double *d_flux_reg, void *d_state, void *stream);

/* Refinement indicator per leaf (Section 3: "we apply coarsening and
 * refinement criteria to the solution on each quadrant").
 * kind 0: max - min of the interior averages of component comp (Sections 4.1,
 * 4.5.2); kind 1: largest |Q_{i+1,j} - Q_{i-1,j}| / (2 dx) or
 * |Q_{i,j+1} - Q_{i,j-1}| / (2 dy) over interior cells whose two neighbours
 * are interior (Section 4.4).  d_tags[p] = 1 if indicator >= refine_thr, -1 if
 * indicator < coarsen_thr, else 0.  d_indicator (FP64) may be NULL. */
af_status af_tag(const af_config *cfg, const af_forest *forest, const void *d_state, int32_t comp,
                 int32_t kind, double dx0, double dy0, double refine_thr, double coarsen_thr, int8_t *d_tags,
                 double *d_indicator, void *stream);

/* Bytes of device scratch af_mass needs for nleaf leaves and ncomp components. */
int64_t af_mass_scratch_bytes(int32_t nleaf, int32_t ncomp);

/* Total of every component, sum over leaves and interior cells of
 * Q_{i,j} dx_l dy_l, in FP64 whatever the state precision (the conserved
 * quantity of Eq. 2dfv).  Deterministic two-pass reduction: per-block partial
 * sums go to d_scratch (af_mass_scratch_bytes, 8-byte aligned), the final sums
 * to d_mass[ncomp]. */
af_status af_mass(const af_config *cfg, const af_forest *forest, const void *d_state, double dx0, double dy0,
                  void *d_scratch, double *d_mass, void *stream);

/* The operations above on a state pair (see af_state_pair): every leaf is
 * read from and written to the current array of its level; the other array
 * is not touched.  af_transfer_pair reads the old forest's state from a pair
 * and writes the new forest's state to the single array d_new.  Results are
 * those of the single-array calls applied to the current arrays. */
af_status af_fill_ghosts_pair(const af_config *cfg, const af_forest *forest, uint32_t dst_levels,
                              uint32_t src_levels, int32_t flags, const af_state_pair *state, void *stream);
af_status af_transfer_pair(const af_config *cfg, const af_forest *old_forest, const af_state_pair *old_state,
                           const af_forest *new_forest, void *d_new, void *stream);
af_status af_reflux_pair(const af_config *cfg, const af_forest *forest, uint32_t sync_levels, double dx0,
                         double dy0, double *d_flux_reg, const af_state_pair *state, void *stream);
af_status af_tag_pair(const af_config *cfg, const af_forest *forest, const af_state_pair *state, int32_t comp,
                      int32_t kind, double dx0, double dy0, double refine_thr, double coarsen_thr, int8_t *d_tags,
                      double *d_indicator, void *stream);
af_status af_mass_pair(const af_config *cfg, const af_forest *forest, const af_state_pair *state, double dx0,
                       double dy0, void *d_scratch, double *d_mass, void *stream);


/* af_mass without any caller-provided scratch.  The paper has no
 * counterpart: this entry point exists for callers that cannot allocate
 * device memory -- for example a host code whose own pool allocator owns the
 * whole device and lends the library only its state arrays, or a time loop
 * that must not call cudaMalloc / cudaFree because those calls synchronise
 * the device and stall every stream.  Same result as af_mass (same blocking,
 * same summation order).
 * The partial sums live in one fixed array inside the library, 1024 doubles
 * (8 KB, room for 256 partial sums of up to 4 components), which every GPU
 * that loads the library keeps until the process exits; AF_ERR_ARG if a
 * call would need more (it never does: af_mass uses at most 256 partial sums
 * per component and ncomp <= 3).  The state must be 32-byte aligned, as for
 * af_mass (else AF_ERR_LAYOUT).  Every call looks up the array's device
 * address (cudaGetSymbolAddress, a runtime query that enqueues no work and
 * allocates nothing) with the caller's device current, so the address always
 * belongs to the current context, also after a device reset.  The first call
 * on a device may load the library's device code; make it before any stream
 * capture.  All calls on one device share that device's copy of the array,
 * which keeps the last call's partial sums: calls that overlap on the GPU
 * (for example on two streams with no ordering between them) race and give
 * wrong totals; calls on different devices use different copies.  Nothing
 * needs clearing between calls: every partial sum is written before it is
 * read. */
af_status af_mass_noalloc(const af_config *cfg, const af_forest *forest, const void *d_state, double dx0,
                          double dy0, double *d_mass, void *stream);

/* ======================================================================
 * Learned refinement tagger.  The paper tags a patch from a per-patch
 * criterion (Section 3; the undivided-difference indicator of Sections 4.4
 * and 4.5.2, af_tag kind 1).  These entry points replace that criterion by a
 * small network trained on the plain criterion's own tags: from a patch's
 * cell averages with a two-cell halo at one regrid, it predicts the tag the
 * plain criterion gives at the next one, so refinement can move ahead of
 * the solution.  The paper has no such network; this is its definition
 * (F = 32 channels, C = ncomp, S = n + 4, n = 8 or 16):
 *   X[c, y, x] = bf16((Q_c(x-2, y-2) - mean of the patch's Q_c) / (2 h_l thr))
 *   A1 = bf16(relu(conv3x3(X, bf16(W1)) + emb[level]))       [F, S-2, S-2]
 *   Z2 = conv3x3(A1, bf16(W2)) + b2                           [F, S-4, S-4]
 *   M[g] = max(0, max over pixels of Z2[g]);  logit = w3 . M + b3
 * conv3x3(A, W)[g, y, x] = sum_{f, ky, kx} W[g, f, ky, kx] A[f, y+ky, x+kx]
 * (no padding), FP32 arithmetic.  The parameters are one FP32 vector
 * (af_cnn_param_count floats): W1 [F][C][3][3], emb [16][F], W2 [F][F][3][3],
 * b2 [F], w3 [F], b3.  X is BF16 (raw uint16 storage), [nsample][C][S][S].
 * Training minimises sum_p weight_p BCE(logit_p, label_p) / sum_p weight_p
 * with Adam.  All arrays are device arrays owned by the caller.
 * ====================================================================== */
int64_t af_cnn_param_count(int32_t ncomp);

/* X for every leaf of the forest (nleaf x C x S x S BF16) from the current
 * state: cells outside the patch are read from the same-level neighbour
 * d_nbr[8p + d] (af_forest_neighbours order) where there is one, else from
 * the leaf's own ghost ring (exchanged by af_fill_ghosts).  h_l = dx0 / 2^l;
 * thr is the plain criterion's refinement threshold. */
af_status af_cnn_inputs(const af_config *cfg, const af_forest *forest, const af_state_pair *state,
                        const int32_t *d_nbr, double dx0, double thr, uint16_t *d_x, void *stream);

/* Forward pass: logits, the pooled maxima M [nsample][F] and their first
 * row-major positions d_arg [nsample][F] (-1 where M = 0), which the
 * backward pass reuses.  d_level[k] in 0..15.  d_arg may be NULL
 * (inference): the positions are then not computed, and the logits and M
 * are the same bit for bit. */
af_status af_cnn_forward(int32_t ncomp, int32_t n, int32_t nsample, const uint16_t *d_x, const int32_t *d_level,
                         const float *d_params, float *d_logit, float *d_m, int32_t *d_arg, void *stream);

/* Floats of scratch af_cnn_backward needs for nblocks CTAs. */
int64_t af_cnn_partial_floats(int32_t ncomp, int32_t nblocks);

/* Gradient of the weighted loss with respect to the parameters into d_grad
 * (overwritten), from the outputs of af_cnn_forward with the same
 * parameters.  weight_sum = sum of d_weight over the batch.  Deterministic:
 * nblocks CTAs write partial sums to d_partial, which are then added in a
 * fixed order.  The BF16 roundings are passed through as identities. */
af_status af_cnn_backward(int32_t ncomp, int32_t n, int32_t nsample, const uint16_t *d_x, const int32_t *d_level,
                          const float *d_params, const float *d_logit, const float *d_m, const int32_t *d_arg,
                          const float *d_label, const float *d_weight, double weight_sum, float *d_partial,
                          int32_t nblocks, float *d_grad, void *stream);

/* One Adam step (Kingma & Ba): moments d_m, d_v updated in place, bias
 * corrections for step `step` (>= 1). */
af_status af_cnn_adam(int64_t nparam, float *d_params, float *d_m, float *d_v, const float *d_grad, int32_t step,
                      double lr, double beta1, double beta2, double eps, void *stream);

/* Final tags from the network and the plain criterion's tags d_plain (af_tag):
 * where the network's confidence |2 sigmoid(logit) - 1| < cmin the plain tag
 * is used (and *d_nfallback, device int32, is incremented); otherwise 1 if
 * the network predicts refinement, else the plain tag with refinement
 * removed (-1 stays, 1 becomes 0). */
af_status af_cnn_tags(int32_t nleaf, const float *d_logit, const int8_t *d_plain, double cmin, int8_t *d_tags,
                      int32_t *d_nfallback, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* AF_H */

/*
 * claw.h -- C ABI of libclaw.so: the wave-propagation level-step of Qin, LeVeque & Motley,
 * "Accelerating wave-propagation algorithms with adaptive mesh refinement using the GPU"
 * (arXiv:1808.02638), as hand-written CUDA kernels for sm_103a (GB300).
 *
 * Problem (Sec. 4.1): linear acoustics q_t + A q_x + B q_y = 0, q = (p, u, v), with cell-wise
 * density rho and bulk modulus K (c = sqrt(K/rho), impedance Z = rho c).  Each level-step is
 * the unsplit wave-propagation update of Eq. wave_form_2d_2nd_order applied to every patch of
 * an AMR level (Sec. 2.2), with limited second-order corrections and transverse propagation.
 * A second system goes through the same step and AMR machinery (the framework takes any system
 * through its normal and transverse Riemann solvers, Sec. 3.1, 3.3): the nonlinear shallow
 * water equations on a flat bottom, q = (h, hu, hv), with the Roe solvers (system =
 * CLAW_SYS_SHALLOW_WATER; the level-step, ghost filling, averaging, regridding, the
 * conservation fix and the CFL control apply; the adjoint is acoustics-only).
 *
 * Conventions shared by every entry point
 *   - Storage: a box (patch) with an nx x ny interior has CLAW_MBC = 2 ghost layers and is
 *     stored as planes of (nx+4) x (ny+4) doubles, x fastest.  A q pool holds, for box b,
 *     the planes p, u, v back to back starting at element qoff[b].  One-plane pools (rho, K)
 *     hold box b at element coff[b]; an aux pool holds CLAW_NAUX planes for box b starting
 *     at element CLAW_NAUX * coff[b].  Offsets must be even (16-byte aligned rows) and nx
 *     even; the pools are allocated and owned by the caller.
 *   - All pointers to pools and to the dt / smax scalars are DEVICE pointers on the context's
 *     device.  The library owns only its own tables, allocated in claw_set_level.
 *   - Every call that takes a stream enqueues work on it and returns without waiting; it
 *     launches no kernel when it returns an error.  Calls on one context are not thread-safe.
 *   - Launches may be captured into CUDA graphs.  A staged level-step reads tensor-map
 *     descriptors of its q_old pool that the context builds on first use outside a capture and
 *     caches per pool; a descriptor that a capture has seen is kept until the level's tables
 *     are rebuilt (claw_set_level, a tile-shape change in claw_set_tiling), so a graph stays
 *     valid until then.
 *   - Errors are status codes (never aborts or traps).  Errors found on the device (NaN or
 *     Inf in a new state, a CFL number above 1, a bounded wait that expired) are recorded in
 *     a device flag and reported by claw_sync_status.
 */
#ifndef CLAW_H
#define CLAW_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CLAW_OK 0
#define CLAW_EINVAL 1   /* bad argument, bad box set (overlap, outside the domain, not nested)  */
#define CLAW_ECUDA 2    /* a CUDA runtime call failed                                          */
#define CLAW_ENOMEM 3   /* device or host allocation failed                                    */
#define CLAW_ECFL 4     /* a level-step ran with a CFL number above 1 (Sec. 2.4)                */
#define CLAW_ENAN 5     /* a new state held NaN or Inf                                         */
#define CLAW_ETIMEOUT 6 /* a bounded device wait expired                                      */
#define CLAW_ESTATE 7   /* call out of order (e.g. level L set before level L-1)               */

#define CLAW_MBC 2
#define CLAW_MAXLEV 8
#define CLAW_NAUX 10

/* limiter ids: phi(theta) of the waves (Sec. 2.1; the benchmark of Sec. 4.1 uses van Leer) */
#define CLAW_LIM_NONE 0
#define CLAW_LIM_MINMOD 1
#define CLAW_LIM_SUPERBEE 2
#define CLAW_LIM_VANLEER 3
#define CLAW_LIM_MC 4

/* systems */
#define CLAW_SYS_ACOUSTICS 0
#define CLAW_SYS_SHALLOW_WATER 1

/* physical boundary conditions (Sec. 2.2 item 1; the benchmark uses outflow = extrapolation) */
#define CLAW_BC_EXTRAP 0
#define CLAW_BC_PERIODIC 1
#define CLAW_BC_WALL 2

typedef struct claw_ctx claw_ctx;

/* One independent problem (a "run").  Level 0 covers [xlo,xhi] x [ylo,yhi] with nx0 x ny0
 * cells; level L > 0 is ratio[L] times finer than level L-1 in x, y and t (Sec. 2.2). */
typedef struct claw_problem {
    double xlo, ylo, xhi, yhi;
    int32_t nx0, ny0;
    int32_t nlev;
    int32_t ratio[CLAW_MAXLEV];  /* ratio[0] is ignored */
    double cfl;                  /* desired CFL number nu_desired of Eq. cfl */
    int32_t limiter;             /* CLAW_LIM_* */
    int32_t order;               /* 1: first order, 2: with the correction fluxes */
    int32_t transverse;          /* 0 none, 1 fluctuations, 2 fluctuations and corrections */
    int32_t bc[4];               /* x-low, x-high, y-low, y-high: CLAW_BC_* */
    int32_t medium;              /* 0: uniform rho0, K0; 1: cell-wise (aux pools) */
    double rho0, K0;
    int32_t system;              /* CLAW_SYS_*: 0 acoustics (all of the above), 1 shallow water */
    int32_t reserved;            /* 0 */
    double grav;                 /* shallow water: gravitational acceleration g > 0 */
} claw_problem;

/* A box of a level in that level's index space [0, NX_L) x [0, NY_L) of run `run`. */
typedef struct claw_box {
    int32_t run;
    int32_t ilo, jlo, nx, ny;
    int32_t reserved;
    int64_t qoff;   /* element offset of the box's p plane in the level's q pool */
    int64_t coff;   /* element offset of the box's plane in one-plane pools */
} claw_box;

/* Creates a context for nruns problems on CUDA device `device`.  All runs must share
 * limiter, order, transverse, medium, system and grav.  Shallow water needs medium = 0 (rho0,
 * K0 are ignored) and grav > 0.  Returns CLAW_OK and sets *out, or an error. */
int claw_create(claw_ctx** out, const claw_problem* runs, int32_t nruns, int32_t device);

/* Frees the context and its device tables (synchronises the device first). */
void claw_destroy(claw_ctx* ctx);

/* Declares the boxes of level `level` of all runs (Sec. 2.2: disjoint boxes, nested in level
 * level-1, aligned to its cells).  Validates them on the host, builds and uploads the patch,
 * tile, ghost-source and averaging tables.  Levels must be set in increasing order; setting a
 * level again replaces its tables (and invalidates the tables of finer levels).  A level's
 * tables live in device memory that the context keeps from one setting of the level to the
 * next (grown when too small) and overwrites after synchronising the device, so CUDA graphs
 * captured before the call must not be replayed after it.
 * Errors: CLAW_EINVAL (overlap, out of domain, misaligned, improper nesting, odd nx/offset),
 * CLAW_ESTATE (level-1 not set), CLAW_ENOMEM, CLAW_ECUDA.  Synchronous. */
int claw_set_level(claw_ctx* ctx, int32_t level, const claw_box* boxes, int32_t nboxes);

/* Chooses the tiling of the fused level-step for a level: tx x ty interior cells per tile,
 * the staging of the tile's q planes into shared memory (0 = cooperative loads,
 * 1 = tensor-memory-accelerator bulk copies into two buffers, 2 = bulk copies into one buffer with
 * three CTAs per SM, acoustics 32x16 with 256 threads only; 1 and 2 only when every box has even
 * nx and offsets) and
 * the threads per CTA (0 = default).  Supported for acoustics: 32x32 with 256 or 512 threads,
 * 32x16 with 256, 16x16 with 128; claw_set_level installs 32x32, 256 threads.  Supported for
 * shallow water: 16x16 with 256 threads, 32x16 with 512; claw_set_level installs 16x16.  Once
 * chosen here, a level's tiling stays through later claw_set_level calls (with staging 0 when
 * the new boxes do not allow bulk copies), as does its claw_set_tile_walk choice.
 * Staging 1 is installed when allowed.  A new tile shape rewrites the level's tile lists in
 * place (after synchronising the device): graphs captured before must not be replayed.
 * Errors: CLAW_EINVAL, CLAW_ENOMEM, CLAW_ECUDA. */
int claw_set_tiling(claw_ctx* ctx, int32_t level, int32_t tx, int32_t ty, int32_t staging,
                    int32_t threads);

/* Chooses how the persistent CTAs of a level's fused step share its tiles (Sec. 3.1.3 merges a
 * level's patch kernels into one launch; this is the order inside it).  walk = 0: each CTA
 * strides over the tiles, largest first.  walk = 1 (acoustics in a uniform medium, shallow water): the
 * tiles form columns, each box's tile columns continued into the same-level box directly above
 * when it has the same run, ilo and nx; every CTA takes one contiguous stretch of about equal
 * cost, and a tile that follows the tile below it in its CTA's stretch takes the edge values of
 * the rows they share from that tile instead of recomputing them.  Both give the same q_new, dt
 * and smax bit for bit.  walk = -1 (claw_set_level installs it): 1 for uniform-medium levels
 * with at least 8 tiles per SM, else 0 (shallow water measured faster striding).  A cell-wise
 * medium accepts 0 and -1 (which means 0).  A
 * change rewrites the level's tile lists like claw_set_tiling.
 * Errors: CLAW_EINVAL, CLAW_ENOMEM, CLAW_ECUDA. */
int claw_set_tile_walk(claw_ctx* ctx, int32_t level, int32_t walk);

/* Failure detection of the staged level-steps (no counterpart in the paper).  With staging 1
 * or 2 a CTA waits on a shared-memory barrier for the bulk copy of each tile; the wait polls
 * the barrier at most `polls` times (default 2^22, far beyond a normal copy).  When it gives
 * up, the CTA records CLAW_ETIMEOUT in the device flag (read by claw_sync_status), waits again
 * with the default bound for every copy it has issued (so that none lands after it exits),
 * and stops without writing its remaining tiles: the new state of that step is incomplete.
 * polls = 0 makes every staged CTA give up at its first tile, which is how the error path is
 * tested.  Applies to the level-step calls issued after it on this context.
 * Errors: CLAW_EINVAL (ctx NULL).  Host only, no device work. */
int claw_set_wait_limit(claw_ctx* ctx, uint32_t polls);

/* The wave limiter of the level-step (Sec. 2.1: a wave's strength scaled by phi(theta), theta
 * the ratio of the upwind edge's strength of the same family to its own), elementwise on the
 * current CUDA device: out[i] = phi(b[i] / a[i]) a[i], computed exactly as the step computes it
 * (0 where a[i] b[i] <= 0; minmod, superbee and MC on the integer pipe, MC's (|a| + |b|) / 2
 * rounded like the IEEE sum; van Leer within a relative 4 * 2^-53 of 2ab / (a + b)).  a, b, out: n device
 * doubles.  For tests of the step's limiters.  Errors: CLAW_EINVAL, CLAW_ECUDA. */
int claw_limiter_eval(int32_t limiter, int64_t n, const double* a, const double* b, double* out, void* stream);

/* Per-cell coefficient planes for medium = 1 from one-plane pools rho, K (ghosts included):
 * aux holds, for every cell, Z = sqrt(K rho), c = sqrt(K/rho), K, c^2, 1/(Z_W+Z) and the
 * two wave-limiter projection factors of the edge to the west, and the same three for the
 * edge to the south.  Enqueued on `stream`.  Errors: CLAW_EINVAL, CLAW_ECUDA. */
int claw_medium_aux(claw_ctx* ctx, int32_t level, const double* rho, const double* K, double* aux,
                    void* stream);

/* Ghost cells of every box of `level` in q (Sec. 2.2): a ghost takes the value at its image
 * under the physical boundary of the domain, where a cell inside the domain is the box's own
 * interior, another box of the level, or (level > 0) the space-time interpolation of the
 * coarser level: (1-tau) qc_old + tau qc_new followed by minmod-limited linear
 * reconstruction in space.  qc_old / qc_new may be NULL for level 0.  Errors: CLAW_EINVAL,
 * CLAW_ESTATE, CLAW_ECUDA. */
int claw_fill_ghost(claw_ctx* ctx, int32_t level, double* q, const double* qc_old,
                    const double* qc_new, double tau, void* stream);

/* Only the ghosts of claw_fill_ghost that are interpolated from the coarser level (nothing on
 * level 0): what a level-step with CLAW_ADVANCE_PULL_GHOSTS still reads from q's ghost cells. */
int claw_fill_ghost_interp(claw_ctx* ctx, int32_t level, double* q, const double* qc_old,
                           const double* qc_new, double tau, void* stream);

/* The same-level and physical-boundary ghosts (Sec. 2.2 items 1-2) of a one-plane pool such as
 * rho or K (box b at element coff[b]; no sign flips at walls).  Ghosts that would need the
 * coarser level are left as they are (coefficients of finer levels are given by the caller).
 * The _adjoint call adds every such ghost's value into its source cell and zeroes the ghost:
 * the gradient with respect to the interior field from one with respect to the padded pool.
 * A context with a uniform medium builds these copy tables on the first call for a level
 * (synchronously; CLAW_ESTATE if that first call is made while `stream` is being captured). */
int claw_fill_ghost_coef(claw_ctx* ctx, int32_t level, double* a, void* stream);
int claw_fill_ghost_coef_adjoint(claw_ctx* ctx, int32_t level, double* g, void* stream);

/* smax[run] = max(smax[run], max c over the cells next to the edges a level-step of `level`
 * solves: the ring [-1, nx] x [-1, ny] of every box), for the first time step (Eq. cfl).
 * aux may be NULL for medium = 0.  smax has one entry per run (zero it before the first use;
 * claw_dt_update resets it).  Acoustics only (CLAW_EINVAL for shallow water). */
int claw_cfl_max(claw_ctx* ctx, int32_t level, const double* aux, double* smax, void* stream);

/* The same for a system whose speeds depend on the state (shallow water): smax[run] =
 * max(smax[run], max over the same ring cells of |u| + sqrt(g h) and |v| + sqrt(g h)) from the
 * level's q pool (ghosts filled).  A cell with h <= 0 gives NaN.  CLAW_EINVAL for acoustics. */
int claw_cfl_max_state(claw_ctx* ctx, int32_t level, const double* q, double* smax, void* stream);

/* Eq. cfl on the device, per run r, with dx, dy of level `level` (normally 0): checks that the
 * step just taken with dt[r] kept smax[r] * dt[r] / min(dx, dy) <= 1 (else the device flag
 * records CLAW_ECFL), sets dt[r] = cfl * min(dx, dy) / smax[r] and resets smax[r] to 0.
 * Because every level's time step is the level-0 step over the product of the ratios, the
 * CFL number is the same on every level, so one dt per run serves the whole hierarchy. */
int claw_dt_update(claw_ctx* ctx, int32_t level, double* smax, double* dt, void* stream);

/* One level-step of every box of `level` (Eq. wave_form_2d_2nd_order) in one persistent
 * fused launch: q_new interior = step(q_old with filled ghosts).  dt[r] is the level-0 time
 * step of run r; level L advances by dt[r] / (ratio[1] ... ratio[L]) (Sec. 2.2: a level R_L
 * times finer takes R_L times smaller steps).  The largest wave speed seen is
 * max-accumulated into smax[r].  Only
 * interior cells of q_new are written.  aux may be NULL for medium = 0.  q_old and q_new must
 * not overlap.  Shallow water: a depth h <= 0 in a cell the step reads is reported as
 * CLAW_ENAN (the Roe solver is for wet states).  Errors: CLAW_EINVAL, CLAW_ESTATE, CLAW_ECUDA. */
int claw_level_step(claw_ctx* ctx, int32_t level, const double* q_old, double* q_new,
                    const double* aux, const double* dt, double* smax, void* stream);

/* claw_level_step with epilogues selected by `flags`:
 *   CLAW_ADVANCE_PUSH_GHOSTS: the same-level copies and physical boundaries of q_new are filled
 *     right after the step (a second launch on the same stream), so the next step of this level
 *     needs no separate fill unless it has interpolated ghosts;
 *   CLAW_ADVANCE_UPDATE_DT: after the step, Eq. cfl is applied on the device by the last CTA
 *     to finish (as claw_dt_update with level-0 dx, dy): dt[r] is replaced by the next time step
 *     and smax[r] reset.  Use it when this level-step ends the coarse step (a hierarchy of one
 *     level); dt is then both read and written by the launch;
 *   CLAW_ADVANCE_PULL_GHOSTS: the step takes every same-level and physical-boundary ghost of
 *     q_old from its source cell (an interior cell of q_old, with the boundary's sign flips)
 *     instead of q_old's ghost cells, so those need no fill at all; ghosts interpolated from the
 *     coarser level are still read from q_old and must be filled (claw_fill_ghost).  The ghost
 *     cells of q_new are not written unless CLAW_ADVANCE_PUSH_GHOSTS is also given.
 * Errors as claw_level_step, CLAW_EINVAL for unknown flags (and for PULL_GHOSTS on a level with
 * more than 2^31 ghost cells). */
#define CLAW_ADVANCE_PUSH_GHOSTS 1
#define CLAW_ADVANCE_UPDATE_DT 2
#define CLAW_ADVANCE_PULL_GHOSTS 4
int claw_level_advance(claw_ctx* ctx, int32_t level, const double* q_old, double* q_new,
                       const double* aux, double* dt, double* smax, int32_t flags, void* stream);

/* claw_level_advance with CLAW_ADVANCE_PULL_GHOSTS (required) in which the step also evaluates
 * the ghosts of q_old that come from the coarser level (Sec. 2.2: space-time interpolation,
 * the same values claw_fill_ghost_interp writes) from qc_old, qc_new (the coarser level's
 * states at the start and end of its step, device pools) at the time fraction tau in [0, 1],
 * instead of reading them from q_old.  So one launch is the whole fine level-step: no ghost of
 * q_old is read from q_old's ghost cells, and none is written.  For level 0, or a level without
 * interpolated ghosts, it is claw_level_advance and qc_old, qc_new may be NULL.  Shallow water
 * (no fused kernel) fills those ghosts of q_old with the interpolation launch first, on the same
 * stream (two launches, the same values).
 * Errors as claw_level_advance; CLAW_EINVAL without the pull flag or without coarse states. */
int claw_level_advance_interp(claw_ctx* ctx, int32_t level, const double* q_old, double* q_new,
                              const double* aux, double* dt, double* smax, int32_t flags,
                              const double* qc_old, const double* qc_new, double tau, void* stream);

/* One fill of a fine level's ghost cells that come from the coarser level, as
 * claw_fill_ghost_interp(ctx, level, q, qc_old, qc_new, tau) writes them. */
typedef struct {
    int32_t level;          /* the fine level (>= 1) */
    int32_t reserved;       /* 0 */
    double* q;              /* that level's pool whose interpolated ghost cells are written */
    const double* qc_old;   /* level - 1 states at the start and end of its step (device pools) */
    const double* qc_new;
    double tau;             /* time fraction in [0, 1] */
} claw_fill_job;

/* claw_level_advance, and in the same launch the interpolated-ghost fills of `jobs` (0, 1 or 2),
 * done by extra CTAs beside those that step the tiles (Sec. 2.2: each fine substep needs its
 * ghosts interpolated from the coarser level at its own time).  A job must concern this level
 * (its next substep, into q_new's ghost cells, which the step does not write) or the next finer
 * one (its first substep: tau 0, from this level's q_old as both coarse states).  The result is
 * that of claw_level_advance followed by claw_fill_ghost_interp for each job, on the same stream.
 * Errors as claw_level_advance; CLAW_EINVAL for more than 2 jobs, a job of another level, a
 * level not set, NULL pools, tau outside [0, 1], a job writing q_old, or a job reading q_new
 * as a coarse state. */
int claw_level_advance_fill(claw_ctx* ctx, int32_t level, const double* q_old, double* q_new,
                            const double* aux, double* dt, double* smax, int32_t flags,
                            const claw_fill_job* jobs, int32_t njobs, void* stream);

/* claw_level_advance restricted to the boxes [box_begin, box_end) of the level (their tiles, in
 * box order): a level-step taken in pieces, so that host copies of some boxes overlap the steps
 * of others.  The pieces of one step, in any order, give bit for bit the claw_level_advance of
 * the whole level.  flags: CLAW_ADVANCE_PULL_GHOSTS only (apply claw_dt_update after the last
 * piece; push ghosts with claw_fill_ghost).  With pulled ghosts a piece reads the boxes it
 * touches and their neighbours' interiors in q_old.  Errors as claw_level_advance. */
int claw_level_advance_boxes(claw_ctx* ctx, int32_t level, int32_t box_begin, int32_t box_end,
                             const double* q_old, double* q_new, const double* aux,
                             const double* dt, double* smax, int32_t flags, void* stream);

/* Packed interiors of a level: box after box in box order, each box's three planes of nx x ny
 * interior cells (x fastest), no ghosts and no padding; box b starts at element
 * 3 * sum over earlier boxes of nx * ny.  claw_packed_size: the doubles of a level's packed
 * form (or minus an error code).  claw_pack_interiors copies the interiors of the boxes
 * [box_begin, box_end) of the pool q into their places in `packed` (the whole level's packed
 * buffer); claw_unpack_interiors the other way (ghost cells of q are not touched).  Device
 * pointers; enqueued on `stream`.  Errors: CLAW_EINVAL, CLAW_ECUDA. */
long long claw_packed_size(claw_ctx* ctx, int32_t level);
int claw_pack_interiors(claw_ctx* ctx, int32_t level, int32_t box_begin, int32_t box_end,
                        const double* q, double* packed, void* stream);
int claw_unpack_interiors(claw_ctx* ctx, int32_t level, int32_t box_begin, int32_t box_end,
                          const double* packed, double* q, void* stream);

/* The same step with one kernel launch per box (the per-patch launch pattern of Sec. 3.1.2,
 * kept as the comparison baseline of the fused launch). */
int claw_level_step_patchwise(claw_ctx* ctx, int32_t level, const double* q_old, double* q_new,
                              const double* aux, const double* dt, double* smax, void* stream);

/* The fused level-step of one box that allocates nothing: for callers that cannot allocate
 * device memory where they step (under a host application's own device-memory pool, in a loop
 * that cannot take cudaMalloc's implicit synchronisation).
 * The paper has no counterpart; it exists for those callers.
 * q_old / q_new hold one box (p, u, v planes of (nx+4) x (ny+4) doubles at offset 0; the
 * ghosts of q_old are filled by the caller); aux (cell-wise medium, CLAW_NAUX planes at
 * offset 0) or NULL for the uniform medium rho0, K0; dt[0] the time step; smax[0] receives
 * the max wave speed (max-accumulated, as in claw_level_step).  32 x 32 tiles, cooperative
 * staging.  The scratch (box descriptor, tile table, error word) is a fixed 256 KiB device
 * array that every device loading the library keeps until exit, so at most 16367 tiles of
 * 32 x 32 cells fit (e.g. 4064 x 4096 cells, not 4096 x 4096): larger boxes, and nx or ny
 * above 4096, return CLAW_EINVAL before any launch.  The first call on a device looks up the
 * array's device address synchronously (once per device, with that device current) and keeps
 * it for the life of the process: after a cudaDeviceReset of that device the kept address is
 * stale, so the entry point must not be called again on it.  Every call
 * rewrites the whole scratch it uses (device errors of this path are not reported), and all
 * calls share the one array: calls whose kernels overlap on the GPU (other streams, other
 * threads) race.  Errors: CLAW_EINVAL, CLAW_ECUDA. */
int claw_level_step_noalloc(int32_t nx, int32_t ny, double dx, double dy, int32_t limiter, int32_t order,
                            int32_t transverse, double rho0, double K0, const double* q_old, double* q_new,
                            const double* aux, const double* dt, double* smax, void* stream);

/* Coarse cells of level fine_level-1 covered by level fine_level := mean of their ratio^2
 * fine cells (the "updating" of Sec. 2.2-2.3). */
int claw_average_down(claw_ctx* ctx, int32_t fine_level, const double* q_fine, double* q_coarse,
                      void* stream);

/* Reverse mode of claw_level_step for a frozen dt (dt as in claw_level_step): given
 * lam_new, the adjoint of q_new (interior cells read), accumulates (+=) the adjoint of q_old
 * over all cells, ghosts included, into lam_old and the adjoint of the medium into g_aux
 * (medium = 1; may be NULL for medium = 0).  g_aux has the aux layout; the c^2 plane's
 * adjoint is folded into the c plane here (that plane of g_aux is left as it is), the two
 * 1/(Z_L+Z_R) planes receive their value times their adjoint (claw_medium_aux_adjoint expects
 * that), every other plane its own adjoint.  The limiter branches of the forward step are recomputed
 * from q_old.  lam_old and g_aux must be zeroed by the caller
 * before the first accumulation. */
int claw_level_step_adjoint(claw_ctx* ctx, int32_t level, const double* q_old, const double* lam_new,
                            double* lam_old, const double* aux, double* g_aux, const double* dt,
                            void* stream);

/* claw_level_step_adjoint with the adjoint of the same-level and physical-boundary ghosts
 * fused in (flags = CLAW_ADVANCE_PULL_GHOSTS; 0 is claw_level_step_adjoint): the kernel adds
 * the adjoint of each such ghost cell of a box straight into the cell it was filled from (its
 * entry in the level's ghost ring, u or v negated across a wall), which is what
 * claw_fill_ghost_adjoint's copy part would do with it; those ghosts of lam_old stay zero.
 * Ghosts interpolated from the coarser level keep their adjoint for
 * claw_fill_ghost_interp_adjoint.  Like the forward claw_level_advance with pulled ghosts, the
 * kernel reads those same-level and boundary ghosts of q_old from their source cells, so only
 * the interpolated ghosts of q_old need to be filled (a state written by a pulled-ghost step
 * and then claw_fill_ghost_interp is enough).  The same linear map as step adjoint +
 * ghost-fill adjoint, summed in another order (FP64 atomics).  Errors: as claw_level_step_adjoint; CLAW_EINVAL for
 * an unknown flag or a level without a ghost ring. */
int claw_level_advance_adjoint(claw_ctx* ctx, int32_t level, const double* q_old, const double* lam_new,
                               double* lam_old, const double* aux, double* g_aux, const double* dt,
                               int32_t flags, void* stream);

/* Differentiation by tape (no counterpart in the paper, which has no adjoint; the map
 * differentiated is the level-step of Eq. wave_form_2d_2nd_order, Sec. 2.1).
 * claw_level_advance_record is claw_level_advance (flags: CLAW_ADVANCE_PULL_GHOSTS and
 * CLAW_ADVANCE_UPDATE_DT, with that call's meaning; without the pull every ghost of q_old must be
 * filled) that also writes the step's intermediates to `tape`, a device
 * buffer of CLAW_NAUX * coff-layout doubles (the size of the level's aux pool, owned by the
 * caller): per padded cell, the normal-solver wave strengths and limited strengths of the
 * edges west and south of the cell (the limiter's branch kept in the three lowest mantissa
 * bits of the limited strength) and the cell's transverse fluctuation pressures.  The new state
 * is the one claw_level_advance computes.  Cell-wise medium (medium = 1), order 2 (and a ghost
 * ring for pulled ghosts).  Errors: CLAW_EINVAL, CLAW_ESTATE, CLAW_ECUDA. */
int claw_level_advance_record(claw_ctx* ctx, int32_t level, const double* q_old, double* q_new,
                              const double* aux, double* dt, double* smax, int32_t flags, double* tape,
                              void* stream);

/* The adjoint of the recorded step from its tape alone (no q_old, no re-run of the forward):
 * the same map as claw_level_advance_adjoint (flags: 0 or CLAW_ADVANCE_PULL_GHOSTS, with that
 * call's meaning), accumulating (+=) into lam_old and g_aux (aux layout, the c^2 plane folded into
 * c), dt frozen at the recorded step's.  The limiter branches are the recorded ones.  Cell-wise
 * medium, order 2.  Errors: CLAW_EINVAL, CLAW_ESTATE, CLAW_ECUDA. */
int claw_level_advance_adjoint_tape(claw_ctx* ctx, int32_t level, const double* tape, const double* lam_new,
                                    double* lam_old, const double* aux, double* g_aux, const double* dt,
                                    int32_t flags, void* stream);

/* Reverse of claw_fill_ghost: every ghost adjoint of lam is added to the adjoint of its
 * source (a box interior of the level, or through the interpolation to lam_c_old /
 * lam_c_new, which may be NULL for level 0) and set to zero.  qc_old / qc_new are the coarse
 * states the forward fill read (for the minmod branches).  claw_fill_ghost_interp_adjoint does
 * the interpolated ghosts only (after claw_level_advance_adjoint with pulled ghosts). */
int claw_fill_ghost_adjoint(claw_ctx* ctx, int32_t level, double* lam, double* lam_c_old,
                            double* lam_c_new, const double* qc_old, const double* qc_new,
                            double tau, void* stream);
int claw_fill_ghost_interp_adjoint(claw_ctx* ctx, int32_t level, double* lam, double* lam_c_old,
                                   double* lam_c_new, const double* qc_old, const double* qc_new,
                                   double tau, void* stream);

/* Reverse of claw_average_down: lam_f += (1/ratio^2) lam_c on the children, lam_c := 0 on the
 * covered coarse cells. */
int claw_average_down_adjoint(claw_ctx* ctx, int32_t fine_level, double* lam_fine,
                              double* lam_coarse, void* stream);

/* Chain rule from the aux planes to rho and K: g_rho += d aux/d rho . g_aux, same for K, with
 * g_aux as the adjoint calls leave it (each 1/(Z_L+Z_R) plane holding that value times its
 * adjoint). */
int claw_medium_aux_adjoint(claw_ctx* ctx, int32_t level, const double* rho, const double* K,
                            const double* g_aux, double* g_rho, double* g_K, void* stream);

/* ---- Conservation fix at coarse-fine interfaces (Sec. 2.3, "refluxing"), uniform medium.
 * For the acoustics system in conservation form (medium = 0) and for shallow water (whose Roe
 * solver is conservative; A (Q_F - Q_C) below is then f(Q_F) - f(Q_C) with the equations'
 * flux), every coarse cell C of level
 * fine_level-1 that the fine level does not cover but that shares an edge e with it is
 * corrected after the average so that the flux through e equals the average of the fine fluxes
 * through the r fine edges over the r substeps.  In flux form, with C left of e:
 *   Q_C += -(dt/dx) [ (1/r^2) sum_{k,b} (A (Q_F^k - Q_C^n) - A+dQ_b^k + F~_b^k) - (A-dQ_e + F~_e) ]
 * (the paper's C1 + C2 + C3; mirrored for C right of e and in y), F~ being the correction flux
 * plus the transverse terms of the edge.  The interface (records, one per coarse cell and side,
 * periodic boundaries wrapping) is built by claw_set_level of the fine level.  `buf` is a device
 * buffer of claw_reflux_buffer_size doubles (3 per record for the coarse parts, then 3 per record
 * and fine edge for the fine parts), owned by the caller; dt are the per-run level-0 time steps
 * (the levels' own steps follow from the ratios).  Sequence per coarse step of level L-1:
 *   claw_reflux_coarse(L, q_{L-1}^n)                       (ghosts of q_{L-1}^n filled)
 *   for each substep k: claw_reflux_fine(L, q_L^k, q_{L-1}^n) (ghosts of q_L^k filled)
 *   claw_average_down(L, ...), then claw_reflux_apply(L, q_{L-1}^{n+1}).
 * Errors: CLAW_EINVAL (medium = 1, NULL pointers, level 0), CLAW_ESTATE, CLAW_ECUDA. */
int claw_reflux_count(claw_ctx* ctx, int32_t fine_level);         /* records, or minus an error code */
int claw_reflux_buffer_size(claw_ctx* ctx, int32_t fine_level);   /* doubles of buf, or minus an error */
/* buf := minus the coarse part (A-dQ_e + F~_e, or -A+dQ_e + F~_e for C right of e) of each record,
 * and zero fine parts */
int claw_reflux_coarse(claw_ctx* ctx, int32_t fine_level, const double* q_c_old, const double* dt,
                       double* buf, void* stream);
/* the fine part of each record's r fine edges (one slot each) += that of one substep, from the
 * fine state q_f of the substep and the coarse state q_c_old the coarse step started from */
int claw_reflux_fine(claw_ctx* ctx, int32_t fine_level, const double* q_f, const double* q_c_old,
                     const double* dt, double* buf, void* stream);
/* q_c_new of every corrected coarse cell += -side (dt_c / h) (coarse part + (1/r^2) fine parts),
 * summed per cell in table order (deterministic) */
int claw_reflux_apply(claw_ctx* ctx, int32_t fine_level, const double* buf, const double* dt,
                      double* q_c_new, void* stream);

/* ---- Regridding (Sec. 2.2: every K steps the finer levels are regenerated from flagged cells
 * clustered with the algorithm of Berger and Rigoutsos; Sec. 4.3: cutoff and regrid interval).
 * The flag grid of a level holds, for each run with that level, NX x NY bytes of the level's
 * index space, row-major, the runs back to back in run order.  Levels are rebuilt top-down:
 * flags of level L -> claw_regrid_boxes -> claw_set_level(L+1, new boxes) ->
 * claw_regrid_transfer(L+1, old boxes, ...). */
long long claw_flag_grid_size(claw_ctx* ctx, int32_t level);   /* bytes, or minus an error code */
/* flags[cell] = 1 where some component of q differs from a face neighbour by more than tol, 0
 * elsewhere, for every interior cell of the level's boxes (ghosts of q filled; other bytes of
 * the grid are not written).  flags: device pointer.  Errors: CLAW_EINVAL, CLAW_ESTATE. */
int claw_flag_cells(claw_ctx* ctx, int32_t level, const double* q, double tol, uint8_t* flags, void* stream);
/* Host only.  New boxes of level+1 for run `run` from its flag grid of `level` (host pointer):
 * the flags grown by `buffer` cells (square neighbourhood, clipped to the domain), kept where
 * the square of radius `nest` around the cell lies in the level's boxes (the domain outside
 * counts as covered), then clustered in level cells: a box is accepted when flags fill at least
 * `cutoff` of it, no side exceeds max_size / ratio and all its cells pass that nesting test;
 * otherwise it is cut at a hole of a row or
 * column signature (the one nearest the middle), else at the strongest sign change of a
 * signature's second difference, else at the middle of its longer side.  Writes (ilo, jlo, nx,
 * ny) in level+1 cells to boxes[4k..4k+3].  Returns the count, -CLAW_ENOMEM when more than
 * max_boxes, -CLAW_EINVAL / -CLAW_ESTATE on bad arguments. */
int claw_regrid_boxes(claw_ctx* ctx, int32_t level, int32_t run, const uint8_t* flags, int32_t buffer, int32_t nest,
                      double cutoff, int32_t max_size, int32_t* boxes, int32_t max_boxes);
/* Host only, no context and no GPU: the same clustering for an nx x ny level whose boxes (for
 * the nesting test; their run, qoff and coff are ignored) are cover[0..ncover), the new boxes in
 * the cells of a level `ratio` times finer.  claw_regrid_boxes calls it with the run's boxes of
 * `level`.  Same returns; -CLAW_EINVAL also for nx, ny or ratio below 1. */
int claw_cluster_flags(int32_t nx, int32_t ny, int32_t ratio, const claw_box* cover, int32_t ncover,
                       const uint8_t* flags, int32_t buffer, int32_t nest, double cutoff, int32_t max_size,
                       int32_t* boxes, int32_t max_boxes);
/* After claw_set_level(level, new boxes): every interior cell of the new boxes takes the value of
 * the old level (old_boxes with their qoff in q_old, host array) where an old box held it, else
 * the conservative space interpolation from q_coarse (level-1, same time), read from the coarse
 * box holding the cell's parent with its ghosts, which must be filled (the new boxes lie two
 * coarse cells inside the coarse level, as claw_regrid_boxes makes them).  On the device: the old
 * boxes and the coarse boxes are painted into level-wide index grids (4 bytes per cell of the
 * level and of the coarse level, kept by the context), then every new cell reads its source from
 * them.  Waits for its launches (its tables sit in a scratch arena of the context that the next
 * call reuses).  Errors: CLAW_EINVAL (an old box outside its level, or a new cell without a coarse
 * parent: not nested; the other cells are written), CLAW_ESTATE, CLAW_ENOMEM, CLAW_ECUDA. */
int claw_regrid_transfer(claw_ctx* ctx, int32_t level, const claw_box* old_boxes, int32_t n_old, const double* q_old,
                         double* q_new, const double* q_coarse, void* stream);

/* Waits for the context's device work, returns and clears the first device-side error
 * (CLAW_ENAN, CLAW_ECFL, CLAW_ETIMEOUT) or CLAW_OK. */
int claw_sync_status(claw_ctx* ctx);

/* Kernels of the library launched so far (every entry point counts its launches). */
int64_t claw_launch_count(claw_ctx* ctx);

const char* claw_strerror(int32_t status);

#ifdef __cplusplus
}
#endif
#endif

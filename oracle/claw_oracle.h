/*
 * claw_oracle.h -- plain, slow CPU FP64 oracle of the wave-propagation level-step
 * (Qin, LeVeque & Motley, "Accelerating wave-propagation algorithms with adaptive
 * mesh refinement using the GPU", arXiv:1808.02638).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or call this
 * code: only the test-suite, the smoke check and the CPU-baseline leg of the benchmark
 * use it.  It shares no code, header, table or constant with the CUDA library.
 *
 * Storage convention (shared with the inputs, not with any code): a patch with an
 * nx x ny interior and mbc ghost layers is stored as planes of W x H doubles,
 * W = nx + 2 mbc, H = ny + 2 mbc, x fastest; cell (i, j) with i in [-mbc, nx+mbc-1]
 * lives at (i + mbc) + (j + mbc) * W.  q = (p, u, v) is three such planes back to back.
 */
#ifndef CLAW_ORACLE_H
#define CLAW_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* limiter ids: 0 none (Lax-Wendroff), 1 minmod, 2 superbee, 3 van Leer, 4 MC */
double orc_philim(int limiter, double theta);

/* The normal Riemann problem at one x-edge (left state pl, ul with rho_l, K_l; right state
 * pr, ur with rho_r, K_r).  waves[0..5] = W1 (p, u, v), W2 (p, u, v); speeds[0..1]. */
void orc_riemann_x(double pl, double ul, double rhol, double Kl,
                   double pr, double ur, double rhor, double Kr,
                   double* waves, double* speeds);

/* One unsplit step on one patch from Q^n with ghosts filled (Eq. wave_form_2d_2nd_order).
 * rho, K: one plane each (ghosts included).  qnew: interior cells written, the rest
 * untouched.  *smax: largest |s| over the edges whose waves enter the update.
 * transverse: 0 none, 1 fluctuations only, 2 fluctuations with the correction flux.
 * Returns 0, or -1 on bad arguments / allocation failure. */
int orc_step(int nx, int ny, int mbc, double dx, double dy, double dt,
             int order, int transverse, int limiter,
             const double* q, const double* rho, const double* K,
             double* qnew, double* smax);

/* orc_step that also returns, in `edges` (18 planes of the patch layout, or NULL), the
 * per-edge quantities of the step: A-dQ, A+dQ at x-edges, B-dQ, B+dQ at y-edges (3 planes
 * each, stored at the edge's right / upper cell), the x-edge correction-plus-transverse flux
 * F~ and the y-edge flux G~ (same storage).  The conservation fix of Sec. 2.3 reads them. */
int orc_step_edges(int nx, int ny, int mbc, double dx, double dy, double dt,
                   int order, int transverse, int limiter,
                   const double* q, const double* rho, const double* K,
                   double* qnew, double* smax, double* edges);

/* Reverse mode of orc_step for a frozen dt: given lam_new (adjoint of qnew, interior
 * cells only are read) accumulate (+=) the adjoint of q (all cells incl. ghosts) into
 * lam_q, and of rho, K (all cells) into g_rho, g_K. */
int orc_step_adjoint(int nx, int ny, int mbc, double dx, double dy, double dt,
                     int order, int transverse, int limiter,
                     const double* q, const double* rho, const double* K,
                     const double* lam_new, double* lam_q, double* g_rho, double* g_K);

/* Physical boundary ghosts of a patch that covers the whole domain.
 * bc[4] = x-low, x-high, y-low, y-high: 0 zero-order extrapolation, 1 periodic,
 * 2 solid wall (mirror, normal velocity negated).  ncomp = 3 for q (u is component 1,
 * v component 2), 1 for a scalar field (no sign flips). */
int orc_fill_bc(int nx, int ny, int mbc, int ncomp, const int* bc, double* a);
/* adjoint of orc_fill_bc: ghost adjoints are added into their sources and zeroed */
int orc_fill_bc_adjoint(int nx, int ny, int mbc, int ncomp, const int* bc, double* g);

/* max of c = sqrt(K/rho) over the cells next to the edges the step solves for its update */
double orc_cfl_max(int nx, int ny, int mbc, const double* rho, const double* K);

/* ---------------------------------------------------------------- shallow water (swe_oracle.c)
 * q = (h, hu, hv).  One unsplit step of the same form with the Roe solver; grav = g.
 * Returns 0, -1 on bad arguments / allocation failure, -2 if a cell of the stencil has
 * h <= 0.  *smax: largest |s| over the edges whose waves enter the update. */
int orc_swe_step(int nx, int ny, int mbc, double dx, double dy, double dt,
                 int order, int transverse, int limiter, double grav,
                 const double* q, double* qnew, double* smax);
/* orc_swe_step that also returns the 18 per-edge planes of orc_step_edges (or NULL) */
int orc_swe_step_edges(int nx, int ny, int mbc, double dx, double dy, double dt,
                       int order, int transverse, int limiter, double grav,
                       const double* q, double* qnew, double* smax, double* edges);
/* Roe solve at one x-edge: waves[0..8] = W1, W2, W3 (h, hu, hv); speeds[0..2] */
void orc_swe_roe_x(double hl, double hul, double hvl, double hr, double hur, double hvr,
                   double grav, double* waves, double* speeds);
/* max over the cells [-1, nx] x [-1, ny] of |u| + sqrt(g h) and |v| + sqrt(g h) */
double orc_swe_cfl_max(int nx, int ny, int mbc, double grav, const double* q);

/* ---------------------------------------------------------------- AMR (one run) */
typedef struct { int32_t ilo, jlo, nx, ny; int64_t off; } orc_box;  /* off: element offset of
                                                                        the box's first plane */

/* Fill every ghost cell of every box of a level (Sec. 2.2 ghost rules):
 *   value(g) = value at b(g), b = the physical-boundary map of the level's domain
 *   [0,NX) x [0,NY) (clamp / wrap / mirror), where a cell inside the domain takes, in this
 *   order, the box's own interior, another box's interior on the same level, or the
 *   space-time interpolation from the coarser level (cboxes, cold, cnew at fraction tau,
 *   refinement ratio r).  ncomp planes per box.  Returns 0, or -2 if a cell needs the coarse
 *   level and none covers it (improper nesting). */
int orc_level_fill_ghost(int nb, const orc_box* boxes, double* pool, int ncomp, int mbc,
                         int NX, int NY, const int* bc,
                         int ncb, const orc_box* cboxes, const double* cold, const double* cnew,
                         double tau, int r, int copy_only);
/* copy_only != 0: ghosts that would need the coarser level are left unchanged (coefficient
 * fields of finer levels are given, not interpolated) */

/* coarse := mean of the r*r fine cells over every coarse interior cell covered by a fine box */
int orc_average_down(int nf, const orc_box* fboxes, const double* fpool,
                     int nc, const orc_box* cboxes, double* cpool, int ncomp, int mbc, int r);

/* Interpolated value of component m at fine cell (fi, fj) (used by the fill above and
 * exposed for the pin tests). */
int orc_interp_cell(int ncb, const orc_box* cboxes, const double* cold, const double* cnew,
                    double tau, int r, int ncomp, int mbc, int cNX, int cNY, const int* bc,
                    int fi, int fj, double* out /* ncomp */);

/* adjoints of the two AMR transfers above (for the batched adjoint):
 * level fill: ghost adjoints flow to their sources (own/other boxes of the level, or the
 * coarse old/new pools through the interpolation); the ghost adjoints are zeroed. */
int orc_level_fill_ghost_adjoint(int nb, const orc_box* boxes, double* gpool, int ncomp, int mbc,
                                 int NX, int NY, const int* bc,
                                 int ncb, const orc_box* cboxes, double* gcold, double* gcnew,
                                 const double* cold, const double* cnew, double tau, int r,
                                 int copy_only);
int orc_average_down_adjoint(int nf, const orc_box* fboxes, double* gfpool,
                             int nc, const orc_box* cboxes, double* gcpool, int ncomp, int mbc, int r);

#ifdef __cplusplus
}
#endif
#endif

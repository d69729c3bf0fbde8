/*
 * swe_oracle.c -- plain CPU FP64 oracle of the unsplit wave-propagation step of
 * arXiv:1808.02638 (Sec. 2.1, Eq. wave_form_2d_2nd_order) for a nonlinear system.  The
 * paper's framework takes any hyperbolic system for which a normal and a transverse Riemann
 * solver are supplied (Sec. 3.1, Sec. 3.3 "Riemann Solvers"); this file supplies them for the
 * two-dimensional shallow water equations on a flat bottom,
 *     h_t  + (hu)_x              + (hv)_y              = 0
 *     hu_t + (hu^2 + g h^2/2)_x  + (huv)_y             = 0
 *     hv_t + (huv)_x             + (hv^2 + g h^2/2)_y  = 0,
 * q = (h, hu, hv), with the Roe linearisation (LeVeque 2002, Sec. 15.3 and 21.7).
 *
 * TEST INFRASTRUCTURE ONLY -- used by the tests, the smoke check and the CPU-baseline leg of
 * the benchmark; never by the product path.  Compiled like claw_oracle.c (-O2
 * -ffp-contract=off, no fast-math): every operation below is one IEEE-754 double operation
 * in the order written.
 *
 * Normal solve at an edge with left state L, right state R, normal momentum component n and
 * tangential component t (x-edges: n = hu, t = hv; y-edges: n = hv, t = hu):
 *   Roe state   hbar = (h_L + h_R)/2,
 *               un = (sqrt(h_L) un_L + sqrt(h_R) un_R) / (sqrt(h_L) + sqrt(h_R)), ut alike,
 *               c = sqrt(g hbar);
 *   speeds      s1 = un - c, s2 = un, s3 = un + c;
 *   vectors     r1 = (1, un - c, ut), r2 = (0, 0, 1), r3 = (1, un + c, ut)   [(h, n, t)];
 *   strengths   dQ = Q_R - Q_L = sum_p alpha_p r_p:
 *               alpha1 = ((un + c) dh - dn) / (2c), alpha2 = dt - ut dh,
 *               alpha3 = (dn - (un - c) dh) / (2c);
 *   waves       W_p = alpha_p r_p;  A-dQ = sum_p min(s_p, 0) W_p, A+dQ = sum_p max(s_p, 0) W_p
 *               (no entropy fix).
 * Limiter and correction flux as for acoustics: theta_p = W_p(upwind edge).W_p / W_p.W_p,
 * W~_p = phi(theta_p) W_p, F~ = 1/2 sum_p |s_p| (1 - dt/dx |s_p|) W~_p.
 * Transverse solve: the fluctuation entering a cell (A+dQ - C into the right cell, A-dQ + C
 * into the left one, C = 2 F~) is decomposed on the eigenvectors of the transverse Jacobian
 * at the same Roe state,
 *   (1, un, ut - c), (0, 1, 0), (1, un, ut + c)   with speeds ut - c, ut, ut + c,
 *   beta1 = ((ut + c) d_h - d_t) / (2c), beta2 = d_n - un d_h, beta3 = (d_t - (ut - c) d_h) / (2c),
 * and dt/(2 dx) times its down-going part (negative speeds) is subtracted from G~ below the
 * cell, its up-going part from G~ above the cell.
 *
 * Readings of points the paper leaves to the solver (same as the CUDA library):
 *   - the transverse split of an edge's fluctuations uses that edge's Roe state;
 *   - wet states only: a cell with h <= 0 in the stencil is an error (-2);
 *   - s_max is the largest |s_p| over the edges whose waves enter the update.
 */
#include "claw_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int nx, ny, mbc, W, H;
} sgeom;

static inline long SIC(const sgeom* g, int i, int j) { return (long)(i + g->mbc) + (long)(j + g->mbc) * g->W; }
static inline long SCELL(const sgeom* g, int dir, int a, int l) { return dir == 0 ? SIC(g, a, l) : SIC(g, l, a); }

/* per-edge record of one normal solve */
typedef struct {
    double w[3][3];     /* waves W1..W3 (components h, hu, hv) */
    double s[3];        /* speeds */
    double un, ut, c;   /* Roe state: normal / tangential velocity, celerity */
    double amdq[3], apdq[3];
} swe_edge;

/* Roe solve between cells L and R; mn / mt = component index of the normal / tangential
 * momentum. */
static void roe_solve(const double* hq, const double* nq, const double* tq, long L, long R,
                      int mn, int mt, double grav, swe_edge* e)
{
    double hl = hq[L], hr = hq[R];
    double sl = sqrt(hl), sr = sqrt(hr);
    double unl = nq[L] / hl, unr = nq[R] / hr;
    double utl = tq[L] / hl, utr = tq[R] / hr;
    double un = (sl * unl + sr * unr) / (sl + sr);
    double ut = (sl * utl + sr * utr) / (sl + sr);
    double c = sqrt(grav * ((hl + hr) / 2.0));
    double dh = hr - hl, dn = nq[R] - nq[L], dt = tq[R] - tq[L];
    double a1 = ((un + c) * dh - dn) / (2.0 * c);
    double a2 = dt - ut * dh;
    double a3 = (dn - (un - c) * dh) / (2.0 * c);
    e->un = un; e->ut = ut; e->c = c;
    e->s[0] = un - c; e->s[1] = un; e->s[2] = un + c;
    e->w[0][0] = a1; e->w[0][mn] = a1 * (un - c); e->w[0][mt] = a1 * ut;
    e->w[1][0] = 0.0; e->w[1][mn] = 0.0; e->w[1][mt] = a2;
    e->w[2][0] = a3; e->w[2][mn] = a3 * (un + c); e->w[2][mt] = a3 * ut;
    for (int m = 0; m < 3; ++m) {
        e->amdq[m] = 0.0;
        e->apdq[m] = 0.0;
        for (int p = 0; p < 3; ++p) {
            if (e->s[p] < 0.0) e->amdq[m] += e->s[p] * e->w[p][m];
            else e->apdq[m] += e->s[p] * e->w[p][m];
        }
    }
}

/* transverse split of delta with the edge's Roe state: bm (negative speeds), bp (positive) */
static void swe_tsplit(const double* d, int mn, int mt, const swe_edge* e, double* bm, double* bp)
{
    double un = e->un, ut = e->ut, c = e->c;
    double b1 = ((ut + c) * d[0] - d[mt]) / (2.0 * c);
    double b2 = d[mn] - un * d[0];
    double b3 = (d[mt] - (ut - c) * d[0]) / (2.0 * c);
    double sp[3] = {ut - c, ut, ut + c};
    double v[3][3];
    v[0][0] = b1; v[0][mn] = b1 * un; v[0][mt] = b1 * (ut - c);
    v[1][0] = 0.0; v[1][mn] = b2; v[1][mt] = 0.0;
    v[2][0] = b3; v[2][mn] = b3 * un; v[2][mt] = b3 * (ut + c);
    for (int m = 0; m < 3; ++m) {
        bm[m] = 0.0;
        bp[m] = 0.0;
        for (int p = 0; p < 3; ++p) {
            if (sp[p] < 0.0) bm[m] += sp[p] * v[p][m];
            else bp[m] += sp[p] * v[p][m];
        }
    }
}

typedef struct {
    const sgeom* g;
    int order, transverse, limiter;
    double grav;
    const double *h, *hu, *hv;
} swe_ctx;

static void swe_sweep(const swe_ctx* S, int dir, double lam, swe_edge* rec,
                      double* amdq, double* apdq, double* fn, double* ft, double* smax)
{
    const sgeom* g = S->g;
    const int nn = dir == 0 ? g->nx : g->ny;
    const int nt = dir == 0 ? g->ny : g->nx;
    const int mn = dir == 0 ? 1 : 2;
    const int mt = dir == 0 ? 2 : 1;
    const long pl = (long)g->W * g->H;
    const double* nq = dir == 0 ? S->hu : S->hv;
    const double* tq = dir == 0 ? S->hv : S->hu;

    for (int l = -1; l <= nt; ++l) {
        for (int a = -1; a <= nn + 1; ++a) {
            swe_edge* e = &rec[a + 1];
            long L = SCELL(g, dir, a - 1, l), R = SCELL(g, dir, a, l);
            roe_solve(S->h, nq, tq, L, R, mn, mt, S->grav, e);
            for (int m = 0; m < 3; ++m) {
                amdq[m * pl + R] = e->amdq[m];
                apdq[m * pl + R] = e->apdq[m];
            }
        }
        for (int a = 0; a <= nn; ++a) {
            swe_edge* e = &rec[a + 1];
            double wt[3][3];
            for (int p = 0; p < 3; ++p) {
                double wn2 = 0.0;
                for (int m = 0; m < 3; ++m) wn2 += e->w[p][m] * e->w[p][m];
                double phi;
                if (S->limiter == 0) phi = 1.0;
                else if (wn2 == 0.0) phi = 0.0;
                else {
                    const swe_edge* up = e->s[p] > 0.0 ? &rec[a] : &rec[a + 2];
                    double dot = 0.0;
                    for (int m = 0; m < 3; ++m) dot += up->w[p][m] * e->w[p][m];
                    phi = orc_philim(S->limiter, dot / wn2);
                }
                for (int m = 0; m < 3; ++m) wt[p][m] = phi * e->w[p][m];
                double as = fabs(e->s[p]);
                if (as > *smax) *smax = as;
            }
            double cq[3] = {0.0, 0.0, 0.0};
            if (S->order == 2) {
                for (int m = 0; m < 3; ++m)
                    for (int p = 0; p < 3; ++p) {
                        double as = fabs(e->s[p]);
                        cq[m] += as * (1.0 - lam * as) * wt[p][m];
                    }
                long E = SCELL(g, dir, a, l);
                for (int m = 0; m < 3; ++m) fn[m * pl + E] += 0.5 * cq[m];
            }
            if (S->transverse) {
                double cw = (S->transverse == 2 && S->order == 2) ? 1.0 : 0.0;
                double dl[3], dr[3];
                for (int m = 0; m < 3; ++m) {
                    dl[m] = e->amdq[m] + cw * cq[m];
                    dr[m] = e->apdq[m] - cw * cq[m];
                }
                for (int side = 0; side < 2; ++side) {
                    int k = side == 0 ? a - 1 : a;
                    double bm[3], bp[3];
                    swe_tsplit(side == 0 ? dl : dr, mn, mt, e, bm, bp);
                    long e0 = SCELL(g, dir, k, l), e1 = SCELL(g, dir, k, l + 1);
                    for (int m = 0; m < 3; ++m) {
                        ft[m * pl + e0] -= 0.5 * lam * bm[m];
                        ft[m * pl + e1] -= 0.5 * lam * bp[m];
                    }
                }
            }
        }
    }
}

static int salloc(double** out, long n)
{
    *out = (double*)calloc((size_t)n, sizeof(double));
    return *out ? 0 : -1;
}

/* One step of every interior cell; with `edges` not NULL it also receives the six per-edge
 * planes-of-3 arrays A-dQ, A+dQ (x-edges), B-dQ, B+dQ (y-edges), F~, G~ stored at the edge's
 * right / upper cell, as orc_step_edges does for acoustics (the conservation fix reads them). */
int orc_swe_step_edges(int nx, int ny, int mbc, double dx, double dy, double dt,
                       int order, int transverse, int limiter, double grav,
                       const double* q, double* qnew, double* smax, double* edges)
{
    if (nx < 1 || ny < 1 || mbc < 2 || !(dx > 0) || !(dy > 0) || !(grav > 0)) return -1;
    sgeom G = {nx, ny, mbc, nx + 2 * mbc, ny + 2 * mbc};
    const long pl = (long)G.W * G.H;
    /* every cell the sweeps read: rows -1..ny of columns -2..nx+1 and columns -1..nx of
     * rows -2..ny+1 */
    for (int j = -2; j <= ny + 1; ++j)
        for (int i = -2; i <= nx + 1; ++i) {
            int inx = (j >= -1 && j <= ny), iny = (i >= -1 && i <= nx);
            if ((inx || iny) && !(q[SIC(&G, i, j)] > 0.0)) return -2;
        }
    int nmax = (nx > ny ? nx : ny) + 3;
    double *amx, *apx, *amy, *apy, *F, *Gt;
    swe_edge* rec = (swe_edge*)calloc((size_t)nmax, sizeof(swe_edge));
    if (!rec || salloc(&amx, 3 * pl) || salloc(&apx, 3 * pl) || salloc(&amy, 3 * pl) ||
        salloc(&apy, 3 * pl) || salloc(&F, 3 * pl) || salloc(&Gt, 3 * pl))
        return -1;
    swe_ctx S = {&G, order, transverse, limiter, grav, q, q + pl, q + 2 * pl};
    double sm = 0.0;
    swe_sweep(&S, 0, dt / dx, rec, amx, apx, F, Gt, &sm);
    swe_sweep(&S, 1, dt / dy, rec, amy, apy, Gt, F, &sm);
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            long k = SIC(&G, i, j), kx = SIC(&G, i + 1, j), ky = SIC(&G, i, j + 1);
            for (int m = 0; m < 3; ++m) {
                long o = m * pl;
                qnew[o + k] = q[o + k]
                    - dt / dx * (apx[o + k] + amx[o + kx])
                    - dt / dy * (apy[o + k] + amy[o + ky])
                    - dt / dx * (F[o + kx] - F[o + k])
                    - dt / dy * (Gt[o + ky] - Gt[o + k]);
            }
        }
    if (smax) *smax = sm;
    if (edges) {
        const double* src[6] = {amx, apx, amy, apy, F, Gt};
        for (int a = 0; a < 6; ++a) memcpy(edges + (long)a * 3 * pl, src[a], sizeof(double) * 3 * pl);
    }
    free(rec); free(amx); free(apx); free(amy); free(apy); free(F); free(Gt);
    return 0;
}

int orc_swe_step(int nx, int ny, int mbc, double dx, double dy, double dt,
                 int order, int transverse, int limiter, double grav,
                 const double* q, double* qnew, double* smax)
{
    return orc_swe_step_edges(nx, ny, mbc, dx, dy, dt, order, transverse, limiter, grav, q, qnew, smax, 0);
}

void orc_swe_roe_x(double hl, double hul, double hvl, double hr, double hur, double hvr,
                   double grav, double* waves, double* speeds)
{
    double h[2] = {hl, hr}, hu[2] = {hul, hur}, hv[2] = {hvl, hvr};
    swe_edge e;
    roe_solve(h, hu, hv, 0, 1, 1, 2, grav, &e);
    for (int p = 0; p < 3; ++p) {
        speeds[p] = e.s[p];
        for (int m = 0; m < 3; ++m) waves[3 * p + m] = e.w[p][m];
    }
}

double orc_swe_cfl_max(int nx, int ny, int mbc, double grav, const double* q)
{
    sgeom G = {nx, ny, mbc, nx + 2 * mbc, ny + 2 * mbc};
    const long pl = (long)G.W * G.H;
    double s = 0.0;
    for (int j = -1; j <= ny; ++j)
        for (int i = -1; i <= nx; ++i) {
            long k = SIC(&G, i, j);
            double h = q[k];
            double c = sqrt(grav * h);
            double su = fabs(q[pl + k] / h) + c, sv = fabs(q[2 * pl + k] / h) + c;
            if (su > s) s = su;
            if (sv > s) s = sv;
        }
    return s;
}

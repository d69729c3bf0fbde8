/*
 * claw_oracle.c -- plain CPU FP64 oracle of the wave-propagation method of
 * arXiv:1808.02638 (Sec. 2.1, Eq. wave_form_2d_2nd_order; Sec. 4.1 acoustics system),
 * with the AMR ghost rules of Sec. 2.2 and the "updating" average of Sec. 2.3.
 *
 * TEST INFRASTRUCTURE ONLY -- used by the tests, the smoke check and the CPU-baseline
 * leg of the benchmark; never by the product path.  Compiled with -O2
 * -ffp-contract=off and no fast-math, so every operation below is one IEEE-754 double
 * operation in the order written.
 *
 * The paper defers the Riemann solver, limiter and transverse solver to LeVeque (2002);
 * the forms used here are the textbook ones specialised to the paper's acoustics matrices
 * A, B (Sec. 4.1) with cell-wise rho, K:  c = sqrt(K/rho), Z = rho c = sqrt(K rho).
 *   normal solve at an edge with left cell L, right cell R, jump (dp, dn) of pressure and
 *   normal velocity:   a1 = (-dp + Z_R dn)/(Z_L+Z_R),  a2 = (dp + Z_L dn)/(Z_L+Z_R),
 *   W1 = a1 (-Z_L, 1_n), s1 = -c_L ;  W2 = a2 (Z_R, 1_n), s2 = +c_R .
 *   limiter: theta = W(upwind edge).W / W.W, W~ = phi(theta) W  (W.W = 0 gives W~ = 0).
 *   correction flux  F~ = 1/2 sum |s| (1 - dt/dx |s|) W~.
 *   transverse: the fluctuations A-dQ + C (into the left cell) and A+dQ - C (into the
 *   right cell), C = sum |s|(1 - dt/dx|s|) W~ (full weight, transverse = 2), are split
 *   across the neighbouring transverse interfaces with the impedances of the cells
 *   below / at / above and subtract dt/(2 dx) times the split parts from G~ there.
 *
 * Ambiguities of the paper settled here (same readings as the CUDA library):
 *   - speeds s1 = -c_L, s2 = +c_R at a material interface;
 *   - the transverse split propagates the correction with full weight;
 *   - unsplit: both sweeps read Q^n;
 *   - x-sweeps cover rows -1..ny, y-sweeps columns -1..nx, two ghost layers.
 */
#include "claw_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ limiters */

/* phi(theta) and its derivative along the branch the value takes */
static double philim_d(int limiter, double th, double* dphi)
{
    double d = 0.0, phi;
    switch (limiter) {
    case 0: /* no limiting */
        phi = 1.0;
        break;
    case 1: /* minmod: max(0, min(1, theta)) */
        if (th <= 0.0) phi = 0.0;
        else if (th < 1.0) { phi = th; d = 1.0; }
        else phi = 1.0;
        break;
    case 2: { /* superbee: max(0, min(1, 2 theta), min(2, theta)) */
        double a = (2.0 * th < 1.0) ? 2.0 * th : 1.0;
        double da = (2.0 * th < 1.0) ? 2.0 : 0.0;
        double b = (th < 2.0) ? th : 2.0;
        double db = (th < 2.0) ? 1.0 : 0.0;
        if (a >= b) { phi = a; d = da; } else { phi = b; d = db; }
        if (phi <= 0.0) { phi = 0.0; d = 0.0; }
        break;
    }
    case 3: /* van Leer: (theta + |theta|) / (1 + |theta|) */
        if (th > 0.0) { phi = (th + th) / (1.0 + th); d = 2.0 / ((1.0 + th) * (1.0 + th)); }
        else phi = 0.0;
        break;
    case 4: { /* MC: max(0, min((1+theta)/2, 2, 2 theta)) */
        double m = (1.0 + th) / 2.0, dm = 0.5;
        if (2.0 < m) { m = 2.0; dm = 0.0; }
        if (2.0 * th < m) { m = 2.0 * th; dm = 2.0; }
        if (m <= 0.0) { m = 0.0; dm = 0.0; }
        phi = m; d = dm;
        break;
    }
    default:
        phi = 0.0;
    }
    if (dphi) *dphi = d;
    return phi;
}

double orc_philim(int limiter, double theta) { return philim_d(limiter, theta, 0); }

/* ------------------------------------------------------------------ geometry */

typedef struct {
    int nx, ny, mbc, W, H;
} geom;

static inline long IC(const geom* g, int i, int j) { return (long)(i + g->mbc) + (long)(j + g->mbc) * g->W; }

/* a sweep runs along "a" (edge index) across lines "l"; dir 0 = x, 1 = y */
static inline long CELL(const geom* g, int dir, int a, int l) { return dir == 0 ? IC(g, a, l) : IC(g, l, a); }

/* per-edge record of the forward sweep (kept for the reverse pass) */
typedef struct {
    double w[2][3];   /* waves W1, W2 (components p, u, v) */
    double s[2];      /* speeds */
    double a[2];      /* wave strengths */
    double amdq[3], apdq[3];
} edge_rec;

/* one transverse split: delta in the cell "mid" between cells lo (below/left) and hi
 * (above/right) across the transverse direction.  tn = transverse normal component index. */
static void tsplit(const double* delta, int tn, double zlo, double zmid, double zhi,
                   double clo, double chi, double* bm, double* bp)
{
    double dm = (-delta[0] + zmid * delta[tn]) / (zlo + zmid);
    double dpc = (delta[0] + zmid * delta[tn]) / (zmid + zhi);
    /* down/left-going: speed -c_lo, eigenvector (-Z_lo, 1_t) */
    bm[0] = -clo * dm * (-zlo);
    bm[1] = 0.0; bm[2] = 0.0;
    bm[tn] = -clo * dm;
    /* up/right-going: speed +c_hi, eigenvector (Z_hi, 1_t) */
    bp[0] = chi * dpc * zhi;
    bp[1] = 0.0; bp[2] = 0.0;
    bp[tn] = chi * dpc;
}

typedef struct {
    const geom* g;
    int order, transverse, limiter;
    const double *p, *u, *v;  /* Q^n planes */
    const double *c, *Z;      /* per-cell sound speed and impedance */
} step_ctx;

/* Forward sweep in direction dir.  Writes the fluctuations (stored at the edge's right
 * cell), adds 1/2 C to the normal correction flux fn and the transverse terms to ft. */
static void sweep_fwd(const step_ctx* S, int dir, double lam, edge_rec* rec,
                      double* amdq, double* apdq, double* fn, double* ft, double* smax)
{
    const geom* g = S->g;
    const int nn = dir == 0 ? g->nx : g->ny;   /* cells along the sweep */
    const int nt = dir == 0 ? g->ny : g->nx;   /* lines */
    const int mn = dir == 0 ? 1 : 2;           /* normal velocity component */
    const int mt = dir == 0 ? 2 : 1;           /* transverse velocity component */
    const long pl = (long)g->W * g->H;
    const double* qn = dir == 0 ? S->u : S->v;

    for (int l = -1; l <= nt; ++l) {
        /* normal Riemann problems at edges a in [-1, nn+1] (edge a between a-1 and a) */
        for (int a = -1; a <= nn + 1; ++a) {
            edge_rec* e = &rec[a + 1];
            long L = CELL(g, dir, a - 1, l), R = CELL(g, dir, a, l);
            double dp = S->p[R] - S->p[L];
            double dn = qn[R] - qn[L];
            double zl = S->Z[L], zr = S->Z[R];
            double a1 = (-dp + zr * dn) / (zl + zr);
            double a2 = (dp + zl * dn) / (zl + zr);
            e->a[0] = a1; e->a[1] = a2;
            e->w[0][0] = -a1 * zl; e->w[0][mn] = a1; e->w[0][mt] = 0.0;
            e->w[1][0] = a2 * zr;  e->w[1][mn] = a2; e->w[1][mt] = 0.0;
            e->s[0] = -S->c[L];
            e->s[1] = S->c[R];
            for (int m = 0; m < 3; ++m) {
                e->amdq[m] = 0.0; e->apdq[m] = 0.0;
                for (int w = 0; w < 2; ++w) {
                    if (e->s[w] < 0.0) e->amdq[m] += e->s[w] * e->w[w][m];
                    else e->apdq[m] += e->s[w] * e->w[w][m];
                }
                amdq[m * pl + R] = e->amdq[m];
                apdq[m * pl + R] = e->apdq[m];
            }
        }
        /* limiter, correction flux and transverse propagation at edges a in [0, nn] */
        for (int a = 0; a <= nn; ++a) {
            edge_rec* e = &rec[a + 1];
            double wt[2][3];
            for (int w = 0; w < 2; ++w) {
                double wn2 = 0.0;
                for (int m = 0; m < 3; ++m) wn2 += e->w[w][m] * e->w[w][m];
                double phi;
                if (S->limiter == 0) phi = 1.0;
                else if (wn2 == 0.0) phi = 0.0;
                else {
                    const edge_rec* up = e->s[w] > 0.0 ? &rec[a] : &rec[a + 2];
                    double dot = 0.0;
                    for (int m = 0; m < 3; ++m) dot += up->w[w][m] * e->w[w][m];
                    phi = philim_d(S->limiter, dot / wn2, 0);
                }
                for (int m = 0; m < 3; ++m) wt[w][m] = phi * e->w[w][m];
                double as = fabs(e->s[w]);
                if (as > *smax) *smax = as;
            }
            double cq[3] = {0.0, 0.0, 0.0};
            if (S->order == 2) {
                for (int m = 0; m < 3; ++m)
                    for (int w = 0; w < 2; ++w) {
                        double as = fabs(e->s[w]);
                        cq[m] += as * (1.0 - lam * as) * wt[w][m];
                    }
                long E = CELL(g, dir, a, l);
                for (int m = 0; m < 3; ++m) fn[m * pl + E] += 0.5 * cq[m];
            }
            if (S->transverse) {
                double cw = (S->transverse == 2 && S->order == 2) ? 1.0 : 0.0;
                double dl[3], dr[3];  /* into cell a-1, into cell a */
                for (int m = 0; m < 3; ++m) {
                    dl[m] = e->amdq[m] + cw * cq[m];
                    dr[m] = e->apdq[m] - cw * cq[m];
                }
                for (int side = 0; side < 2; ++side) {
                    int k = side == 0 ? a - 1 : a;
                    const double* d = side == 0 ? dl : dr;
                    long lo = CELL(g, dir, k, l - 1), mid = CELL(g, dir, k, l), hi = CELL(g, dir, k, l + 1);
                    double bm[3], bp[3];
                    tsplit(d, mt, S->Z[lo], S->Z[mid], S->Z[hi], S->c[lo], S->c[hi], bm, bp);
                    long e0 = CELL(g, dir, k, l), e1 = CELL(g, dir, k, l + 1);
                    for (int m = 0; m < 3; ++m) {
                        ft[m * pl + e0] -= 0.5 * lam * bm[m];
                        ft[m * pl + e1] -= 0.5 * lam * bp[m];
                    }
                }
            }
        }
    }
}

static int alloc_zero(double** out, long n)
{
    *out = (double*)calloc((size_t)n, sizeof(double));
    return *out ? 0 : -1;
}

static void cell_speeds(const geom* g, const double* rho, const double* K, double* c, double* Z)
{
    long n = (long)g->W * g->H;
    for (long k = 0; k < n; ++k) {
        c[k] = sqrt(K[k] / rho[k]);
        Z[k] = sqrt(K[k] * rho[k]);
    }
}

/* One step of every interior cell (Eq. wave_form_2d_2nd_order).  When `edges` is not NULL it
 * receives six planes-of-3 arrays of the patch layout: A-dQ, A+dQ at x-edges, B-dQ, B+dQ at
 * y-edges (each stored at the edge's right / upper cell), the x-edge correction-plus-transverse
 * flux F~ and the y-edge flux G~ (same storage): the per-edge quantities the conservation fix of
 * Sec. 2.3 reads at coarse-fine interfaces. */
int orc_step_edges(int nx, int ny, int mbc, double dx, double dy, double dt,
                   int order, int transverse, int limiter,
                   const double* q, const double* rho, const double* K,
                   double* qnew, double* smax, double* edges)
{
    if (nx < 1 || ny < 1 || mbc < 2 || !(dx > 0) || !(dy > 0)) return -1;
    geom G = {nx, ny, mbc, nx + 2 * mbc, ny + 2 * mbc};
    const geom* g = &G;
    long pl = (long)G.W * G.H;
    int nmax = (nx > ny ? nx : ny) + 3;
    double *c, *Z, *amx, *apx, *amy, *apy, *F, *Gt;
    edge_rec* rec = (edge_rec*)calloc((size_t)nmax, sizeof(edge_rec));
    if (!rec || alloc_zero(&c, pl) || alloc_zero(&Z, pl) || alloc_zero(&amx, 3 * pl) ||
        alloc_zero(&apx, 3 * pl) || alloc_zero(&amy, 3 * pl) || alloc_zero(&apy, 3 * pl) ||
        alloc_zero(&F, 3 * pl) || alloc_zero(&Gt, 3 * pl))
        return -1;
    cell_speeds(g, rho, K, c, Z);
    step_ctx S = {g, order, transverse, limiter, q, q + pl, q + 2 * pl, c, Z};
    double sm = 0.0;
    sweep_fwd(&S, 0, dt / dx, rec, amx, apx, F, Gt, &sm);
    sweep_fwd(&S, 1, dt / dy, rec, amy, apy, Gt, F, &sm);
    /* conservative update of the interior (Eq. wave_form_2d_2nd_order) */
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            long k = IC(g, i, j), kx = IC(g, i + 1, j), ky = IC(g, i, j + 1);
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
    free(rec); free(c); free(Z); free(amx); free(apx); free(amy); free(apy); free(F); free(Gt);
    return 0;
}

int orc_step(int nx, int ny, int mbc, double dx, double dy, double dt,
             int order, int transverse, int limiter,
             const double* q, const double* rho, const double* K,
             double* qnew, double* smax)
{
    return orc_step_edges(nx, ny, mbc, dx, dy, dt, order, transverse, limiter, q, rho, K, qnew, smax, 0);
}

void orc_riemann_x(double pl, double ul, double rhol, double Kl,
                   double pr, double ur, double rhor, double Kr,
                   double* waves, double* speeds)
{
    double zl = sqrt(Kl * rhol), zr = sqrt(Kr * rhor);
    double dp = pr - pl, du = ur - ul;
    double a1 = (-dp + zr * du) / (zl + zr);
    double a2 = (dp + zl * du) / (zl + zr);
    waves[0] = -a1 * zl; waves[1] = a1; waves[2] = 0.0;
    waves[3] = a2 * zr;  waves[4] = a2; waves[5] = 0.0;
    speeds[0] = -sqrt(Kl / rhol);
    speeds[1] = sqrt(Kr / rhor);
}

/* ------------------------------------------------------------ reverse mode */

/* adjoint of tsplit: accumulates into dbar (3), and the cell coefficient adjoints */
static void tsplit_adj(const double* delta, int tn, double zlo, double zmid, double zhi,
                       double clo, double chi, const double* bmbar, const double* bpbar,
                       double* dbar, double* zlo_b, double* zmid_b, double* zhi_b,
                       double* clo_b, double* chi_b)
{
    double den_m = zlo + zmid, den_p = zmid + zhi;
    double dm = (-delta[0] + zmid * delta[tn]) / den_m;
    double dpc = (delta[0] + zmid * delta[tn]) / den_p;
    /* bm = (clo*dm*zlo, [tn]: -clo*dm) */
    double dm_b = bmbar[0] * clo * zlo - bmbar[tn] * clo;
    *clo_b += bmbar[0] * dm * zlo - bmbar[tn] * dm;
    *zlo_b += bmbar[0] * clo * dm;
    /* bp = (chi*dpc*zhi, [tn]: chi*dpc) */
    double dp_b = bpbar[0] * chi * zhi + bpbar[tn] * chi;
    *chi_b += bpbar[0] * dpc * zhi + bpbar[tn] * dpc;
    *zhi_b += bpbar[0] * chi * dpc;
    /* dm = (-d0 + zmid d_tn)/den_m */
    dbar[0] += -dm_b / den_m;
    dbar[tn] += zmid * dm_b / den_m;
    *zmid_b += delta[tn] * dm_b / den_m;
    *zlo_b += -dm_b * dm / den_m;
    *zmid_b += -dm_b * dm / den_m;
    /* dpc = (d0 + zmid d_tn)/den_p */
    dbar[0] += dp_b / den_p;
    dbar[tn] += zmid * dp_b / den_p;
    *zmid_b += delta[tn] * dp_b / den_p;
    *zmid_b += -dp_b * dpc / den_p;
    *zhi_b += -dp_b * dpc / den_p;
}

typedef struct {
    double *pb, *ub, *vb;  /* adjoints of Q^n planes */
    double *cb, *Zb;       /* adjoints of c, Z */
} adj_out;

static void sweep_adj(const step_ctx* S, int dir, double lam, edge_rec* rec, edge_rec* recb,
                      const double* amdqb, const double* apdqb, const double* fnb,
                      const double* ftb, adj_out* A)
{
    const geom* g = S->g;
    const int nn = dir == 0 ? g->nx : g->ny;
    const int nt = dir == 0 ? g->ny : g->nx;
    const int mn = dir == 0 ? 1 : 2;
    const int mt = dir == 0 ? 2 : 1;
    const long pl = (long)g->W * g->H;
    const double* qn = dir == 0 ? S->u : S->v;
    double* qnb = dir == 0 ? A->ub : A->vb;

    for (int l = -1; l <= nt; ++l) {
        /* recompute the forward records of this line */
        for (int a = -1; a <= nn + 1; ++a) {
            edge_rec* e = &rec[a + 1];
            long L = CELL(g, dir, a - 1, l), R = CELL(g, dir, a, l);
            double dp = S->p[R] - S->p[L];
            double dn = qn[R] - qn[L];
            double zl = S->Z[L], zr = S->Z[R];
            double a1 = (-dp + zr * dn) / (zl + zr);
            double a2 = (dp + zl * dn) / (zl + zr);
            e->a[0] = a1; e->a[1] = a2;
            e->w[0][0] = -a1 * zl; e->w[0][mn] = a1; e->w[0][mt] = 0.0;
            e->w[1][0] = a2 * zr;  e->w[1][mn] = a2; e->w[1][mt] = 0.0;
            e->s[0] = -S->c[L];
            e->s[1] = S->c[R];
            for (int m = 0; m < 3; ++m) {
                e->amdq[m] = 0.0; e->apdq[m] = 0.0;
                for (int w = 0; w < 2; ++w) {
                    if (e->s[w] < 0.0) e->amdq[m] += e->s[w] * e->w[w][m];
                    else e->apdq[m] += e->s[w] * e->w[w][m];
                }
            }
            memset(&recb[a + 1], 0, sizeof(edge_rec));
            /* fluctuation adjoints from the update */
            for (int m = 0; m < 3; ++m) {
                recb[a + 1].amdq[m] = amdqb[m * pl + R];
                recb[a + 1].apdq[m] = apdqb[m * pl + R];
            }
        }
        /* reverse of the limiter / correction / transverse part, edges a in [0, nn] */
        for (int a = 0; a <= nn; ++a) {
            edge_rec* e = &rec[a + 1];
            edge_rec* eb = &recb[a + 1];
            /* forward values */
            double wt[2][3], phi[2], dphi[2], wn2[2], dot[2];
            const edge_rec* up[2];
            for (int w = 0; w < 2; ++w) {
                wn2[w] = 0.0;
                for (int m = 0; m < 3; ++m) wn2[w] += e->w[w][m] * e->w[w][m];
                up[w] = e->s[w] > 0.0 ? &rec[a] : &rec[a + 2];
                dot[w] = 0.0;
                dphi[w] = 0.0;
                if (S->limiter == 0) phi[w] = 1.0;
                else if (wn2[w] == 0.0) phi[w] = 0.0;
                else {
                    for (int m = 0; m < 3; ++m) dot[w] += up[w]->w[w][m] * e->w[w][m];
                    phi[w] = philim_d(S->limiter, dot[w] / wn2[w], &dphi[w]);
                }
                for (int m = 0; m < 3; ++m) wt[w][m] = phi[w] * e->w[w][m];
            }
            double cq[3] = {0.0, 0.0, 0.0};
            if (S->order == 2)
                for (int m = 0; m < 3; ++m)
                    for (int w = 0; w < 2; ++w) {
                        double as = fabs(e->s[w]);
                        cq[m] += as * (1.0 - lam * as) * wt[w][m];
                    }
            /* adjoints */
            double cqb[3] = {0.0, 0.0, 0.0};
            if (S->transverse) {
                double cw = (S->transverse == 2 && S->order == 2) ? 1.0 : 0.0;
                double dl[3], dr[3];
                for (int m = 0; m < 3; ++m) {
                    dl[m] = e->amdq[m] + cw * cq[m];
                    dr[m] = e->apdq[m] - cw * cq[m];
                }
                for (int side = 0; side < 2; ++side) {
                    int k = side == 0 ? a - 1 : a;
                    const double* d = side == 0 ? dl : dr;
                    long lo = CELL(g, dir, k, l - 1), mid = CELL(g, dir, k, l), hi = CELL(g, dir, k, l + 1);
                    long e0 = CELL(g, dir, k, l), e1 = CELL(g, dir, k, l + 1);
                    double bmb[3], bpb[3], db[3] = {0.0, 0.0, 0.0};
                    for (int m = 0; m < 3; ++m) {
                        bmb[m] = -0.5 * lam * ftb[m * pl + e0];
                        bpb[m] = -0.5 * lam * ftb[m * pl + e1];
                    }
                    tsplit_adj(d, mt, S->Z[lo], S->Z[mid], S->Z[hi], S->c[lo], S->c[hi], bmb, bpb,
                               db, &A->Zb[lo], &A->Zb[mid], &A->Zb[hi], &A->cb[lo], &A->cb[hi]);
                    for (int m = 0; m < 3; ++m) {
                        if (side == 0) { eb->amdq[m] += db[m]; cqb[m] += cw * db[m]; }
                        else { eb->apdq[m] += db[m]; cqb[m] -= cw * db[m]; }
                    }
                }
            }
            if (S->order == 2) {
                long E = CELL(g, dir, a, l);
                for (int m = 0; m < 3; ++m) cqb[m] += 0.5 * fnb[m * pl + E];
                for (int w = 0; w < 2; ++w) {
                    double as = fabs(e->s[w]);
                    double kap = as * (1.0 - lam * as);
                    double wtb[3], kapb = 0.0;
                    for (int m = 0; m < 3; ++m) {
                        wtb[m] = kap * cqb[m];
                        kapb += cqb[m] * wt[w][m];
                    }
                    double asb = kapb * (1.0 - 2.0 * lam * as);
                    eb->s[w] += (e->s[w] >= 0.0 ? asb : -asb);
                    /* wt = phi * w */
                    double phib = 0.0;
                    for (int m = 0; m < 3; ++m) {
                        eb->w[w][m] += phi[w] * wtb[m];
                        phib += wtb[m] * e->w[w][m];
                    }
                    if (S->limiter != 0 && wn2[w] != 0.0) {
                        double th = dot[w] / wn2[w];
                        double thb = dphi[w] * phib;
                        double dotb = thb / wn2[w];
                        double wn2b = -thb * th / wn2[w];
                        edge_rec* upb = e->s[w] > 0.0 ? &recb[a] : &recb[a + 2];
                        for (int m = 0; m < 3; ++m) {
                            upb->w[w][m] += dotb * e->w[w][m];
                            eb->w[w][m] += dotb * up[w]->w[w][m];
                            eb->w[w][m] += 2.0 * wn2b * e->w[w][m];
                        }
                    }
                }
            }
        }
        /* reverse of the normal Riemann problems */
        for (int a = -1; a <= nn + 1; ++a) {
            edge_rec* e = &rec[a + 1];
            edge_rec* eb = &recb[a + 1];
            long L = CELL(g, dir, a - 1, l), R = CELL(g, dir, a, l);
            for (int w = 0; w < 2; ++w)
                for (int m = 0; m < 3; ++m) {
                    double fb = e->s[w] < 0.0 ? eb->amdq[m] : eb->apdq[m];
                    eb->w[w][m] += e->s[w] * fb;
                    eb->s[w] += fb * e->w[w][m];
                }
            A->cb[L] -= eb->s[0];
            A->cb[R] += eb->s[1];
            double zl = S->Z[L], zr = S->Z[R], den = zl + zr;
            double a1 = e->a[0], a2 = e->a[1];
            double a1b = -zl * eb->w[0][0] + eb->w[0][mn];
            double a2b = zr * eb->w[1][0] + eb->w[1][mn];
            double zlb = -a1 * eb->w[0][0];
            double zrb = a2 * eb->w[1][0];
            double dp = S->p[R] - S->p[L];
            double dn = qn[R] - qn[L];
            (void)dp;
            double dpb = -a1b / den + a2b / den;
            double dnb = zr * a1b / den + zl * a2b / den;
            zrb += dn * a1b / den;
            zlb += dn * a2b / den;
            double denb = -a1b * a1 / den - a2b * a2 / den;
            zlb += denb; zrb += denb;
            A->Zb[L] += zlb; A->Zb[R] += zrb;
            A->pb[R] += dpb; A->pb[L] -= dpb;
            qnb[R] += dnb; qnb[L] -= dnb;
        }
    }
}

int orc_step_adjoint(int nx, int ny, int mbc, double dx, double dy, double dt,
                     int order, int transverse, int limiter,
                     const double* q, const double* rho, const double* K,
                     const double* lam_new, double* lam_q, double* g_rho, double* g_K)
{
    if (nx < 1 || ny < 1 || mbc < 2 || !(dx > 0) || !(dy > 0)) return -1;
    geom G = {nx, ny, mbc, nx + 2 * mbc, ny + 2 * mbc};
    const geom* g = &G;
    long pl = (long)G.W * G.H;
    int nmax = (nx > ny ? nx : ny) + 3;
    double *c, *Z, *cb, *Zb, *amxb, *apxb, *amyb, *apyb, *Fb, *Gb;
    edge_rec* rec = (edge_rec*)calloc((size_t)nmax, sizeof(edge_rec));
    edge_rec* recb = (edge_rec*)calloc((size_t)nmax, sizeof(edge_rec));
    if (!rec || !recb || alloc_zero(&c, pl) || alloc_zero(&Z, pl) || alloc_zero(&cb, pl) ||
        alloc_zero(&Zb, pl) || alloc_zero(&amxb, 3 * pl) || alloc_zero(&apxb, 3 * pl) ||
        alloc_zero(&amyb, 3 * pl) || alloc_zero(&apyb, 3 * pl) || alloc_zero(&Fb, 3 * pl) ||
        alloc_zero(&Gb, 3 * pl))
        return -1;
    cell_speeds(g, rho, K, c, Z);
    step_ctx S = {g, order, transverse, limiter, q, q + pl, q + 2 * pl, c, Z};
    /* reverse of the update */
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            long k = IC(g, i, j), kx = IC(g, i + 1, j), ky = IC(g, i, j + 1);
            for (int m = 0; m < 3; ++m) {
                long o = m * pl;
                double lb = lam_new[o + k];
                lam_q[o + k] += lb;
                apxb[o + k] -= dt / dx * lb;
                amxb[o + kx] -= dt / dx * lb;
                apyb[o + k] -= dt / dy * lb;
                amyb[o + ky] -= dt / dy * lb;
                Fb[o + kx] -= dt / dx * lb;
                Fb[o + k] += dt / dx * lb;
                Gb[o + ky] -= dt / dy * lb;
                Gb[o + k] += dt / dy * lb;
            }
        }
    adj_out A = {lam_q, lam_q + pl, lam_q + 2 * pl, cb, Zb};
    sweep_adj(&S, 1, dt / dy, rec, recb, amyb, apyb, Gb, Fb, &A);
    sweep_adj(&S, 0, dt / dx, rec, recb, amxb, apxb, Fb, Gb, &A);
    /* c = sqrt(K/rho), Z = sqrt(K rho) */
    for (long k = 0; k < pl; ++k) {
        g_K[k] += cb[k] * c[k] / (2.0 * K[k]) + Zb[k] * Z[k] / (2.0 * K[k]);
        g_rho[k] += -cb[k] * c[k] / (2.0 * rho[k]) + Zb[k] * Z[k] / (2.0 * rho[k]);
    }
    free(rec); free(recb); free(c); free(Z); free(cb); free(Zb);
    free(amxb); free(apxb); free(amyb); free(apyb); free(Fb); free(Gb);
    return 0;
}

/* ------------------------------------------------------- physical boundaries */

/* boundary map of index k on [0, n): returns the source index and whether a wall flips */
static int bc_map(int k, int n, int bclo, int bchi, int* flip)
{
    *flip = 0;
    if (k < 0) {
        if (bclo == 1) return ((k % n) + n) % n;
        if (bclo == 2) { *flip = 1; return -1 - k; }
        return 0;
    }
    if (k >= n) {
        if (bchi == 1) return k % n;
        if (bchi == 2) { *flip = 1; return 2 * n - 1 - k; }
        return n - 1;
    }
    return k;
}

int orc_fill_bc(int nx, int ny, int mbc, int ncomp, const int* bc, double* a)
{
    geom G = {nx, ny, mbc, nx + 2 * mbc, ny + 2 * mbc};
    long pl = (long)G.W * G.H;
    /* x sides on the interior rows, then y sides over all columns (corners included) */
    for (int j = 0; j < ny; ++j)
        for (int i = -mbc; i < nx + mbc; ++i) {
            if (i >= 0 && i < nx) continue;
            int fl;
            int si = bc_map(i, nx, bc[0], bc[1], &fl);
            for (int m = 0; m < ncomp; ++m) {
                double s = (fl && ncomp == 3 && m == 1) ? -1.0 : 1.0;
                a[m * pl + IC(&G, i, j)] = s * a[m * pl + IC(&G, si, j)];
            }
        }
    for (int j = -mbc; j < ny + mbc; ++j) {
        if (j >= 0 && j < ny) continue;
        int fl;
        int sj = bc_map(j, ny, bc[2], bc[3], &fl);
        for (int i = -mbc; i < nx + mbc; ++i)
            for (int m = 0; m < ncomp; ++m) {
                double s = (fl && ncomp == 3 && m == 2) ? -1.0 : 1.0;
                a[m * pl + IC(&G, i, j)] = s * a[m * pl + IC(&G, i, sj)];
            }
    }
    return 0;
}

int orc_fill_bc_adjoint(int nx, int ny, int mbc, int ncomp, const int* bc, double* gr)
{
    geom G = {nx, ny, mbc, nx + 2 * mbc, ny + 2 * mbc};
    long pl = (long)G.W * G.H;
    /* reverse order of orc_fill_bc: y sides first (they may read x-side ghosts) */
    for (int j = ny + mbc - 1; j >= -mbc; --j) {
        if (j >= 0 && j < ny) continue;
        int fl;
        int sj = bc_map(j, ny, bc[2], bc[3], &fl);
        for (int i = -mbc; i < nx + mbc; ++i)
            for (int m = 0; m < ncomp; ++m) {
                double s = (fl && ncomp == 3 && m == 2) ? -1.0 : 1.0;
                long d = m * pl + IC(&G, i, j);
                gr[m * pl + IC(&G, i, sj)] += s * gr[d];
                gr[d] = 0.0;
            }
    }
    for (int j = ny - 1; j >= 0; --j)
        for (int i = nx + mbc - 1; i >= -mbc; --i) {
            if (i >= 0 && i < nx) continue;
            int fl;
            int si = bc_map(i, nx, bc[0], bc[1], &fl);
            for (int m = 0; m < ncomp; ++m) {
                double s = (fl && ncomp == 3 && m == 1) ? -1.0 : 1.0;
                long d = m * pl + IC(&G, i, j);
                gr[m * pl + IC(&G, si, j)] += s * gr[d];
                gr[d] = 0.0;
            }
        }
    return 0;
}

double orc_cfl_max(int nx, int ny, int mbc, const double* rho, const double* K)
{
    geom G = {nx, ny, mbc, nx + 2 * mbc, ny + 2 * mbc};
    double sm = 0.0;
    for (int j = -1; j <= ny; ++j)
        for (int i = -1; i <= nx; ++i) {
            long k = IC(&G, i, j);
            double c = sqrt(K[k] / rho[k]);
            if (c > sm) sm = c;
        }
    return sm;
}

/* ------------------------------------------------------------------- AMR */

static inline long box_plane(const orc_box* b, int mbc) { return (long)(b->nx + 2 * mbc) * (b->ny + 2 * mbc); }
static inline long box_cell(const orc_box* b, int mbc, int gi, int gj)
{   /* gi, gj: level index of a cell inside the box's padded region */
    return b->off + (long)(gi - b->ilo + mbc) + (long)(gj - b->jlo + mbc) * (b->nx + 2 * mbc);
}
static inline int box_has(const orc_box* b, int gi, int gj)
{
    return gi >= b->ilo && gi < b->ilo + b->nx && gj >= b->jlo && gj < b->jlo + b->ny;
}
static int find_box(int nb, const orc_box* bx, int gi, int gj)
{
    for (int n = 0; n < nb; ++n)
        if (box_has(&bx[n], gi, gj)) return n;
    return -1;
}

/* coarse value at coarse cell (I, J) at time fraction tau, through the coarse domain's
 * physical-boundary map; returns -2 if no coarse box covers the mapped cell */
static int coarse_value(int ncb, const orc_box* cb, const double* cold, const double* cnew, double tau,
                        int ncomp, int mbc, int cNX, int cNY, const int* bc, int I, int J, double* out)
{
    int fx, fy;
    int si = bc_map(I, cNX, bc[0], bc[1], &fx);
    int sj = bc_map(J, cNY, bc[2], bc[3], &fy);
    int n = find_box(ncb, cb, si, sj);
    if (n < 0) return -2;
    long k = box_cell(&cb[n], mbc, si, sj), pl = box_plane(&cb[n], mbc);
    for (int m = 0; m < ncomp; ++m) {
        double s = 1.0;
        if (ncomp == 3 && ((m == 1 && fx) || (m == 2 && fy))) s = -1.0;
        out[m] = s * ((1.0 - tau) * cold[m * pl + k] + tau * cnew[m * pl + k]);
    }
    return 0;
}

static double minmod(double a, double b)
{
    if (a * b <= 0.0) return 0.0;
    return fabs(a) < fabs(b) ? a : b;
}

static int floordiv(int a, int r) { return a >= 0 ? a / r : -((-a + r - 1) / r); }

int orc_interp_cell(int ncb, const orc_box* cb, const double* cold, const double* cnew,
                    double tau, int r, int ncomp, int mbc, int cNX, int cNY, const int* bc,
                    int fi, int fj, double* out)
{
    int I = floordiv(fi, r), J = floordiv(fj, r);
    double q0[8], qw[8], qe[8], qs[8], qn[8];
    if (coarse_value(ncb, cb, cold, cnew, tau, ncomp, mbc, cNX, cNY, bc, I, J, q0) ||
        coarse_value(ncb, cb, cold, cnew, tau, ncomp, mbc, cNX, cNY, bc, I - 1, J, qw) ||
        coarse_value(ncb, cb, cold, cnew, tau, ncomp, mbc, cNX, cNY, bc, I + 1, J, qe) ||
        coarse_value(ncb, cb, cold, cnew, tau, ncomp, mbc, cNX, cNY, bc, I, J - 1, qs) ||
        coarse_value(ncb, cb, cold, cnew, tau, ncomp, mbc, cNX, cNY, bc, I, J + 1, qn))
        return -2;
    /* offsets of the fine cell centre from the coarse centre, in coarse cells */
    double xi = ((double)(fi - I * r) + 0.5) / r - 0.5;
    double eta = ((double)(fj - J * r) + 0.5) / r - 0.5;
    for (int m = 0; m < ncomp; ++m) {
        double sx = minmod(qe[m] - q0[m], q0[m] - qw[m]);
        double sy = minmod(qn[m] - q0[m], q0[m] - qs[m]);
        out[m] = q0[m] + xi * sx + eta * sy;
    }
    return 0;
}

int orc_level_fill_ghost(int nb, const orc_box* boxes, double* pool, int ncomp, int mbc,
                         int NX, int NY, const int* bc,
                         int ncb, const orc_box* cboxes, const double* cold, const double* cnew,
                         double tau, int r, int copy_only)
{
    int cNX = r > 0 ? NX / r : 0, cNY = r > 0 ? NY / r : 0;
    for (int n = 0; n < nb; ++n) {
        const orc_box* b = &boxes[n];
        long pl = box_plane(b, mbc);
        for (int gj = b->jlo - mbc; gj < b->jlo + b->ny + mbc; ++gj)
            for (int gi = b->ilo - mbc; gi < b->ilo + b->nx + mbc; ++gi) {
                if (box_has(b, gi, gj)) continue;
                int fx, fy;
                int si = bc_map(gi, NX, bc[0], bc[1], &fx);
                int sj = bc_map(gj, NY, bc[2], bc[3], &fy);
                double val[8];
                int src = box_has(b, si, sj) ? n : find_box(nb, boxes, si, sj);
                if (src >= 0) {
                    long k = box_cell(&boxes[src], mbc, si, sj), spl = box_plane(&boxes[src], mbc);
                    for (int m = 0; m < ncomp; ++m) val[m] = pool[m * spl + k];
                } else {
                    if (copy_only) continue;
                    if (ncb <= 0 || r <= 0) return -2;
                    if (orc_interp_cell(ncb, cboxes, cold, cnew, tau, r, ncomp, mbc, cNX, cNY, bc,
                                        si, sj, val))
                        return -2;
                }
                long d = box_cell(b, mbc, gi, gj);
                for (int m = 0; m < ncomp; ++m) {
                    double s = 1.0;
                    if (ncomp == 3 && ((m == 1 && fx) || (m == 2 && fy))) s = -1.0;
                    pool[m * pl + d] = s * val[m];
                }
            }
    }
    return 0;
}

int orc_average_down(int nf, const orc_box* fb, const double* fpool,
                     int nc, const orc_box* cb, double* cpool, int ncomp, int mbc, int r)
{
    for (int c = 0; c < nc; ++c) {
        const orc_box* C = &cb[c];
        long cpl = box_plane(C, mbc);
        for (int J = C->jlo; J < C->jlo + C->ny; ++J)
            for (int I = C->ilo; I < C->ilo + C->nx; ++I) {
                int f = find_box(nf, fb, I * r, J * r);
                if (f < 0) continue;
                const orc_box* F = &fb[f];
                long fpl = box_plane(F, mbc);
                for (int m = 0; m < ncomp; ++m) {
                    double s = 0.0;
                    for (int b = 0; b < r; ++b)
                        for (int a = 0; a < r; ++a)
                            s += fpool[m * fpl + box_cell(F, mbc, I * r + a, J * r + b)];
                    cpool[m * cpl + box_cell(C, mbc, I, J)] = s / (double)(r * r);
                }
            }
    }
    return 0;
}

int orc_average_down_adjoint(int nf, const orc_box* fb, double* gf,
                             int nc, const orc_box* cb, double* gc, int ncomp, int mbc, int r)
{
    for (int c = 0; c < nc; ++c) {
        const orc_box* C = &cb[c];
        long cpl = box_plane(C, mbc);
        for (int J = C->jlo; J < C->jlo + C->ny; ++J)
            for (int I = C->ilo; I < C->ilo + C->nx; ++I) {
                int f = find_box(nf, fb, I * r, J * r);
                if (f < 0) continue;
                const orc_box* F = &fb[f];
                long fpl = box_plane(F, mbc);
                for (int m = 0; m < ncomp; ++m) {
                    long kc = m * cpl + box_cell(C, mbc, I, J);
                    double g = gc[kc] / (double)(r * r);
                    gc[kc] = 0.0;
                    for (int b = 0; b < r; ++b)
                        for (int a = 0; a < r; ++a)
                            gf[m * fpl + box_cell(F, mbc, I * r + a, J * r + b)] += g;
                }
            }
    }
    return 0;
}

/* adjoint of coarse_value: spread gbar (ncomp) to the mapped coarse cell of the pools */
static int coarse_value_adj(int ncb, const orc_box* cb, double* gold, double* gnew, double tau,
                            int ncomp, int mbc, int cNX, int cNY, const int* bc, int I, int J,
                            const double* gbar)
{
    int fx, fy;
    int si = bc_map(I, cNX, bc[0], bc[1], &fx);
    int sj = bc_map(J, cNY, bc[2], bc[3], &fy);
    int n = find_box(ncb, cb, si, sj);
    if (n < 0) return -2;
    long k = box_cell(&cb[n], mbc, si, sj), pl = box_plane(&cb[n], mbc);
    for (int m = 0; m < ncomp; ++m) {
        double s = 1.0;
        if (ncomp == 3 && ((m == 1 && fx) || (m == 2 && fy))) s = -1.0;
        gold[m * pl + k] += (1.0 - tau) * s * gbar[m];
        gnew[m * pl + k] += tau * s * gbar[m];
    }
    return 0;
}

static int interp_cell_adj(int ncb, const orc_box* cb, const double* cold, const double* cnew,
                           double* gold, double* gnew, double tau, int r, int ncomp, int mbc,
                           int cNX, int cNY, const int* bc, int fi, int fj, const double* gout)
{
    int I = floordiv(fi, r), J = floordiv(fj, r);
    double q0[8], qw[8], qe[8], qs[8], qn[8];
    if (coarse_value(ncb, cb, cold, cnew, tau, ncomp, mbc, cNX, cNY, bc, I, J, q0) ||
        coarse_value(ncb, cb, cold, cnew, tau, ncomp, mbc, cNX, cNY, bc, I - 1, J, qw) ||
        coarse_value(ncb, cb, cold, cnew, tau, ncomp, mbc, cNX, cNY, bc, I + 1, J, qe) ||
        coarse_value(ncb, cb, cold, cnew, tau, ncomp, mbc, cNX, cNY, bc, I, J - 1, qs) ||
        coarse_value(ncb, cb, cold, cnew, tau, ncomp, mbc, cNX, cNY, bc, I, J + 1, qn))
        return -2;
    double xi = ((double)(fi - I * r) + 0.5) / r - 0.5;
    double eta = ((double)(fj - J * r) + 0.5) / r - 0.5;
    double g0[8], gw[8], ge[8], gs[8], gn[8];
    for (int m = 0; m < ncomp; ++m) {
        g0[m] = gout[m]; gw[m] = ge[m] = gs[m] = gn[m] = 0.0;
        /* sx = minmod(a, b), a = qe - q0, b = q0 - qw: derivative along the chosen branch */
        double a = qe[m] - q0[m], b = q0[m] - qw[m];
        double sxb = xi * gout[m];
        if (a * b > 0.0) {
            if (fabs(a) < fabs(b)) { ge[m] += sxb; g0[m] -= sxb; }
            else { g0[m] += sxb; gw[m] -= sxb; }
        }
        a = qn[m] - q0[m]; b = q0[m] - qs[m];
        double syb = eta * gout[m];
        if (a * b > 0.0) {
            if (fabs(a) < fabs(b)) { gn[m] += syb; g0[m] -= syb; }
            else { g0[m] += syb; gs[m] -= syb; }
        }
    }
    coarse_value_adj(ncb, cb, gold, gnew, tau, ncomp, mbc, cNX, cNY, bc, I, J, g0);
    coarse_value_adj(ncb, cb, gold, gnew, tau, ncomp, mbc, cNX, cNY, bc, I - 1, J, gw);
    coarse_value_adj(ncb, cb, gold, gnew, tau, ncomp, mbc, cNX, cNY, bc, I + 1, J, ge);
    coarse_value_adj(ncb, cb, gold, gnew, tau, ncomp, mbc, cNX, cNY, bc, I, J - 1, gs);
    coarse_value_adj(ncb, cb, gold, gnew, tau, ncomp, mbc, cNX, cNY, bc, I, J + 1, gn);
    return 0;
}

int orc_level_fill_ghost_adjoint(int nb, const orc_box* boxes, double* gpool, int ncomp, int mbc,
                                 int NX, int NY, const int* bc,
                                 int ncb, const orc_box* cboxes, double* gcold, double* gcnew,
                                 const double* cold, const double* cnew, double tau, int r,
                                 int copy_only)
{
    /* every ghost value of the forward fill is a function of interior cells only (its own
     * box, another box, or the coarse level), so the reverse is order independent */
    int cNX = r > 0 ? NX / r : 0, cNY = r > 0 ? NY / r : 0;
    for (int n = nb - 1; n >= 0; --n) {
        const orc_box* b = &boxes[n];
        long pl = box_plane(b, mbc);
        for (int gj = b->jlo + b->ny + mbc - 1; gj >= b->jlo - mbc; --gj)
            for (int gi = b->ilo + b->nx + mbc - 1; gi >= b->ilo - mbc; --gi) {
                if (box_has(b, gi, gj)) continue;
                int fx, fy;
                int si = bc_map(gi, NX, bc[0], bc[1], &fx);
                int sj = bc_map(gj, NY, bc[2], bc[3], &fy);
                long d = box_cell(b, mbc, gi, gj);
                int src = box_has(b, si, sj) ? n : find_box(nb, boxes, si, sj);
                if (src < 0 && copy_only) continue;
                double gval[8];
                for (int m = 0; m < ncomp; ++m) {
                    double s = 1.0;
                    if (ncomp == 3 && ((m == 1 && fx) || (m == 2 && fy))) s = -1.0;
                    gval[m] = s * gpool[m * pl + d];
                    gpool[m * pl + d] = 0.0;
                }
                if (src >= 0) {
                    long k = box_cell(&boxes[src], mbc, si, sj), spl = box_plane(&boxes[src], mbc);
                    for (int m = 0; m < ncomp; ++m) gpool[m * spl + k] += gval[m];
                } else {
                    if (ncb <= 0 || r <= 0) return -2;
                    if (interp_cell_adj(ncb, cboxes, cold, cnew, gcold, gcnew, tau, r, ncomp, mbc,
                                        cNX, cNY, bc, si, sj, gval))
                        return -2;
                }
            }
    }
    return 0;
}

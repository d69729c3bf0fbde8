// claw_reflux.cu -- the conservation fix of Sec. 2.3 ("refluxing") for a uniform medium, where
// the acoustics system is in conservation form: f(Q) = A Q, g(Q) = B Q, and for the shallow water
// equations, whose Roe solver is conservative (A-dQ + A+dQ = f(Q_R) - f(Q_L)): there A (Q_F - Q_C)
// below becomes f(Q_F) - f(Q_C) with the equations' own flux.
//
// A coarse cell C next to the fine region (not covered by it) is updated by the coarse step with
// the flux F_e through its edge e; the fine cells along e see r fine fluxes per substep.  After
// the fine substeps and the average, C is corrected so that the flux through e is the average
// of the fine ones.  With C left of e and fine cells F_b right of their edges e_b:
//   F_e   - f(Q_C^n) = A-dQ_e + F~_e                                  (coarse part)
//   F_b^k - f(Q_C^n) = A (Q_F^k - Q_C^n) - A+dQ_b^k + F~_b^k            (fine part, substep k)
//   Q_C^{n+1} += -(dt/dx) [ (1/r^2) sum_{k,b} (F_b^k - f(Q_C^n)) - (F_e - f(Q_C^n)) ]
// (the paper's C1 + C2 + C3), mirrored for C right of e (+A-dQ_b, -A+dQ_e, opposite sign) and
// in y.  F~ is the correction flux plus the transverse terms the other direction's sweep puts
// on the edge.  Each edge's quantities are evaluated here from the state the step read, with the
// step's own formulation (wave strengths scaled by 2, the same limiter functions), so the fix
// matches the fused kernel's update to rounding.
#include <cuda_runtime.h>

#include "claw_step.cuh"

namespace claw {
namespace {

struct UMed {
    double c, Z, iZ, K, irho;
};

// A-dQ, A+dQ and F~ of the edge between normal indices e-1 and e on line t of a box (local
// interior coordinates; dir 0: x-edge, normal index i, line j; dir 1: y-edge), components in
// the edge's order (p, normal velocity, transverse velocity).
template <int LIM>
__device__ void edge_terms(const double* q, int W, long long WH, int dir, int e, int t, const UMed& md, double ln,
                           double lt, int order, int transverse, double am[3], double ap[3], double f[3])
{
    const int mn = dir == 0 ? 1 : 2, mt = dir == 0 ? 2 : 1;
    auto Q = [&](int m, int n, int l) -> double {
        const int i = dir == 0 ? n : l, j = dir == 0 ? l : n;
        return q[m * WH + (long long)(j + 2) * W + (i + 2)];
    };
    // normal strengths (x2) of the edge between n-1 and n on line l
    auto strengths = [&](int n, int l, double& a1, double& a2) {
        const double dp = Q(0, n, l) - Q(0, n - 1, l), du = Q(mn, n, l) - Q(mn, n - 1, l);
        a1 = fma(-dp, md.iZ, du);
        a2 = fma(dp, md.iZ, du);
    };
    // transverse strengths (x2) of the edge between lines l-1 and l on normal index n
    auto tstrengths = [&](int n, int l, double& b1, double& b2) {
        const double dp = Q(0, n, l) - Q(0, n, l - 1), dv = Q(mt, n, l) - Q(mt, n, l - 1);
        b1 = fma(-dp, md.iZ, dv);
        b2 = fma(dp, md.iZ, dv);
    };
    const double c = md.c, Z = md.Z;
    double a1, a2;
    strengths(e, t, a1, a2);
    am[0] = 0.5 * c * Z * a1;
    am[1] = -0.5 * c * a1;
    am[2] = 0.0;
    ap[0] = 0.5 * c * Z * a2;
    ap[1] = 0.5 * c * a2;
    ap[2] = 0.0;
    f[0] = f[1] = f[2] = 0.0;
    const bool second = order == 2;
    if (second) {   // normal correction flux: (1/2) sum |s| (1 - ln |s|) W~
        double b1, b2, c1, c2;
        strengths(e + 1, t, b1, b2);
        strengths(e - 1, t, c1, c2);
        const double m1 = Lim<LIM>::f(a1, b1), m2 = Lim<LIM>::f(a2, c2);
        const double kap = c * (1.0 - ln * c);
        f[0] += 0.25 * kap * Z * (m2 - m1);
        f[1] += 0.25 * kap * (m1 + m2);
    }
    if (transverse) {
        const bool cw = transverse == 2 && second;
        // pressure of the transverse fluctuations into cell (n, t): the up-going part of the
        // transverse edge t (with -C) and the down-going part of edge t+1 (with +C)
        auto P = [&](int n) -> double {
            double lo1, lo2, hi1, hi2;
            tstrengths(n, t, lo1, lo2);
            tstrengths(n, t + 1, hi1, hi2);
            double r = 0.5 * c * Z * (lo2 + hi1);
            if (cw) {
                double p1, p2, q1, q2;
                tstrengths(n, t - 1, p1, p2);
                tstrengths(n, t + 2, q1, q2);
                const double s_lo = Lim<LIM>::f(lo2, p2) - Lim<LIM>::f(lo1, hi1);
                const double s_hi = Lim<LIM>::f(hi2, lo2) - Lim<LIM>::f(hi1, q1);
                r += 0.5 * c * (1.0 - lt * c) * Z * (s_hi - s_lo);
            }
            return r;
        };
        const double PL = P(e - 1), PR = P(e);
        f[0] -= 0.25 * lt * c * (PL - PR);
        f[1] -= 0.25 * lt * c * md.iZ * (PL + PR);
    }
}

// ------------------------------------------------------------------ shallow water
// Roe state and wave strengths of one edge (the step kernel's formulation: per-cell sqrt(h) and
// momenta over sqrt(h), one reciprocal, one reciprocal square root for c and 1/(2c))
struct SEdge {
    double un, ut, c, i2c, a1, a2, a3;
};

__device__ __forceinline__ SEdge swe_solve(double hl, double nl, double tl, double hr, double nr, double tr, double hg)
{
    const double rl = rsqrt(hl), rr = rsqrt(hr);
    const double inv = 1.0 / (hl * rl + hr * rr);
    SEdge E;
    E.un = (nl * rl + nr * rr) * inv;
    E.ut = (tl * rl + tr * rr) * inv;
    const double x = (hl + hr) * hg;
    const double rc = rsqrt(x);
    E.c = x * rc;
    E.i2c = 0.5 * rc;
    const double dh = hr - hl, dn = nr - nl, dt = tr - tl;
    E.a1 = fma(E.un + E.c, dh, -dn) * E.i2c;
    E.a2 = fma(-E.ut, dh, dt);
    E.a3 = fma(-(E.un - E.c), dh, dn) * E.i2c;
    return E;
}

// h_p = |s_p| (1 - l |s_p|) mu_p / 2 of an edge from itself and its two neighbours along the sweep
template <int LIM>
__device__ __forceinline__ void swe_limited(const SEdge& E, const SEdge& Eb, const SEdge& Ef, double l, double h[3])
{
    const double s1 = E.un - E.c, s3 = E.un + E.c;
    const SEdge& U1 = s1 > 0.0 ? Eb : Ef;
    const SEdge& U2 = E.un > 0.0 ? Eb : Ef;
    const SEdge& U3 = s3 > 0.0 ? Eb : Ef;
    const double w = fma(E.ut, E.ut, 1.0);
    const double rr1 = fma(s1, s1, w), rr3 = fma(s3, s3, w);
    const double ip = 1.0 / (rr1 * rr3);
    const double ri1 = fma(U1.un - U1.c, s1, fma(U1.ut, E.ut, 1.0));
    const double ri3 = fma(U3.un + U3.c, s3, fma(U3.ut, E.ut, 1.0));
    const double mu1 = Lim<LIM>::f(E.a1, U1.a1 * ri1 * (rr3 * ip));
    const double mu2 = Lim<LIM>::f(E.a2, U2.a2);
    const double mu3 = Lim<LIM>::f(E.a3, U3.a3 * ri3 * (rr1 * ip));
    const double k1 = fabs(s1), k2 = fabs(E.un), k3 = fabs(s3), hl = -0.5 * l;
    h[0] = fma(hl * k1, k1, 0.5 * k1) * mu1;
    h[1] = fma(hl * k2, k2, 0.5 * k2) * mu2;
    h[2] = fma(hl * k3, k3, 0.5 * k3) * mu3;
}

// the fluctuation an edge sends into the cell on its right (right) or left, with the correction
// at the weight the transverse mode gives (hw = +1: full C, -1: none), split across the sweep:
// adds the part going to lower transverse indices to bm and the rest to bp, (h, n, t) order
__device__ __forceinline__ void swe_side_split(const SEdge& E, const double h[3], bool right, double hw,
                                               double bm[3], double bp[3])
{
    const double s[3] = {E.un - E.c, E.un, E.un + E.c};
    const double a[3] = {E.a1, E.a2, E.a3};
    double d[3];
    for (int p = 0; p < 3; ++p) {
        const double hp = right ? -h[p] : h[p];
        const double lam = right ? (s[p] > 0.0 ? s[p] : 0.0) : (s[p] < 0.0 ? s[p] : 0.0);
        d[p] = fma(hw, hp, fma(lam, a[p], hp));
    }
    const double dh = d[0] + d[2], t = d[1] * E.i2c;
    const double b[3] = {fma(0.5, dh, -t), E.c * (d[2] - d[0]), fma(0.5, dh, t)};
    const double m[3] = {E.ut - E.c, E.ut, E.ut + E.c};
    double gm[3], gp[3];
    for (int q = 0; q < 3; ++q) {
        const double g = m[q] * b[q];
        gm[q] = m[q] < 0.0 ? g : 0.0;
        gp[q] = m[q] < 0.0 ? 0.0 : g;
    }
    const double Gm = gm[0] + gm[2], Gp = gp[0] + gp[2];
    bm[0] += Gm;
    bm[1] += fma(E.un, Gm, gm[1]);
    bm[2] += fma(E.ut, Gm, E.c * (gm[2] - gm[0]));
    bp[0] += Gp;
    bp[1] += fma(E.un, Gp, gp[1]);
    bp[2] += fma(E.ut, Gp, E.c * (gp[2] - gp[0]));
}

// A-dQ, A+dQ and F~ (correction plus the other sweep's transverse terms) of the edge between
// normal indices e-1 and e on line t, components (h, normal momentum, transverse momentum)
template <int LIM>
__device__ void swe_edge_terms(const double* q, int W, long long WH, int dir, int e, int t, double hg, double ln,
                               double lt, int order, int transverse, double am[3], double ap[3], double f[3])
{
    const int mn = dir == 0 ? 1 : 2, mt = dir == 0 ? 2 : 1;
    auto Q = [&](int m, int n, int l) -> double {
        const int i = dir == 0 ? n : l, j = dir == 0 ? l : n;
        return q[m * WH + (long long)(j + 2) * W + (i + 2)];
    };
    // along the normal: edge between (n-1, l) and (n, l); across: between (n, l-1) and (n, l)
    auto solve = [&](bool along, int n, int l) -> SEdge {
        const int nm = along ? mn : mt, tm = along ? mt : mn;
        const int n0 = along ? n - 1 : n, l0 = along ? l : l - 1;
        return swe_solve(Q(0, n0, l0), Q(nm, n0, l0), Q(tm, n0, l0), Q(0, n, l), Q(nm, n, l), Q(tm, n, l), hg);
    };
    const bool second = order == 2;
    const double hw = (transverse == 2 && second) ? 1.0 : -1.0;
    const SEdge E = solve(true, e, t);
    const double s[3] = {E.un - E.c, E.un, E.un + E.c};
    const double a[3] = {E.a1, E.a2, E.a3};
    double cm[3] = {0.0, 0.0, 0.0}, cp[3] = {0.0, 0.0, 0.0};   // coefficients on r_p
    for (int p = 0; p < 3; ++p) {
        if (s[p] < 0.0) cm[p] = s[p] * a[p];
        else cp[p] = s[p] * a[p];
    }
    auto vec = [&](const double c3[3], double out[3]) {   // sum_p c_p r_p, r = (1, un -/+ c, ut), (0, 0, 1)
        out[0] = c3[0] + c3[2];
        out[1] = fma(s[0], c3[0], s[2] * c3[2]);
        out[2] = fma(E.ut, c3[0] + c3[2], c3[1]);
    };
    vec(cm, am);
    vec(cp, ap);
    f[0] = f[1] = f[2] = 0.0;
    if (second) {
        double h[3];
        swe_limited<LIM>(E, solve(true, e - 1, t), solve(true, e + 1, t), ln, h);
        vec(h, f);
    }
    if (transverse) {
        // the transverse sweep's fluctuations entering cell (k, t), split along the normal
        auto parts = [&](int k, double bm[3], double bp[3]) {
            const SEdge lo = solve(false, k, t), hi = solve(false, k, t + 1);
            double hlo[3] = {0.0, 0.0, 0.0}, hhi[3] = {0.0, 0.0, 0.0};
            if (second) {
                swe_limited<LIM>(lo, solve(false, k, t - 1), hi, lt, hlo);
                swe_limited<LIM>(hi, lo, solve(false, k, t + 2), lt, hhi);
            }
            swe_side_split(lo, hlo, true, hw, bm, bp);
            swe_side_split(hi, hhi, false, hw, bm, bp);
        };
        double m0[3] = {0.0, 0.0, 0.0}, p0[3] = {0.0, 0.0, 0.0}, m1[3] = {0.0, 0.0, 0.0}, p1[3] = {0.0, 0.0, 0.0};
        parts(e - 1, m0, p0);   // its part going to higher normal indices crosses the edge
        parts(e, m1, p1);       // its part going to lower normal indices crosses the edge
        // the transverse sweep's (h, its normal = our t, its tangential = our n)
        f[0] -= 0.5 * lt * (p0[0] + m1[0]);
        f[1] -= 0.5 * lt * (p0[2] + m1[2]);
        f[2] -= 0.5 * lt * (p0[1] + m1[1]);
    }
}

// f(Q_F) - f(Q_C) of the shallow water equations along the edge's normal, (h, n, t) order
__device__ __forceinline__ void swe_flux_diff(const double qf[3], const double qc[3], int mn, double grav, double o[3])
{
    const int mt = 3 - mn;
    auto flux = [&](const double* v, double* fl) {
        const double ih = 1.0 / v[0];
        fl[0] = v[mn];
        fl[1] = fma(v[mn] * v[mn], ih, 0.5 * grav * v[0] * v[0]);
        fl[2] = v[mn] * v[mt] * ih;
    };
    double a[3], b[3];
    flux(qf, a);
    flux(qc, b);
    for (int m = 0; m < 3; ++m) o[m] = a[m] - b[m];
}

__device__ __forceinline__ UMed umed(const StepArgs& k)
{
    UMed m;
    m.Z = sqrt(k.K0 * k.rho0);
    m.c = sqrt(k.K0 / k.rho0);
    m.iZ = 1.0 / m.Z;
    m.K = k.K0;
    m.irho = 1.0 / k.rho0;
    return m;
}

// edge-local (p, normal, transverse) -> (p, u, v)
__device__ __forceinline__ void to_puv(int dir, const double in[3], double out[3])
{
    out[0] = in[0];
    out[1] = dir == 0 ? in[1] : in[2];
    out[2] = dir == 0 ? in[2] : in[1];
}

template <int LIM>
__global__ void reflux_coarse_kernel(const RefluxRec* __restrict__ recs, int n, const PatchDev* __restrict__ cp,
                                     const double* __restrict__ qc, const double* __restrict__ dt,
                                     double* __restrict__ buf, int ratio, const StepArgs k)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const RefluxRec R = recs[r];
    const PatchDev P = cp[R.cbox];
    const int W = P.nx + 4;
    const long long WH = (long long)W * (P.ny + 4);
    const double d = __ldg(dt + P.run) * P.dtscale;
    const double lx = d * P.dxinv, ly = d * P.dyinv;
    const int cn = R.dir == 0 ? R.ci : R.cj, cl = R.dir == 0 ? R.cj : R.ci;
    const int e = R.side > 0 ? cn + 1 : cn;   // C's east / north edge, or its west / south edge
    double am[3], ap[3], f[3], t[3], o[3];
    if (k.swe)
        swe_edge_terms<LIM>(qc + P.qoff, W, WH, R.dir, e, cl, 0.5 * k.grav, R.dir == 0 ? lx : ly,
                            R.dir == 0 ? ly : lx, k.order, k.transverse, am, ap, f);
    else
        edge_terms<LIM>(qc + P.qoff, W, WH, R.dir, e, cl, umed(k), R.dir == 0 ? lx : ly, R.dir == 0 ? ly : lx,
                        k.order, k.transverse, am, ap, f);
    for (int m = 0; m < 3; ++m) t[m] = (R.side > 0 ? am[m] : -ap[m]) + f[m];
    to_puv(R.dir, t, o);
    for (int m = 0; m < 3; ++m) buf[3 * r + m] = -o[m];
    for (int b = 0; b < ratio; ++b)
        for (int m = 0; m < 3; ++m) buf[3 * (n + r * ratio + b) + m] = 0.0;
}

// one thread per (record, fine edge b): slot (r, b) of the fine part accumulates over substeps
// (buf holds the coarse parts first, 3 per record, then the fine slots, 3 per record and edge)
template <int LIM>
__global__ void reflux_fine_kernel(const RefluxRec* __restrict__ recs, int n, const PatchDev* __restrict__ cp,
                                   const PatchDev* __restrict__ fp, const double* __restrict__ qf,
                                   const double* __restrict__ qc, const double* __restrict__ dt,
                                   double* __restrict__ buf, int ratio, const StepArgs k)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * ratio) return;
    const int r = t / ratio, b = t - r * ratio;
    const RefluxRec R = recs[r];
    const PatchDev C = cp[R.cbox], F = fp[R.fbox];
    const int Wc = C.nx + 4, Wf = F.nx + 4;
    const long long WHc = (long long)Wc * (C.ny + 4), WHf = (long long)Wf * (F.ny + 4);
    const double d = __ldg(dt + F.run) * F.dtscale;
    const double lx = d * F.dxinv, ly = d * F.dyinv;
    const long long co = C.qoff + (long long)(R.cj + 2) * Wc + (R.ci + 2);
    double qC[3];
    for (int m = 0; m < 3; ++m) qC[m] = qc[co + m * WHc];
    const int mn = R.dir == 0 ? 1 : 2;
    {
        const int fi = R.dir == 0 ? R.fi : R.fi + b, fj = R.dir == 0 ? R.fj + b : R.fj;
        const int fn = R.dir == 0 ? fi : fj, fl = R.dir == 0 ? fj : fi;
        const int e = R.side > 0 ? fn : fn + 1;   // the fine cell's west / south or east / north edge
        double am[3], ap[3], f[3], fl3[3];
        const long long fo = F.qoff + (long long)(fj + 2) * Wf + (fi + 2);
        if (k.swe) {
            swe_edge_terms<LIM>(qf + F.qoff, Wf, WHf, R.dir, e, fl, 0.5 * k.grav, R.dir == 0 ? lx : ly,
                                R.dir == 0 ? ly : lx, k.order, k.transverse, am, ap, f);
            const double qF[3] = {qf[fo], qf[fo + WHf], qf[fo + 2 * WHf]};
            swe_flux_diff(qF, qC, mn, k.grav, fl3);   // f(Q_F) - f(Q_C) in the edge's order
        } else {
            const UMed md = umed(k);
            edge_terms<LIM>(qf + F.qoff, Wf, WHf, R.dir, e, fl, md, R.dir == 0 ? lx : ly, R.dir == 0 ? ly : lx,
                            k.order, k.transverse, am, ap, f);
            const double dp = qf[fo] - qC[0], dn = qf[fo + mn * WHf] - qC[mn];
            // A (Q_F - Q_C) in the edge's order: (K dn, dp / rho, 0)
            fl3[0] = md.K * dn;
            fl3[1] = dp * md.irho;
            fl3[2] = 0.0;
        }
        double tt[3], o[3];
        for (int m = 0; m < 3; ++m) tt[m] = fl3[m] + (R.side > 0 ? -ap[m] : am[m]) + f[m];
        to_puv(R.dir, tt, o);
        double* slot = buf + 3 * (n + t);
        for (int m = 0; m < 3; ++m) slot[m] += o[m];
    }
}

// one thread per corrected coarse cell: its records in table order (deterministic sums)
__global__ void reflux_apply_kernel(const RefluxRec* __restrict__ recs, int n, const int* __restrict__ group, int ng,
                                    int ratio, const PatchDev* __restrict__ cp, const double* __restrict__ dt,
                                    const double* __restrict__ buf, double* __restrict__ qc)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ng) return;
    const int r0 = group[g], r1 = group[g + 1];
    const RefluxRec R0 = recs[r0];
    const PatchDev C = cp[R0.cbox];
    const double d = __ldg(dt + C.run) * C.dtscale;
    const double w = 1.0 / ((double)ratio * ratio);
    double corr[3] = {0.0, 0.0, 0.0};
    for (int r = r0; r < r1; ++r) {
        const RefluxRec R = recs[r];
        const double s = -R.side * d * (R.dir == 0 ? C.dxinv : C.dyinv);
        for (int m = 0; m < 3; ++m) {
            double fine = 0.0;
            for (int b = 0; b < ratio; ++b) fine += buf[3 * (n + r * ratio + b) + m];
            corr[m] = fma(s, fma(w, fine, buf[3 * r + m]), corr[m]);
        }
    }
    const int W = C.nx + 4;
    const long long WH = (long long)W * (C.ny + 4);
    const long long o = C.qoff + (long long)(R0.cj + 2) * W + (R0.ci + 2);
    for (int m = 0; m < 3; ++m) qc[o + m * WH] += corr[m];
}

}  // namespace

static inline int blocks_for(int n) { return (n + 127) / 128; }

cudaError_t launch_reflux_coarse(const RefluxRec* rec, int n, const PatchDev* cp, const double* qc, const double* dt,
                                 double* buf, int ratio, const StepArgs& k, int limiter, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    switch (limiter) {
    case CLAW_LIM_NONE: reflux_coarse_kernel<CLAW_LIM_NONE><<<blocks_for(n), 128, 0, s>>>(rec, n, cp, qc, dt, buf, ratio, k); break;
    case CLAW_LIM_MINMOD: reflux_coarse_kernel<CLAW_LIM_MINMOD><<<blocks_for(n), 128, 0, s>>>(rec, n, cp, qc, dt, buf, ratio, k); break;
    case CLAW_LIM_SUPERBEE: reflux_coarse_kernel<CLAW_LIM_SUPERBEE><<<blocks_for(n), 128, 0, s>>>(rec, n, cp, qc, dt, buf, ratio, k); break;
    case CLAW_LIM_VANLEER: reflux_coarse_kernel<CLAW_LIM_VANLEER><<<blocks_for(n), 128, 0, s>>>(rec, n, cp, qc, dt, buf, ratio, k); break;
    case CLAW_LIM_MC: reflux_coarse_kernel<CLAW_LIM_MC><<<blocks_for(n), 128, 0, s>>>(rec, n, cp, qc, dt, buf, ratio, k); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_reflux_fine(const RefluxRec* rec, int n, const PatchDev* cp, const PatchDev* fp, const double* qf,
                               const double* qc, const double* dt, double* buf, int ratio, const StepArgs& k,
                               int limiter, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    switch (limiter) {
    case CLAW_LIM_NONE: reflux_fine_kernel<CLAW_LIM_NONE><<<blocks_for(n * ratio), 128, 0, s>>>(rec, n, cp, fp, qf, qc, dt, buf, ratio, k); break;
    case CLAW_LIM_MINMOD: reflux_fine_kernel<CLAW_LIM_MINMOD><<<blocks_for(n * ratio), 128, 0, s>>>(rec, n, cp, fp, qf, qc, dt, buf, ratio, k); break;
    case CLAW_LIM_SUPERBEE: reflux_fine_kernel<CLAW_LIM_SUPERBEE><<<blocks_for(n * ratio), 128, 0, s>>>(rec, n, cp, fp, qf, qc, dt, buf, ratio, k); break;
    case CLAW_LIM_VANLEER: reflux_fine_kernel<CLAW_LIM_VANLEER><<<blocks_for(n * ratio), 128, 0, s>>>(rec, n, cp, fp, qf, qc, dt, buf, ratio, k); break;
    case CLAW_LIM_MC: reflux_fine_kernel<CLAW_LIM_MC><<<blocks_for(n * ratio), 128, 0, s>>>(rec, n, cp, fp, qf, qc, dt, buf, ratio, k); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_reflux_apply(const RefluxRec* rec, int n, const int* group, int ngroups, int ratio,
                                const PatchDev* cp, const double* dt, const double* buf, double* qc, cudaStream_t s)
{
    if (ngroups <= 0) return cudaSuccess;
    reflux_apply_kernel<<<blocks_for(ngroups), 128, 0, s>>>(rec, n, group, ngroups, ratio, cp, dt, buf, qc);
    return cudaGetLastError();
}

}  // namespace claw

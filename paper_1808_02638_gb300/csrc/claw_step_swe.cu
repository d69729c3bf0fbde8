// claw_step_swe.cu -- the fused, persistent level-step for a nonlinear system: the shallow
// water equations on a flat bottom, q = (h, hu, hv), with the Roe normal and transverse
// solvers (the framework takes any system through its Riemann solvers, Sec. 3.1 and 3.3).
//
// Same skeleton as the acoustics kernel (claw_step.cuh): persistent CTAs walk the level's
// tile table, the (tx+4) x (ty+4) x 3 input tile is staged into shared memory by a tensor
// bulk copy (double-buffered) or by coalesced loads, every edge is solved once per tile, the
// tile's largest wave speed is folded on the integer pipe and the last CTA applies Eq. cfl.
// The physics differs in every phase:
//   P0  per staged cell: sqrt(h), hu / sqrt(h), hv / sqrt(h) (one reciprocal square root)
//   PA  per edge: Roe state (normal velocity un, tangential ut, celerity c, 1/(2c)) and the
//       strengths alpha_1..3 of the waves on r1 = (1, un - c, ut), r2 = (0, 0, 1),
//       r3 = (1, un + c, ut)  [components (h, normal momentum, tangential momentum)]
//   PB  per limited edge: mu_p = phi(theta_p) alpha_p without a division by alpha (the upwind
//       strength is projected on r_p: alpha_I (r_I . r_p) / (r_p . r_p)), and the correction
//       part h_p = |s_p| (1 - dt/dx |s_p|) mu_p / 2, so that F~ = sum_p h_p r_p
//   PC  per cell: the two fluctuations entering it (from the edge on either side) as
//       coefficients on the r_p of their edge, the normal update, and the transverse split
//       of each with the same edge's Roe state into down- and up-going parts
//   PD  per cell: the update of Eq. wave_form_2d_2nd_order from Q^n, the normal parts and
//       the differences of the transverse parts.
// A fluctuation with coefficients d_p on r_p splits on the transverse eigenvectors
// (1, un, ut - c), (0, 1, 0), (1, un, ut + c) with strengths (d1 + d3)/2 - d2/(2c),
// c (d3 - d1), (d1 + d3)/2 + d2/(2c): no second Roe solve is needed.
//
// Algorithmic FP64 instructions per cell-update (each edge once, no halo recomputation; a
// reciprocal or reciprocal square root costs 5 FP64-pipe instructions and a division 8, as the
// profiler's instruction counters show for the CUDA routines):
//   P0  rsqrt + 3 DMUL                                                        8
//   PA  per edge: sum, reciprocal, two averages (4), celerity (2 + rsqrt + 2),
//       jumps 3, strengths 7                                         2 x 29 = 58
//   PB  per edge: speeds 2, |r|^2 of waves 1, 3 with one reciprocal (11), upwind projections
//       2 x (1 + 2 + 2), limiters 3, h_p 3 x 4 + 1                    2 x 39 = 78
//   PC  per cell and direction: two sides of 42 (speeds 2, parts 3, normal 7, transverse input
//       3, split 27) less the 9 accumulations into zero; the update Q - l N   2 x 75 + 6 = 156
//   PD  transverse differences, 3 x 8                                        24
//   total 324 (the tile's halo adds about a third in the kernel).
#include "claw_step.cuh"

namespace claw {

template <int TX, int TY> struct SweGeo {
    using Q = Geo<TX, TY>;
    static constexpr int XE = Q::XEW * Q::XEH;   // x-edges a in [-1, TX+1], rows [-1, TY]
    static constexpr int YE = Q::YEW * Q::YEH;   // y-edges b in [-1, TY+1], columns [-1, TX]
    static constexpr int XL = Q::XLW * Q::XLH;   // limited x-edges a in [0, TX], rows [-1, TY]
    static constexpr int YL = Q::YLW * Q::YLH;   // limited y-edges b in [0, TY], columns [-1, TX]
    static constexpr int DC = Q::DW * Q::DH;     // cells [0, TX) x [-1, TY]
    static constexpr int EC = Q::EW * Q::EH;     // cells [-1, TX] x [0, TY)
    static constexpr int NE = 7;                 // per edge: un, ut, c, 1/(2c), alpha_1..3
    static constexpr int DER = 3 * Q::QPL;       // P0 planes; reused for the x-edge h_p in PB
    static_assert(3 * XL <= DER, "limited x-edge parts fit over the derived planes");
    static constexpr int NWORK = DER + NE * (XE + YE) + 3 * YL + 6 * (DC + EC);
    // rows a tile hands to the tile above it in a column walk: x-edge Roe states and strengths
    // 2 rows, y-edge ones 3, limited x-edge parts 2, limited y-edge parts 1, the transverse parts
    // of D one row
    static constexpr int C_XE = 0, C_YE = NE * 2 * Q::XEW, C_XH = C_YE + NE * 3 * Q::YEW,
                         C_YH = C_XH + 3 * 2 * Q::XLW, C_D = C_YH + 3 * Q::YLW, NCARRY = C_D + 6 * Q::DW;
    // q buffers, work arrays, 64 bytes of barriers, then (column walks only) the carried rows
    static size_t smem_bytes(int nbuf, bool walk = false)
    {
        return (size_t)(nbuf * Q::QSTRIDE + NWORK) * 8 + 64 + (walk ? (size_t)NCARRY * 8 : 0);
    }
};

namespace swe {
// max(s, 0) and min(s, 0) by the sign bit (integer pipe)
__device__ __forceinline__ double pos(double s) { return __double_as_longlong(s) < 0 ? 0.0 : s; }
__device__ __forceinline__ double neg(double s) { return __double_as_longlong(s) < 0 ? s : 0.0; }
__device__ __forceinline__ unsigned long long mag(double s)
{
    return (unsigned long long)(__double_as_longlong(s) & 0x7fffffffffffffffLL);
}

// fluctuation with coefficients d1..d3 on the normal eigenvectors of an edge with Roe state
// (un, ut, c, i2c): adds its down-going (negative transverse speeds) part to bm and its
// up-going part to bp, components (h, normal, tangential)
__device__ __forceinline__ void tsplit(double d1, double d2, double d3, double un, double ut, double c,
                                       double i2c, double* bm, double* bp)
{
    const double dh = d1 + d3;
    const double t = d2 * i2c;
    const double b1 = fma(0.5, dh, -t);
    const double b3 = fma(0.5, dh, t);
    const double b2 = c * (d3 - d1);
    const double m1 = ut - c, m3 = ut + c;
    // each family goes one way: its product lands in the down- or the up-going part
    const double g1 = m1 * b1, g2 = ut * b2, g3 = m3 * b3;
    const bool n1 = __double_as_longlong(m1) < 0, n2 = __double_as_longlong(ut) < 0,
               n3 = __double_as_longlong(m3) < 0;
    const double gm1 = n1 ? g1 : 0.0, gm2 = n2 ? g2 : 0.0, gm3 = n3 ? g3 : 0.0;
    const double gp1 = n1 ? 0.0 : g1, gp2 = n2 ? 0.0 : g2, gp3 = n3 ? 0.0 : g3;
    const double Gm = gm1 + gm3, Gp = gp1 + gp3;
    bm[0] += Gm;
    bm[1] += fma(un, Gm, gm2);
    bm[2] += fma(ut, Gm, c * (gm3 - gm1));
    bp[0] += Gp;
    bp[1] += fma(un, Gp, gp2);
    bp[2] += fma(ut, Gp, c * (gp3 - gp1));
}
}  // namespace swe

// STAGE: 0 cooperative loads, 1 tensor bulk copies (double buffered).  PULL: ghosts taken from
// their source cells (separate instantiations, as for acoustics).
template <int LIM, int TX, int TY, int NT, int STAGE, bool PULL>
__global__ void __launch_bounds__(NT, 1) swe_step_kernel(const StepArgs A)
{
    using G = Geo<TX, TY>;
    using S = SweGeo<TX, TY>;
    constexpr int NBUF = STAGE ? 2 : 1;
    constexpr int NPER = (TX * TY + NT - 1) / NT;
    if (A.step_grid && blockIdx.x >= A.step_grid) {   // a fill CTA (as in the acoustics kernel)
        fill_jobs<NT>(A);
        if (threadIdx.x == 0) finish_cta(A);
        return;
    }
    const int nstep = A.step_grid ? A.step_grid : (int)gridDim.x;   // the CTAs that step tiles
    extern __shared__ __align__(128) double smem[];
    double* qbuf = smem;
    double* der = smem + NBUF * G::QSTRIDE;   // sqrt(h), hu/sqrt(h), hv/sqrt(h)
    double* XE = der + S::DER;                // S::NE planes of S::XE
    double* YE = XE + S::NE * S::XE;          // S::NE planes of S::YE
    double* YH = YE + S::NE * S::YE;          // 3 planes of S::YL
    double* Dm = YH + 3 * S::YL;              // x-fluctuation transverse parts: 3 planes of S::DC
    double* Dp = Dm + 3 * S::DC;
    double* Em = Dp + 3 * S::DC;              // y-fluctuation transverse parts: 3 planes of S::EC
    double* Ep = Em + 3 * S::EC;
    unsigned long long* bar = reinterpret_cast<unsigned long long*>(Ep + 3 * S::EC);
    double* Cy = reinterpret_cast<double*>(bar) + 8;   // carried rows (walking launches only)
    double* XH = der;                         // h_p of the limited x-edges (after PA)
    __shared__ unsigned long long s_tmax[2];
    __shared__ int s_flag;
    __shared__ int s_range[2];

    const int tid = threadIdx.x;
    if (tid == 0) {
        s_tmax[0] = s_tmax[1] = 0ull;
        s_flag = 0;
        if (STAGE) {
            mbar_init(&bar[0], 1);
            mbar_init(&bar[1], 1);
            fence_barrier_init();
        }
        if (A.tcum) {
            s_range[0] = walk_start(A.tcum, A.ntiles, blockIdx.x, nstep);
            s_range[1] = walk_start(A.tcum, A.ntiles, blockIdx.x + 1, nstep);
        } else {
            s_range[0] = blockIdx.x;
            s_range[1] = A.ntiles;
        }
    }
    __syncthreads();
    // column walks as in the acoustics kernel: a contiguous stretch of tiles per CTA, the rows a
    // tile shares with the tile below it taken from that tile (through Cy) instead of recomputed
    const int t_begin = s_range[0], t_end = s_range[1];
    const int t_step = A.tcum ? 1 : nstep;
    const bool walk = A.tcum != nullptr;

    const CUtensorMap* tmaps = reinterpret_cast<const CUtensorMap*>(A.tmaps);
    int my_flag = 0;
    int cur_run = -1;
    unsigned long long cur_max = 0ull;
    auto flush = [&]() {
        if (cur_run >= 0 && cur_max)
            atomicMax(reinterpret_cast<unsigned long long*>(A.smax) + cur_run, cur_max);
    };
    const double hg = 0.5 * A.grav;
    const bool second = A.order == 2 && LIM >= 0;
    const bool trans = A.transverse != 0;
    // transverse input = normal-update part -/+ hw h_p: the full correction C rides the split
    // for transverse = 2, none of it for transverse = 1
    const double hw = (A.transverse == 2 && A.order == 2) ? 1.0 : -1.0;

    auto issue = [&](int t, int b) {
        const TileDev T = A.tiles[t];
        mbar_expect_tx(&bar[b], (unsigned)G::QBYTES);
        tma_load_3d(qbuf + b * G::QSTRIDE, &tmaps[T.patch], T.x0, T.y0, 0, &bar[b]);
    };
    if (STAGE && tid == 0 && t_begin < t_end) issue(t_begin, 0);

    int it = 0;
    for (int t = t_begin; t < t_end; t += t_step, ++it) {
        const int b = STAGE ? (it & 1) : 0;
        const TileDev T = A.tiles[t];
        const bool carry = walk && t > t_begin && (T.flags & TILE_CARRY);
        const bool hand = walk && t + 1 < t_end && (A.tiles[t + 1].flags & TILE_CARRY);
        // first rows computed: with a carry, the rows below come from the previous tile
        const int rx0 = carry ? 1 : -1;   // x-edges and limited x-edges: rows [rx0, ty]
        const int by0 = carry ? 2 : -1;   // y-edges: b in [by0, ty + 1]
        const int ly0 = carry ? 1 : 0;    // limited y-edges: b in [ly0, ty]
        const PatchDev P = A.patches[T.patch];
        const int tx = T.tx, ty = T.ty, x0 = T.x0, y0 = T.y0;
        const int W = P.nx + 4;
        const long long WH = (long long)W * (P.ny + 4);
        double* sq = qbuf + b * G::QSTRIDE;
        const double* sh = sq;
        const double* su = sq + G::QPL;
        const double* sv = sq + 2 * G::QPL;

        if (STAGE) {
            const int tn = t + t_step;
            if (tid == 0 && tn < t_end) issue(tn, b ^ 1);
            const unsigned par = (unsigned)((it >> 1) & 1);
            bool ok = mbar_wait_bounded(&bar[b], par, A.wait_polls);
            if (__syncthreads_or(!ok)) {   // late or lost copy: report, drain what is in flight, stop
                if (tid == 0) {
                    atomicOr(A.err, ERR_TIMEOUT);
                    mbar_wait_bounded(&bar[b], par);
                    if (tn < t_end) mbar_wait_bounded(&bar[b ^ 1], (unsigned)(((it + 1) >> 1) & 1));
                    finish_cta(A);
                }
                return;
            }
        } else {
            const double* src = A.qold + P.qoff;
            for (int k = tid; k < 3 * G::QPL; k += NT) {
                const int m = k / G::QPL, rem = k - m * G::QPL;
                const int jj = rem / G::SW, ii = rem - jj * G::SW;
                double v = 0.0;
                if (ii < tx + 4 && jj < ty + 4) v = __ldg(src + m * WH + (long long)(y0 + jj) * W + (x0 + ii));
                sq[k] = v;
            }
            __syncthreads();
        }
        if (PULL && P.ring >= 0) {
            pull_ghosts<G::SW, G::QPL, NT>(A, P, sq, x0, y0, tx, ty);
            __syncthreads();
        }
        const double dt = __ldg(A.dt + P.run) * P.dtscale;
        const double lx = dt * P.dxinv, ly = dt * P.dyinv;

        // ------------------------------------------------------------ P0: per staged cell
        // (with a carry only the staged rows from 3 on, tile rows 1.., feed this tile's edges)
        // The carried edge rows land in the lowest rows of XE, YE, YH and D, which this tile
        // writes no earlier than PA; the previous tile's last reads of them were behind its
        // end-of-tile barrier.  (XH shares memory with der and is restored after PA.)
        if (carry) {
            for (int k = tid; k < S::C_XH; k += NT) {
                if (k < S::C_YE) {
                    const int q = k / (2 * G::XEW), o = k - q * 2 * G::XEW;
                    XE[q * S::XE + o] = Cy[k];
                } else {
                    const int kk = k - S::C_YE, q = kk / (3 * G::YEW), o = kk - q * 3 * G::YEW;
                    YE[q * S::YE + o] = Cy[k];
                }
            }
            for (int k = tid; k < S::NCARRY - S::C_YH; k += NT) {
                if (k < 3 * G::YLW) {
                    const int q = k / G::YLW;
                    YH[q * S::YL + (k - q * G::YLW)] = Cy[S::C_YH + k];
                } else {
                    const int kk = k - 3 * G::YLW, q = kk / G::DW, o = kk - q * G::DW;
                    (q < 3 ? Dm + q * S::DC : Dp + (q - 3) * S::DC)[o] = Cy[S::C_D + kk];
                }
            }
        }
        {
            const int w = tx + 4, j0 = carry ? 3 : 0, n = (ty + 4 - j0) * w;
            for (int k = tid; k < n; k += NT) {
                const int jj = k / w + j0, ii = k - (jj - j0) * w;
                const int i = ii + jj * G::SW;
                const double h = sh[i];
                const bool corner = (ii == 0 || ii == w - 1) && (jj == 0 || jj == ty + 3);
                if (!corner && __double_as_longlong(h) <= 0) my_flag |= ERR_NAN;   // not wet
                const double r = rsqrt(h);
                der[i] = h * r;
                der[G::QPL + i] = su[i] * r;
                der[2 * G::QPL + i] = sv[i] * r;
            }
        }
        __syncthreads();

        // ------------------------------------------------------------ PA: Roe solves
        unsigned long long m = 0ull;
        {   // x-edge a (cells a-1 | a) on rows r in [-1, ty]
            const int w = tx + 3, n = (ty + 1 - rx0) * w;
            for (int k = tid; k < n; k += NT) {
                const int r = k / w + rx0, a = k - (r - rx0) * w - 1;
                const int iR = (a + 2) + (r + 2) * G::SW, iL = iR - 1;
                const double inv = 1.0 / (der[iL] + der[iR]);
                const double un = (der[G::QPL + iL] + der[G::QPL + iR]) * inv;
                const double ut = (der[2 * G::QPL + iL] + der[2 * G::QPL + iR]) * inv;
                const double x = (sh[iL] + sh[iR]) * hg;
                const double rc = rsqrt(x);
                const double c = x * rc, i2c = 0.5 * rc;
                const double dh = sh[iR] - sh[iL], dn = su[iR] - su[iL], dtg = sv[iR] - sv[iL];
                const int e = (r + 1) * G::XEW + (a + 1);
                XE[e] = un;
                XE[S::XE + e] = ut;
                XE[2 * S::XE + e] = c;
                XE[3 * S::XE + e] = i2c;
                XE[4 * S::XE + e] = fma(un + c, dh, -dn) * i2c;
                XE[5 * S::XE + e] = fma(-ut, dh, dtg);
                XE[6 * S::XE + e] = fma(-(un - c), dh, dn) * i2c;
                if (a >= 0 && a <= tx) {
                    const unsigned long long s1 = swe::mag(un - c), s3 = swe::mag(un + c);
                    m = umax64(m, umax64(s1, s3));
                }
            }
        }
        {   // y-edge b (rows b-1 | b) on columns c in [-1, tx]; normal momentum hv
            const int w = tx + 2, n = (ty + 2 - by0) * w;
            for (int k = tid; k < n; k += NT) {
                const int bb = k / w + by0, cc = k - (bb - by0) * w - 1;
                const int iR = (cc + 2) + (bb + 2) * G::SW, iL = iR - G::SW;
                const double inv = 1.0 / (der[iL] + der[iR]);
                const double un = (der[2 * G::QPL + iL] + der[2 * G::QPL + iR]) * inv;
                const double ut = (der[G::QPL + iL] + der[G::QPL + iR]) * inv;
                const double x = (sh[iL] + sh[iR]) * hg;
                const double rc = rsqrt(x);
                const double c = x * rc, i2c = 0.5 * rc;
                const double dh = sh[iR] - sh[iL], dn = sv[iR] - sv[iL], dtg = su[iR] - su[iL];
                const int e = (bb + 1) * G::YEW + (cc + 1);
                YE[e] = un;
                YE[S::YE + e] = ut;
                YE[2 * S::YE + e] = c;
                YE[3 * S::YE + e] = i2c;
                YE[4 * S::YE + e] = fma(un + c, dh, -dn) * i2c;
                YE[5 * S::YE + e] = fma(-ut, dh, dtg);
                YE[6 * S::YE + e] = fma(-(un - c), dh, dn) * i2c;
                if (bb >= 0 && bb <= ty) {
                    const unsigned long long s1 = swe::mag(un - c), s3 = swe::mag(un + c);
                    m = umax64(m, umax64(s1, s3));
                }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = umax64(m, __shfl_xor_sync(0xffffffffu, m, o));
        if ((tid & 31) == 0 && m) atomicMax(&s_tmax[it & 1], m);
        __syncthreads();

        // ------------------------------------------------------------ PB: limiter, correction
        // h_p = |s_p| (1 - l |s_p|) mu_p / 2 for the limited edges; the upwind edge of wave p
        // is the one behind it (s_p > 0: the edge before), as in theta_p's definition
        auto limited = [&](const double* E, int plane, int e, int eb, int ef, double l, double* out, int o, int ol) {
            const double un = E[e], ut = E[plane + e], c = E[2 * plane + e];
            const double s1 = un - c, s3 = un + c;
            const double a1 = E[4 * plane + e], a2 = E[5 * plane + e], a3 = E[6 * plane + e];
            const int u1 = __double_as_longlong(s1) > 0 ? eb : ef;
            const int u2 = __double_as_longlong(un) > 0 ? eb : ef;
            const int u3 = __double_as_longlong(s3) > 0 ? eb : ef;
            // 1 / (r1 . r1) and 1 / (r3 . r3) from one reciprocal of their product
            const double w = fma(ut, ut, 1.0);
            const double rr1 = fma(s1, s1, w), rr3 = fma(s3, s3, w);
            const double ip = 1.0 / (rr1 * rr3);
            double mu1, mu2, mu3;
            {   // wave 1 on (1, un - c, ut)
                const double unI = E[u1], utI = E[plane + u1], cI = E[2 * plane + u1];
                const double ri = fma(unI - cI, s1, fma(utI, ut, 1.0));
                mu1 = Lim<LIM>::f(a1, E[4 * plane + u1] * ri * (rr3 * ip));
            }
            mu2 = Lim<LIM>::f(a2, E[5 * plane + u2]);
            {   // wave 3 on (1, un + c, ut)
                const double unI = E[u3], utI = E[plane + u3], cI = E[2 * plane + u3];
                const double ri = fma(unI + cI, s3, fma(utI, ut, 1.0));
                mu3 = Lim<LIM>::f(a3, E[6 * plane + u3] * ri * (rr1 * ip));
            }
            const double k1 = fabs(s1), k2 = fabs(un), k3 = fabs(s3);
            const double hl = -0.5 * l;
            out[o] = fma(hl * k1, k1, 0.5 * k1) * mu1;
            out[ol + o] = fma(hl * k2, k2, 0.5 * k2) * mu2;
            out[2 * ol + o] = fma(hl * k3, k3, 0.5 * k3) * mu3;
        };
        if (second) {
            if (carry)   // the carried limited x-edge rows, now that PA has read der
                for (int k = tid; k < S::C_YH - S::C_XH; k += NT) {
                    const int q = k / (2 * G::XLW), o = k - q * 2 * G::XLW;
                    XH[q * S::XL + o] = Cy[S::C_XH + k];
                }
            {
                const int w = tx + 1, n = (ty + 1 - rx0) * w;
                for (int k = tid; k < n; k += NT) {
                    const int r = k / w + rx0, a = k - (r - rx0) * w;
                    const int e = (r + 1) * G::XEW + (a + 1);
                    limited(XE, S::XE, e, e - 1, e + 1, lx, XH, (r + 1) * G::XLW + a, S::XL);
                }
            }
            {
                const int w = tx + 2, n = (ty + 1 - ly0) * w;
                for (int k = tid; k < n; k += NT) {
                    const int bb = k / w + ly0, cc = k - (bb - ly0) * w - 1;
                    const int e = (bb + 1) * G::YEW + (cc + 1);
                    limited(YE, S::YE, e, e - G::YEW, e + G::YEW, ly, YH, bb * G::YLW + (cc + 1), S::YL);
                }
            }
            __syncthreads();
        }

        // ------------------------------------------------------------ PC: per-cell parts
        // One side of an edge: the fluctuation entering the cell from edge e (right = the cell
        // is right of / above the edge).  Adds the normal-update part (A+dQ - F~ for the cell
        // on the right, A-dQ + F~ on the left; (h, n, t) components) to nrm and the transverse
        // split of the transverse input to bm / bp.
        auto side = [&](const double* E, int plane, int e, const double* H, int lo, int lplane, bool right,
                        double* nrm, double* bm, double* bp) {
            const double un = E[e], ut = E[plane + e], c = E[2 * plane + e], i2c = E[3 * plane + e];
            const double s1 = un - c, s3 = un + c;
            const double a1 = E[4 * plane + e], a2 = E[5 * plane + e], a3 = E[6 * plane + e];
            double h1 = 0.0, h2 = 0.0, h3 = 0.0;
            if (second) {
                h1 = H[lo];
                h2 = H[lplane + lo];
                h3 = H[2 * lplane + lo];
                if (right) {
                    h1 = -h1;
                    h2 = -h2;
                    h3 = -h3;
                }
            }
            const double e1 = fma(right ? swe::pos(s1) : swe::neg(s1), a1, h1);
            const double e2 = fma(right ? swe::pos(un) : swe::neg(un), a2, h2);
            const double e3 = fma(right ? swe::pos(s3) : swe::neg(s3), a3, h3);
            if (nrm) {
                const double eh = e1 + e3;
                nrm[0] += eh;
                nrm[1] += fma(s1, e1, s3 * e3);
                nrm[2] += fma(ut, eh, e2);
            }
            if (trans) {
                double d1 = e1, d2 = e2, d3 = e3;
                if (second) {
                    d1 = fma(hw, h1, e1);
                    d2 = fma(hw, h2, e2);
                    d3 = fma(hw, h3, e3);
                }
                swe::tsplit(d1, d2, d3, un, ut, c, i2c, bm, bp);
            }
        };
        // x-parts of cell (c, r), r in [-1, ty]: edges c (cell on the right) and c+1
        auto xcell = [&](int c, int r, double* nrm) {
            double bm[3] = {0.0, 0.0, 0.0}, bp[3] = {0.0, 0.0, 0.0};
            const int e = (r + 1) * G::XEW + (c + 1), lo = (r + 1) * G::XLW + c;
            side(XE, S::XE, e, XH, lo, S::XL, true, nrm, bm, bp);
            side(XE, S::XE, e + 1, XH, lo + 1, S::XL, false, nrm, bm, bp);
            if (trans) {   // (h, hu, hv) = (h, n, t)
                const int d = (r + 1) * G::DW + c;
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    Dm[q * S::DC + d] = bm[q];
                    Dp[q * S::DC + d] = bp[q];
                }
            }
        };
        // y-parts of cell (c, r), c in [-1, tx]: edges r (cell above) and r+1; (h, n, t) = (h, hv, hu)
        auto ycell = [&](int c, int r, double* nrm) {
            double bm[3] = {0.0, 0.0, 0.0}, bp[3] = {0.0, 0.0, 0.0};
            const int e = (r + 1) * G::YEW + (c + 1), lo = r * G::YLW + (c + 1);
            side(YE, S::YE, e, YH, lo, S::YL, true, nrm, bm, bp);
            side(YE, S::YE, e + G::YEW, YH, lo + G::YLW, S::YL, false, nrm, bm, bp);
            if (trans) {
                const int d = r * G::EW + (c + 1);
                Em[d] = bm[0];
                Em[S::EC + d] = bm[2];
                Em[2 * S::EC + d] = bm[1];
                Ep[d] = bp[0];
                Ep[S::EC + d] = bp[2];
                Ep[2 * S::EC + d] = bp[1];
            }
        };
        double dQ[NPER][3];
#pragma unroll
        for (int n = 0; n < NPER; ++n) {
            dQ[n][0] = dQ[n][1] = dQ[n][2] = 0.0;
            const int ci = tid + n * NT;
            const int c = ci % TX, r = ci / TX;
            if (ci >= TX * TY || c >= tx || r >= ty) continue;
            const int iq = (c + 2) + (r + 2) * G::SW;
            double nx[3] = {0.0, 0.0, 0.0}, ny[3] = {0.0, 0.0, 0.0};
            xcell(c, r, nx);
            ycell(c, r, ny);
            dQ[n][0] = fma(-lx, nx[0], fma(-ly, ny[0], sh[iq]));
            dQ[n][1] = fma(-lx, nx[1], fma(-ly, ny[2], su[iq]));
            dQ[n][2] = fma(-lx, nx[2], fma(-ly, ny[1], sv[iq]));
        }
        if (trans) {   // transverse parts of the ghost rows -1, ty (x) and ghost columns -1, tx (y)
            const int n = 2 * (tx + ty);
            for (int k = tid + (carry ? tx : 0); k < n; k += NT) {   // row -1 is carried
                if (k < 2 * tx) xcell(k % tx, k < tx ? -1 : ty, nullptr);
                else {
                    const int kk = k - 2 * tx;
                    ycell(kk < ty ? -1 : tx, kk % ty, nullptr);
                }
            }
        }
        // hand the top rows of the edge arrays to the next tile (all final by now)
        if (hand) {
            for (int k = tid; k < S::C_D; k += NT) {
                double v;
                if (k < S::C_YE) {
                    const int q = k / (2 * G::XEW), o = k - q * 2 * G::XEW;
                    v = XE[q * S::XE + ty * G::XEW + o];
                } else if (k < S::C_XH) {
                    const int kk = k - S::C_YE, q = kk / (3 * G::YEW), o = kk - q * 3 * G::YEW;
                    v = YE[q * S::YE + ty * G::YEW + o];
                } else if (k < S::C_YH) {
                    const int kk = k - S::C_XH, q = kk / (2 * G::XLW), o = kk - q * 2 * G::XLW;
                    v = XH[q * S::XL + ty * G::XLW + o];
                } else {
                    const int kk = k - S::C_YH, q = kk / G::YLW, o = kk - q * G::YLW;
                    v = YH[q * S::YL + ty * G::YLW + o];
                }
                Cy[k] = v;
            }
        }
        __syncthreads();

        // ------------------------------------------------------------ PD: update, store
        // D of row ty - 1 becomes the next tile's row -1 (final since the barrier ending PC)
        if (hand)
            for (int k = tid; k < 6 * G::DW; k += NT) {
                const int q = k / G::DW, o = k - q * G::DW;
                Cy[S::C_D + k] = (q < 3 ? Dm + q * S::DC : Dp + (q - 3) * S::DC)[ty * G::DW + o];
            }
        const double kT = 0.5 * lx * ly;
        double* dst = A.qnew + P.qoff;
#pragma unroll
        for (int n = 0; n < NPER; ++n) {
            const int ci = tid + n * NT;
            const int c = ci % TX, r = ci / TX;
            if (ci >= TX * TY || c >= tx || r >= ty) continue;
            double out[3] = {dQ[n][0], dQ[n][1], dQ[n][2]};
            if (trans) {
                const int d = (r + 1) * G::DW + c;       // D rows r-1, r, r+1 at d - DW, d, d + DW
                const int f = r * G::EW + (c + 1);       // E columns c-1, c, c+1 at f - 1, f, f + 1
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    const double* dm = Dm + q * S::DC;
                    const double* dp = Dp + q * S::DC;
                    const double* em = Em + q * S::EC;
                    const double* ep = Ep + q * S::EC;
                    const double tr = ((dp[d] - dp[d - G::DW]) + (dm[d + G::DW] - dm[d])) +
                                      ((ep[f] - ep[f - 1]) + (em[f + 1] - em[f]));
                    out[q] = fma(kT, tr, out[q]);
                }
            }
            if (not_finite(out[0]) | not_finite(out[1]) | not_finite(out[2])) my_flag |= ERR_NAN;
            const long long o = (long long)(y0 + r + 2) * W + (x0 + c + 2);
            dst[o] = out[0];
            dst[WH + o] = out[1];
            dst[2 * WH + o] = out[2];
        }
        __syncthreads();   // staged tile and work arrays are reused by the next tile
        if (tid == 0) {
            const unsigned long long mm = s_tmax[it & 1];
            s_tmax[it & 1] = 0ull;
            if (P.run != cur_run) {
                flush();
                cur_run = P.run;
                cur_max = mm;
            } else {
                cur_max = umax64(cur_max, mm);
            }
        }
    }

    if (tid == 0) flush();
    if (my_flag) atomicOr(&s_flag, my_flag);
    __syncthreads();
    if (tid == 0 && s_flag) atomicOr(A.err, s_flag);
    if (tid == 0) finish_cta(A);
}

template <int LIM, int TX, int TY, int NT, int STAGE, bool PULL>
static StepKernel swe_entry()
{
    StepKernel k;
    k.fn = swe_step_kernel<LIM, TX, TY, NT, STAGE, PULL>;
    k.smem = SweGeo<TX, TY>::smem_bytes(STAGE ? 2 : 1);
    k.smem_walk = SweGeo<TX, TY>::smem_bytes(STAGE ? 2 : 1, true);
    k.nt = NT;
    return k;
}

template <int LIM, bool PULL>
static StepKernel swe_select(int tx, int ty, int nt, int staging)
{
    if (tx == 16 && ty == 16 && (nt == 0 || nt == 256))
        return staging ? swe_entry<LIM, 16, 16, 256, 1, PULL>() : swe_entry<LIM, 16, 16, 256, 0, PULL>();
    if (tx == 32 && ty == 16 && (nt == 0 || nt == 512))
        return staging ? swe_entry<LIM, 32, 16, 512, 1, PULL>() : swe_entry<LIM, 32, 16, 512, 0, PULL>();
    return StepKernel{nullptr, 0, 0, 0};
}

template <bool PULL>
static StepKernel swe_for(int lim, int tx, int ty, int nt, int staging)
{
    switch (lim) {
    case CLAW_LIM_NONE: return swe_select<CLAW_LIM_NONE, PULL>(tx, ty, nt, staging);
    case CLAW_LIM_MINMOD: return swe_select<CLAW_LIM_MINMOD, PULL>(tx, ty, nt, staging);
    case CLAW_LIM_SUPERBEE: return swe_select<CLAW_LIM_SUPERBEE, PULL>(tx, ty, nt, staging);
    case CLAW_LIM_VANLEER: return swe_select<CLAW_LIM_VANLEER, PULL>(tx, ty, nt, staging);
    case CLAW_LIM_MC: return swe_select<CLAW_LIM_MC, PULL>(tx, ty, nt, staging);
    }
    return StepKernel{nullptr, 0, 0, 0};
}

StepKernel step_kernel_swe(int lim, int tx, int ty, int nt, int staging)
{
    return swe_for<false>(lim, tx, ty, nt, staging);
}

StepKernel step_kernel_swe_pull(int lim, int tx, int ty, int nt, int staging)
{
    return swe_for<true>(lim, tx, ty, nt, staging);
}

}  // namespace claw

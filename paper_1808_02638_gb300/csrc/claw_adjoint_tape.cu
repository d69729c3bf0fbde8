// claw_adjoint_tape.cu -- reverse mode of the cell-wise level-step (second order), driven by the
// step's tape (claw_level_advance_record): the discrete adjoint of the step of claw_step.cuh with
// dt frozen, without re-running any forward phase.
//
// The tape holds, per padded cell, the wave strengths of its west / south edges, their limited
// strengths (with the limiter branch in the lowest mantissa bits) and the cell's transverse
// fluctuation pressures D, E.  So the reverse needs neither q nor a limiter evaluation: it is
// the transposed stencil of the step with the branches frozen, plus the medium adjoint.  Per tile
// (16 x 16 cells, 256 threads, four CTAs per SM, five barriers):
//   1. transverse fluxes: adjoints of D (y-edges) and E (x-edges) per edge, and the medium terms;
//   2. per cell: the adjoints of ap, au, bp, bu (normal update and transverse pressures);
//   3. per edge: gather those, reverse the correction and the limiter (own wave strengths, and
//      the upwind edge's share for a gather in 4);
//   4. per edge: reverse the normal Riemann solve into the jumps dp, du (dv);
//   5. per cell: gather the jumps' adjoints into lam_old (global reductions; ghosts the forward
//      pulled from a cell of the level go to that cell through the ghost ring).
// Every medium adjoint is a global FP64 reduction into g_aux (carried out in the L2, not on the
// FP64 pipe), with the aux layout and meaning of claw_level_step_adjoint (the 1/(Z_L+Z_R) planes
// receive that value times its adjoint).  Accumulating the cell planes in shared memory instead
// (one reduction per cell and plane) was measured slower: shared-memory FP64 atomics take
// FP64-pipe slots.
#include <cuda_runtime.h>

#include "claw_step.cuh"

namespace claw {
namespace {

constexpr int TTX = 16, TTY = 16, TNT = 256;

struct TGeo {
    static constexpr int YT = TTX * (TTY + 1);        // transverse y-edges jj in [0,ty], c in [0,tx)
    static constexpr int XT = (TTX + 1) * TTY;        // transverse x-edges a in [0,tx], r in [0,ty)
    static constexpr int DN = TTX * (TTY + 2);        // D cells: c in [0,tx), r in [-1,ty]
    static constexpr int EN = (TTX + 2) * TTY;        // E cells: c in [-1,tx], r in [0,ty)
    static constexpr int XEW = TTX + 3, XE = XEW * (TTY + 2);   // x-edges a in [-1,tx+1], r in [-1,ty]
    static constexpr int YEW = TTX + 2, YE = YEW * (TTY + 3);   // y-edges b in [-1,ty+1], c in [-1,tx]
    static constexpr int XLW = TTX + 1, XL = XLW * (TTY + 2);   // limited x-edges a in [0,tx]
    static constexpr int YLW = TTX + 2, YL = YLW * (TTY + 1);   // limited y-edges b in [0,ty]
    // the transverse gD / gE slots (read up to phase 2) share their space with the limiters'
    // upwind slots (written from phase 3)
    static constexpr int UN = (2 * YT + 2 * XT) > (2 * XL + 2 * YL) ? (2 * YT + 2 * XT) : (2 * XL + 2 * YL);
    static constexpr int O_GYLO = 0, O_GYHI = O_GYLO + YT, O_GXLO = O_GYHI + YT, O_GXHI = O_GXLO + XT;
    static constexpr int O_U1X = 0, O_U2X = O_U1X + XL, O_U1Y = O_U2X + XL, O_U2Y = O_U1Y + YL;
    static constexpr int O_CGX = UN;                  // gap, gau, gbp, gbu of the D cells
    static constexpr int O_CGY = O_CGX + 4 * DN;      // gap, gav, gbp, gbv of the E cells
    static constexpr int O_A1B = O_CGY + 4 * EN, O_A2B = O_A1B + XE, O_B1B = O_A2B + XE, O_B2B = O_B1B + YE;
    static constexpr int O_END = O_B2B + YE;
    static size_t smem_bytes() { return (size_t)O_END * 8; }
};

__device__ __forceinline__ bool nonzero(double x)   // integer test: a double compare is FP64 work
{
    return ((unsigned long long)__double_as_longlong(x) << 1) != 0ull;
}
__device__ __forceinline__ double flip_sign(double x, int f)
{
    return __longlong_as_double(__double_as_longlong(x) ^ ((long long)(f & 1) << 63));
}

// x 2^e for e in {-1, 0, 1} on the integer pipe (an exponent increment), the FP64 product where
// that would leave the normal range (zeros, subnormals, overflow)
__device__ __forceinline__ double mul_pow2(double x, int e)
{
    const long long b = __double_as_longlong(x);
    const int ex = (int)((b >> 52) & 0x7ff);
    if (e == 0) return x;
    if (ex > 1 && ex < 0x7fe) return __longlong_as_double(b + ((long long)e << 52));
    return x * (e > 0 ? 2.0 : 0.5);
}

// the adjoint of a limited strength m = phi(b/a) a at the branch the forward took (code in the
// tagged value m): own = g + (dm/da) gm, returns (dm/db) gm.  Every branch but van Leer's has
// partials in {0, 1/2, 1, 2}, applied as exponent shifts; van Leer (2ab/(a+b)) needs b, which
// the caller computes only then
__device__ __forceinline__ double lim_adjoint(int code, double a, double b, double gm, double g, double& own)
{
    switch (code) {
    case LIMC_A: own = g + gm; return 0.0;
    case LIMC_B: own = g; return gm;
    case LIMC_2A: own = g + mul_pow2(gm, 1); return 0.0;
    case LIMC_2B: own = g; return mul_pow2(gm, 1);
    case LIMC_HALF: {
        const double h = mul_pow2(gm, -1);
        own = g + h;
        return h;
    }
    case LIMC_SMOOTH: {
        const double s = a + b, is2 = 1.0 / (s * s);
        own = fma(2.0 * b * b * is2, gm, g);
        return 2.0 * a * a * is2 * gm;
    }
    default: own = g; return 0.0;
    }
}

template <int LIM>
__global__ void __launch_bounds__(TNT, 4)
    step_adjoint_tape_kernel(const StepArgs A, const double* __restrict__ lam_new, double* __restrict__ lam_old,
                             double* __restrict__ g_aux)
{
    using G = TGeo;
    extern __shared__ __align__(128) double sm[];
    double* GYlo = sm + G::O_GYLO;
    double* GYhi = sm + G::O_GYHI;
    double* GXlo = sm + G::O_GXLO;
    double* GXhi = sm + G::O_GXHI;
    double* cgx = sm + G::O_CGX;
    double* cgy = sm + G::O_CGY;
    double* A1b = sm + G::O_A1B;
    double* A2b = sm + G::O_A2B;
    double* B1b = sm + G::O_B1B;
    double* B2b = sm + G::O_B2B;
    double* U1x = sm + G::O_U1X;
    double* U2x = sm + G::O_U2X;
    double* U1y = sm + G::O_U1Y;
    double* U2y = sm + G::O_U2Y;

    const int tid = threadIdx.x;
    const bool trans = A.transverse != 0;
    const bool w = A.transverse == 2;   // the correction rides the transverse split

    auto XE = [](int a, int r) { return (a + 1) + (r + 1) * G::XEW; };
    auto YE = [](int c, int b) { return (c + 1) + (b + 1) * G::YEW; };
    auto XL = [](int a, int r) { return a + (r + 1) * G::XLW; };
    auto YL = [](int c, int b) { return (c + 1) + b * G::YLW; };
    auto DI = [](int c, int r) { return c + (r + 1) * TTX; };
    auto EI = [](int c, int r) { return (c + 1) + r * (TTX + 2); };

    for (int t = blockIdx.x; t < A.ntiles; t += gridDim.x) {
        const TileDev T = A.tiles[t];
        const PatchDev P = A.patches[T.patch];
        const int tx = T.tx, ty = T.ty, x0 = T.x0, y0 = T.y0;
        const int W = P.nx + 4;
        const long long WH = (long long)W * (P.ny + 4);
        const double dt = __ldg(A.dt + P.run) * P.dtscale;
        const double lx = dt * P.dxinv, ly = dt * P.dyinv;
        const double kT = -0.5 * lx * ly;
        const double* aux = A.aux + P.aoff;
        const double* tape = A.tape + P.aoff;
        double* gm = g_aux + P.aoff;
        const double* ln = lam_new + P.qoff;
        auto cell = [&](int i, int j) -> long long { return (long long)(y0 + j + 2) * W + (x0 + i + 2); };
        auto AX = [&](int k, int i, int j) -> double { return __ldg(aux + k * WH + cell(i, j)); };
        auto TP = [&](int k, int i, int j) -> double { return __ldg(tape + k * WH + cell(i, j)); };
        auto LAM = [&](int m, int c, int r) -> double {
            if (c < 0 || c >= tx || r < 0 || r >= ty) return 0.0;
            return __ldg(ln + m * WH + cell(c, r));
        };
        auto medadd = [&](int k, int i, int j, double v) {
            if (nonzero(v)) atomicAdd(gm + k * WH + cell(i, j), v);
        };

        // ------------------------------------------------------------ 1. transverse fluxes
        // y-edge jj of column c (lo = (c, jj-1), hi = (c, jj)):
        //   Gp = -lx/2 is (K_hi D_lo - K_lo D_hi),  Gv = -lx/2 is (c_hi D_lo + c_lo D_hi),
        //   adjoints gGp = ly (lam_p(hi) - lam_p(lo)), gGv likewise; U = -lx/2 gGp, V = -lx/2 gGv
        if (trans) {
            for (int k = tid; k < (ty + 1) * tx; k += TNT) {
                const int jj = k / tx, c = k - jj * tx;
                const double U = kT * (LAM(0, c, jj) - LAM(0, c, jj - 1));
                const double V = kT * (LAM(2, c, jj) - LAM(2, c, jj - 1));
                if (!nonzero(U) && !nonzero(V)) {
                    GYlo[c + jj * TTX] = 0.0;
                    GYhi[c + jj * TTX] = 0.0;
                    continue;
                }
                const double Khi = AX(AUX_K, c, jj), chi = AX(AUX_C, c, jj);
                const double Klo = AX(AUX_K, c, jj - 1), clo = AX(AUX_C, c, jj - 1);
                const double is = AX(AUX_IYS, c, jj);
                const double Dlo = TP(TAPE_D, c, jj - 1), Dhi = TP(TAPE_D, c, jj);
                const double X = fma(Khi, U, chi * V), Y = fma(clo, V, -(Klo * U));
                GYlo[c + jj * TTX] = is * X;
                GYhi[c + jj * TTX] = is * Y;
                medadd(AUX_IYS, c, jj, fma(Dlo, GYlo[c + jj * TTX], Dhi * GYhi[c + jj * TTX]));   // is x its adjoint
                const double sl = is * Dlo, sh = is * Dhi;
                medadd(AUX_K, c, jj, sl * U);
                medadd(AUX_C, c, jj, sl * V);
                medadd(AUX_K, c, jj - 1, -(sh * U));
                medadd(AUX_C, c, jj - 1, sh * V);
            }
            // x-edge a of row r (L = (a-1, r), R = (a, r)): Fp, Fu from E, mirrored
            for (int k = tid; k < (tx + 1) * ty; k += TNT) {
                const int r = k / (tx + 1), a = k - r * (tx + 1);
                const double U = kT * (LAM(0, a, r) - LAM(0, a - 1, r));
                const double V = kT * (LAM(1, a, r) - LAM(1, a - 1, r));
                if (!nonzero(U) && !nonzero(V)) {
                    GXlo[a + r * (TTX + 1)] = 0.0;
                    GXhi[a + r * (TTX + 1)] = 0.0;
                    continue;
                }
                const double KR = AX(AUX_K, a, r), cR = AX(AUX_C, a, r);
                const double KL = AX(AUX_K, a - 1, r), cL = AX(AUX_C, a - 1, r);
                const double is = AX(AUX_IXS, a, r);
                const double EL = TP(TAPE_E, a - 1, r), ER = TP(TAPE_E, a, r);
                const double X = fma(KR, U, cR * V), Y = fma(cL, V, -(KL * U));
                GXlo[a + r * (TTX + 1)] = is * X;
                GXhi[a + r * (TTX + 1)] = is * Y;
                medadd(AUX_IXS, a, r, fma(EL, GXlo[a + r * (TTX + 1)], ER * GXhi[a + r * (TTX + 1)]));
                const double sl = is * EL, sh = is * ER;
                medadd(AUX_K, a, r, sl * U);
                medadd(AUX_C, a, r, sl * V);
                medadd(AUX_K, a - 1, r, -(sh * U));
                medadd(AUX_C, a - 1, r, sh * V);
            }
        }
        __syncthreads();

        // ------------------------------------------------------------ 2. per-cell terms
        // D = K ap + w bp; interior: dP = -lx (K ap + bp/2), dU = -lx (c au + bu/2);
        // ap = a2(west edge) + a1(east edge), au = a2(west) - a1(east), bp, bu: correction jumps
        for (int k = tid; k < (ty + 2) * tx; k += TNT) {
            const int r = k / tx - 1, c = k - (r + 1) * tx;
            double gD = 0.0;
            if (trans) {
                if (r <= ty - 1) gD += GYlo[c + (r + 1) * TTX];   // lo cell of y-edge r+1
                if (r >= 0) gD += GYhi[c + r * TTX];              // hi cell of y-edge r
            }
            const bool in = r >= 0 && r < ty;
            const double Kc = AX(AUX_K, c, r);
            const double a2w = TP(TAPE_A2, c, r), a1e = TP(TAPE_A1, c + 1, r);
            const double ap = a2w + a1e;
            double t = gD, gbp = w ? gD : 0.0, gau = 0.0, gbu = 0.0;
            if (in) {
                const double tp = -lx * LAM(0, c, r), tu = -lx * LAM(1, c, r);
                t += tp;
                gbp = fma(0.5, tp, gbp);
                gau = AX(AUX_C, c, r) * tu;
                gbu = 0.5 * tu;
                medadd(AUX_C, c, r, (a2w - a1e) * tu);
            }
            cgx[0 * G::DN + DI(c, r)] = Kc * t;
            cgx[1 * G::DN + DI(c, r)] = gau;
            cgx[2 * G::DN + DI(c, r)] = gbp;
            cgx[3 * G::DN + DI(c, r)] = gbu;
            medadd(AUX_K, c, r, ap * t);
        }
        for (int k = tid; k < ty * (tx + 2); k += TNT) {
            const int r = k / (tx + 2), c = k - r * (tx + 2) - 1;
            double gE = 0.0;
            if (trans) {
                if (c <= tx - 1) gE += GXlo[(c + 1) + r * (TTX + 1)];   // L cell of x-edge c+1
                if (c >= 0) gE += GXhi[c + r * (TTX + 1)];              // R cell of x-edge c
            }
            const bool in = c >= 0 && c < tx;
            const double Kc = AX(AUX_K, c, r);
            const double b2s = TP(TAPE_B2, c, r), b1n = TP(TAPE_B1, c, r + 1);
            const double ap = b2s + b1n;
            double t = gE, gbp = w ? gE : 0.0, gav = 0.0, gbv = 0.0;
            if (in) {
                const double tp = -ly * LAM(0, c, r), tv = -ly * LAM(2, c, r);
                t += tp;
                gbp = fma(0.5, tp, gbp);
                gav = AX(AUX_C, c, r) * tv;
                gbv = 0.5 * tv;
                medadd(AUX_C, c, r, (b2s - b1n) * tv);
            }
            cgy[0 * G::EN + EI(c, r)] = Kc * t;
            cgy[1 * G::EN + EI(c, r)] = gav;
            cgy[2 * G::EN + EI(c, r)] = gbp;
            cgy[3 * G::EN + EI(c, r)] = gbv;
            medadd(AUX_K, c, r, ap * t);
        }
        __syncthreads();

        // ------------------------------------------------------------ 3. correction and limiter
        // Cp = Z_R e2 - Z_L e1, Cu = e1 + e2, e = kappa m, kappa = c - l c^2;
        // m1 = phi(a1, f1 a1(edge+1)), m2 = phi(a2, f2 a2(edge-1)) at the recorded branch
        for (int k = tid; k < (ty + 2) * (tx + 3); k += TNT) {
            const int r = k / (tx + 3) - 1, a = k - (r + 1) * (tx + 3) - 1;
            if (a < 0 || a > tx) {   // edges only the limiter of their neighbour reads
                A1b[XE(a, r)] = 0.0;
                A2b[XE(a, r)] = 0.0;
                continue;
            }
            const bool hasL = a >= 1, hasR = a <= tx - 1;
            double g1 = 0.0, g2 = 0.0, gcp = 0.0, gcu = 0.0;
            if (hasL) {   // cell a-1 holds this edge as its east edge
                g1 = cgx[DI(a - 1, r)] - cgx[G::DN + DI(a - 1, r)];
                gcp = cgx[2 * G::DN + DI(a - 1, r)];
                gcu = cgx[3 * G::DN + DI(a - 1, r)];
            }
            if (hasR) {   // cell a holds it as its west edge
                g2 = cgx[DI(a, r)] + cgx[G::DN + DI(a, r)];
                gcp -= cgx[2 * G::DN + DI(a, r)];
                gcu -= cgx[3 * G::DN + DI(a, r)];
            }
            const double zr = AX(AUX_Z, a, r), zl = AX(AUX_Z, a - 1, r);
            const double cl = AX(AUX_C, a - 1, r), cr = AX(AUX_C, a, r);
            const double kl = fma(-lx, AX(AUX_C2, a - 1, r), cl), kr = fma(-lx, AX(AUX_C2, a, r), cr);
            const double m1 = TP(TAPE_M1, a, r), m2 = TP(TAPE_M2, a, r);
            const double ge2 = fma(zr, gcp, gcu), ge1 = fma(-zl, gcp, gcu);
            const double gm1 = kl * ge1, gm2 = kr * ge2;
            // kappa = c - l c^2: d kappa / dc = 1 - 2 l c (the c^2 plane folded into c)
            medadd(AUX_C, a - 1, r, fma(-2.0 * lx, cl, 1.0) * (m1 * ge1));
            medadd(AUX_C, a, r, fma(-2.0 * lx, cr, 1.0) * (m2 * ge2));
            medadd(AUX_Z, a, r, (kr * m2) * gcp);
            medadd(AUX_Z, a - 1, r, -((kl * m1) * gcp));
            {   // left-going wave: upwind edge a+1
                const double up = TP(TAPE_A1, a + 1, r), f = AX(AUX_FX1, a, r);
                const int code = (int)(__double_as_longlong(m1) & 7);
                double own;
                const double dg = lim_adjoint(code, TP(TAPE_A1, a, r), code == LIMC_SMOOTH ? up * f : 0.0, gm1, g1, own);
                A1b[XE(a, r)] = own;
                U1x[XL(a, r)] = f * dg;   // to edge a+1
                medadd(AUX_FX1, a, r, up * dg);
            }
            {   // right-going wave: upwind edge a-1
                const double up = TP(TAPE_A2, a - 1, r), f = AX(AUX_FX2, a, r);
                const int code = (int)(__double_as_longlong(m2) & 7);
                double own;
                const double dg = lim_adjoint(code, TP(TAPE_A2, a, r), code == LIMC_SMOOTH ? up * f : 0.0, gm2, g2, own);
                A2b[XE(a, r)] = own;
                U2x[XL(a, r)] = f * dg;   // to edge a-1
                medadd(AUX_FX2, a, r, up * dg);
            }
        }
        for (int k = tid; k < (ty + 3) * (tx + 2); k += TNT) {
            const int b = k / (tx + 2) - 1, c = k - (b + 1) * (tx + 2) - 1;
            if (b < 0 || b > ty) {
                B1b[YE(c, b)] = 0.0;
                B2b[YE(c, b)] = 0.0;
                continue;
            }
            const bool hasL = b >= 1, hasR = b <= ty - 1;
            double g1 = 0.0, g2 = 0.0, gcp = 0.0, gcv = 0.0;
            if (hasL) {   // cell (c, b-1) holds this edge as its north edge
                g1 = cgy[EI(c, b - 1)] - cgy[G::EN + EI(c, b - 1)];
                gcp = cgy[2 * G::EN + EI(c, b - 1)];
                gcv = cgy[3 * G::EN + EI(c, b - 1)];
            }
            if (hasR) {
                g2 = cgy[EI(c, b)] + cgy[G::EN + EI(c, b)];
                gcp -= cgy[2 * G::EN + EI(c, b)];
                gcv -= cgy[3 * G::EN + EI(c, b)];
            }
            const double zr = AX(AUX_Z, c, b), zl = AX(AUX_Z, c, b - 1);
            const double cl = AX(AUX_C, c, b - 1), cr = AX(AUX_C, c, b);
            const double kl = fma(-ly, AX(AUX_C2, c, b - 1), cl), kr = fma(-ly, AX(AUX_C2, c, b), cr);
            const double m1 = TP(TAPE_N1, c, b), m2 = TP(TAPE_N2, c, b);
            const double ge2 = fma(zr, gcp, gcv), ge1 = fma(-zl, gcp, gcv);
            const double gm1 = kl * ge1, gm2 = kr * ge2;
            medadd(AUX_C, c, b - 1, fma(-2.0 * ly, cl, 1.0) * (m1 * ge1));
            medadd(AUX_C, c, b, fma(-2.0 * ly, cr, 1.0) * (m2 * ge2));
            medadd(AUX_Z, c, b, (kr * m2) * gcp);
            medadd(AUX_Z, c, b - 1, -((kl * m1) * gcp));
            {
                const double up = TP(TAPE_B1, c, b + 1), f = AX(AUX_FY1, c, b);
                const int code = (int)(__double_as_longlong(m1) & 7);
                double own;
                const double dg = lim_adjoint(code, TP(TAPE_B1, c, b), code == LIMC_SMOOTH ? up * f : 0.0, gm1, g1, own);
                B1b[YE(c, b)] = own;
                U1y[YL(c, b)] = f * dg;   // to edge b+1
                medadd(AUX_FY1, c, b, up * dg);
            }
            {
                const double up = TP(TAPE_B2, c, b - 1), f = AX(AUX_FY2, c, b);
                const int code = (int)(__double_as_longlong(m2) & 7);
                double own;
                const double dg = lim_adjoint(code, TP(TAPE_B2, c, b), code == LIMC_SMOOTH ? up * f : 0.0, gm2, g2, own);
                B2b[YE(c, b)] = own;
                U2y[YL(c, b)] = f * dg;   // to edge b-1
                medadd(AUX_FY2, c, b, up * dg);
            }
        }
        __syncthreads();

        // ------------------------------------------------------------ 4. normal Riemann solves
        // a1 = is (Z_R du - dp), a2 = is (Z_L du + dp): the adjoints of the edge's jumps dp, du
        // replace those of a1, a2 in the edge's slots
        for (int k = tid; k < (ty + 2) * (tx + 3); k += TNT) {
            const int r = k / (tx + 3) - 1, a = k - (r + 1) * (tx + 3) - 1;
            double g1 = A1b[XE(a, r)], g2 = A2b[XE(a, r)];
            if (a - 1 >= 0 && a - 1 <= tx) g1 += U1x[XL(a - 1, r)];
            if (a + 1 >= 0 && a + 1 <= tx) g2 += U2x[XL(a + 1, r)];
            if (!nonzero(g1) && !nonzero(g2)) {
                A1b[XE(a, r)] = 0.0;
                A2b[XE(a, r)] = 0.0;
                continue;
            }
            const double is = AX(AUX_IXS, a, r), zr = AX(AUX_Z, a, r), zl = AX(AUX_Z, a - 1, r);
            const double gn1 = is * g1, gn2 = is * g2;
            A1b[XE(a, r)] = gn2 - gn1;                // adjoint of dp = p_a - p_{a-1}
            A2b[XE(a, r)] = fma(zr, gn1, zl * gn2);   // adjoint of du
            const double a1 = TP(TAPE_A1, a, r), a2 = TP(TAPE_A2, a, r);
            const double du = a1 + a2;                // is (Z_L + Z_R) du
            medadd(AUX_Z, a, r, du * gn1);
            medadd(AUX_Z, a - 1, r, du * gn2);
            medadd(AUX_IXS, a, r, fma(a1, g1, a2 * g2));   // is x the adjoint of is
        }
        for (int k = tid; k < (ty + 3) * (tx + 2); k += TNT) {
            const int b = k / (tx + 2) - 1, c = k - (b + 1) * (tx + 2) - 1;
            double g1 = B1b[YE(c, b)], g2 = B2b[YE(c, b)];
            if (b - 1 >= 0 && b - 1 <= ty) g1 += U1y[YL(c, b - 1)];
            if (b + 1 >= 0 && b + 1 <= ty) g2 += U2y[YL(c, b + 1)];
            if (!nonzero(g1) && !nonzero(g2)) {
                B1b[YE(c, b)] = 0.0;
                B2b[YE(c, b)] = 0.0;
                continue;
            }
            const double is = AX(AUX_IYS, c, b), zr = AX(AUX_Z, c, b), zl = AX(AUX_Z, c, b - 1);
            const double gn1 = is * g1, gn2 = is * g2;
            B1b[YE(c, b)] = gn2 - gn1;
            B2b[YE(c, b)] = fma(zr, gn1, zl * gn2);
            const double b1 = TP(TAPE_B1, c, b), b2 = TP(TAPE_B2, c, b);
            const double dv = b1 + b2;
            medadd(AUX_Z, c, b, dv * gn1);
            medadd(AUX_Z, c, b - 1, dv * gn2);
            medadd(AUX_IYS, c, b, fma(b1, g1, b2 * g2));
        }
        __syncthreads();

        // ------------------------------------------------------------ 5. flush to lam_old
        {
            auto gx = [&](const double* arr, int a, int r) -> double {
                return (a >= -1 && a <= tx + 1 && r >= -1 && r <= ty) ? arr[XE(a, r)] : 0.0;
            };
            auto gy = [&](const double* arr, int c, int b) -> double {
                return (b >= -1 && b <= ty + 1 && c >= -1 && c <= tx) ? arr[YE(c, b)] : 0.0;
            };
            double* lo = lam_old + P.qoff;
            const int w4 = tx + 4, n4 = w4 * (ty + 4);
            for (int k = tid; k < n4; k += TNT) {
                const int j = k / w4 - 2, i = k - (j + 2) * w4 - 2;
                double p = gx(A1b, i, j) - gx(A1b, i + 1, j) + gy(B1b, i, j) - gy(B1b, i, j + 1);
                double u = gx(A2b, i, j) - gx(A2b, i + 1, j);
                double v = gy(B2b, i, j) - gy(B2b, i, j + 1);
                if (i >= 0 && i < tx && j >= 0 && j < ty) {   // the identity part of the update
                    p += LAM(0, i, j);
                    u += LAM(1, i, j);
                    v += LAM(2, i, j);
                }
                const int bx = x0 + i, by = y0 + j;
                if (A.ring && P.ring >= 0 && (bx < 0 || bx >= P.nx || by < 0 || by >= P.ny)) {
                    // a ghost the forward pulled from a cell of the level: its adjoint goes there
                    const longlong2 e = A.ring[P.ring + ring_index(bx + 2, by + 2, P.nx, P.ny)];
                    if (e.x >= 0) {
                        const long long pl = e.y & ((1LL << kRingFlagShift) - 1);
                        const int fl = (int)(e.y >> kRingFlagShift);
                        if (nonzero(p)) atomicAdd(lam_old + e.x, p);
                        if (nonzero(u)) atomicAdd(lam_old + e.x + pl, flip_sign(u, fl & 1));
                        if (nonzero(v)) atomicAdd(lam_old + e.x + 2 * pl, flip_sign(v, (fl >> 1) & 1));
                        continue;
                    }
                }
                const long long o = cell(i, j);
                if (nonzero(p)) atomicAdd(lo + o, p);
                if (nonzero(u)) atomicAdd(lo + WH + o, u);
                if (nonzero(v)) atomicAdd(lo + 2 * WH + o, v);
            }
        }
        __syncthreads();   // shared memory is reused by the next tile
    }
}

void (*tape_kernel(int limiter))(const StepArgs, const double*, double*, double*)
{
    switch (limiter) {
    case CLAW_LIM_NONE: return step_adjoint_tape_kernel<CLAW_LIM_NONE>;
    case CLAW_LIM_MINMOD: return step_adjoint_tape_kernel<CLAW_LIM_MINMOD>;
    case CLAW_LIM_SUPERBEE: return step_adjoint_tape_kernel<CLAW_LIM_SUPERBEE>;
    case CLAW_LIM_VANLEER: return step_adjoint_tape_kernel<CLAW_LIM_VANLEER>;
    case CLAW_LIM_MC: return step_adjoint_tape_kernel<CLAW_LIM_MC>;
    }
    return nullptr;
}

}  // namespace

int adjoint_tape_tile() { return TTX; }

cudaError_t launch_step_adjoint_tape(const StepArgs& a, const double* lam_new, double* lam_old, double* g_aux,
                                     int limiter, int nsm, cudaStream_t s)
{
    constexpr int kDev = 64;
    static int cached[kDev][5] = {};
    void (*fn)(const StepArgs, const double*, double*, double*) = tape_kernel(limiter);
    if (!fn || limiter < 0 || limiter > 4) return cudaErrorInvalidValue;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kDev) return cudaErrorInvalidDevice;
    const size_t smem = TGeo::smem_bytes();
    int& per_sm = cached[dev][limiter];
    if (!per_sm) {
        e = cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int n = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, TNT, smem);
        if (e != cudaSuccess) return e;
        per_sm = n > 0 ? n : 1;
    }
    const int grid = a.ntiles < per_sm * nsm ? a.ntiles : per_sm * nsm;
    if (grid <= 0) return cudaSuccess;
    fn<<<grid, TNT, smem, s>>>(a, lam_new, lam_old, g_aux);
    return cudaGetLastError();
}

}  // namespace claw

// claw_adjoint.cu -- reverse mode of the fused level-step (the discrete adjoint of the
// cell-wise formulation of claw_step.cuh, dt frozen).
//
// Per tile the kernel re-runs the forward phases (normal Riemann strengths, limited strengths,
// corrections, transverse pressures) from q_old to recover every intermediate and every limiter
// branch, then walks the phases backwards:
//   update -> transverse fluxes -> per-cell terms -> edge gathers -> limiter / correction ->
//   normal Riemann -> q_old and the medium planes.
// Each reverse phase is a gather where it can be (every adjoint written by one thread): the
// wave-strength and state adjoints are stored per edge and summed per cell by the thread of
// the cell (a shared-memory FP64 atomic costs an FP64-pipe slot on this part, like a DFMA).
// The medium adjoints (per cell: Z, c, K; per edge: 1/(Z_L+Z_R), as that value times its
// adjoint, and the limiter projection factors) go straight to g_aux with global FP64 reductions, which the L2 carries out, not
// the FP64 pipe; the chain rule of the edge planes to Z runs once per gradient in
// claw_medium_aux_adjoint, not once per step.  Zero tests of doubles are integer tests (a
// double compare is an FP64-pipe instruction).  The c^2 plane is folded
// into c where it is read.  Contributions to cells shared with neighbouring tiles (the two
// ghost layers) reach lam_old / g_aux through global FP64 atomics.  Given the level's ghost ring
// (A.ring), the contributions to the box's own ghost cells that the forward filled from cells of
// the level go straight to those cells (the adjoint of the ghost copy, fused).  A uniform medium
// runs the same code with constant medium planes and no medium adjoint.
#include <cuda_runtime.h>

#include "claw_step.cuh"

namespace claw {
namespace {

// phi(b/a) a and its partial derivatives along the branch the forward (claw_step.cuh) takes
template <int L> struct LimD;
template <> struct LimD<CLAW_LIM_NONE> {
    static __device__ __forceinline__ double f(double a, double, double& da, double& db)
    {
        da = 1.0;
        db = 0.0;
        return a;
    }
};
template <> struct LimD<CLAW_LIM_MINMOD> {
    static __device__ __forceinline__ double f(double a, double b, double& da, double& db)
    {
        using namespace lim_bits;
        const long long ia = bits(a), ib = bits(b), ma = ia & MAG, mb = ib & MAG;
        da = db = 0.0;
        if (!same_sign_nonzero(ia, ib, ma, mb)) return 0.0;
        if (ma < mb) { da = 1.0; return a; }
        db = 1.0;
        return b;
    }
};
template <> struct LimD<CLAW_LIM_SUPERBEE> {
    static __device__ __forceinline__ double f(double a, double b, double& da, double& db)
    {
        using namespace lim_bits;
        const long long ia = bits(a), ib = bits(b), ma = ia & MAG, mb = ib & MAG;
        da = db = 0.0;
        if (!same_sign_nonzero(ia, ib, ma, mb)) return 0.0;
        const long long a2 = ma + ONE_EXP, b2 = mb + ONE_EXP;
        const bool first_a = ma < b2;    // min(|a|, 2|b|)
        const bool second_a2 = a2 < mb;  // min(2|a|, |b|)
        const long long m1 = first_a ? ma : b2, m2 = second_a2 ? a2 : mb;
        if (m1 > m2) {
            if (first_a) { da = 1.0; return a; }
            db = 2.0;
            return val(b2 | (ia & SIGN));
        }
        if (second_a2) { da = 2.0; return val(a2 | (ia & SIGN)); }
        db = 1.0;
        return b;
    }
};
template <> struct LimD<CLAW_LIM_VANLEER> {
    static __device__ __forceinline__ double f(double a, double b, double& da, double& db)
    {
        da = db = 0.0;
        if (!(a * b > 0.0)) return 0.0;
        const double s = a + b, is2 = 1.0 / (s * s);
        da = 2.0 * b * b * is2;
        db = 2.0 * a * a * is2;
        return (2.0 * a * b) / s;
    }
};
template <> struct LimD<CLAW_LIM_MC> {
    static __device__ __forceinline__ double f(double a, double b, double& da, double& db)
    {
        using namespace lim_bits;
        const long long ia = bits(a), ib = bits(b), ma = ia & MAG, mb = ib & MAG;
        da = db = 0.0;
        if (!same_sign_nonzero(ia, ib, ma, mb)) return 0.0;
        const bool amin = ma < mb;
        const long long t2 = (amin ? ma : mb) + ONE_EXP;
        long long sh = bits(val(ma) + val(mb)) - ONE_EXP;
        sh = sh > 0 ? sh : 0;
        if (sh < t2) {
            da = db = 0.5;
            return val(sh | (ia & SIGN));
        }
        if (amin) da = 2.0;
        else db = 2.0;
        return val(t2 | (ia & SIGN));
    }
};

constexpr int ATX = 16, ATY = 16, ANT = 384;

// x != 0 on the integer pipe (+0 and -0 are zero)
__device__ __forceinline__ bool nonzero(double x)
{
    return ((unsigned long long)__double_as_longlong(x) << 1) != 0ull;
}
// x with its sign flipped when f is 1 (a sign-bit xor, not an FP64 negation)
__device__ __forceinline__ double flip_sign(double x, int f)
{
    return __longlong_as_double(__double_as_longlong(x) ^ ((long long)(f & 1) << 63));
}

struct AGeo {
    static constexpr int SW = ATX + 4, SH = ATY + 4, QPL = SW * SH;
    static constexpr int XEW = ATX + 3, XEH = ATY + 2, XE = XEW * XEH;
    static constexpr int YEW = ATX + 2, YEH = ATY + 3, YE = YEW * YEH;
    static constexpr int XLW = ATX + 1, XLH = ATY + 2, XL = XLW * XLH;
    static constexpr int YLW = ATX + 2, YLH = ATY + 1, YL = YLW * YLH;
    static constexpr int DW = ATX, DH = ATY + 2, DN = DW * DH;
    static constexpr int EW = ATX + 2, EH = ATY, EN = EW * EH;
    static constexpr int FN = (ATX + 1) * ATY, GN = ATX * (ATY + 1);
    // shared-memory carve (doubles)
    static constexpr int O_Q = 0;                       // p, u, v
    static constexpr int O_A1 = O_Q + 3 * QPL;
    static constexpr int O_A2 = O_A1 + XE;
    static constexpr int O_B1 = O_A2 + XE;
    static constexpr int O_B2 = O_B1 + YE;
    static constexpr int O_A1B = O_B2 + YE;             // wave-strength adjoints, then the per-edge
    static constexpr int O_A2B = O_A1B + XE;            // state adjoints of the normal solver
    static constexpr int O_B1B = O_A2B + XE;
    static constexpr int O_B2B = O_B1B + YE;
    static constexpr int O_M1X = O_B2B + YE;            // limited strengths, then the limiter's
                                                        // contributions to the upwind edge's adjoint
    static constexpr int O_M2X = O_M1X + XL;
    static constexpr int O_M1Y = O_M2X + XL;
    static constexpr int O_M2Y = O_M1Y + YL;
    static constexpr int O_CPX = O_M2Y + YL;            // corrections (forward), then their adjoints
    static constexpr int O_CUX = O_CPX + XL;
    static constexpr int O_CPY = O_CUX + XL;
    static constexpr int O_CVY = O_CPY + YL;
    static constexpr int O_D = O_CVY + YL;
    static constexpr int O_E = O_D + DN;
    static constexpr int O_DB = O_E + EN;
    static constexpr int O_EB = O_DB + DN;
    static constexpr int O_APX = O_EB + EN;             // per-cell adjoints of ap, au, bp, bu (x)
    static constexpr int O_AUX = O_APX + DN;
    static constexpr int O_BPX = O_AUX + DN;
    static constexpr int O_BUX = O_BPX + DN;
    static constexpr int O_APY = O_BUX + DN;            // (y)
    static constexpr int O_AVY = O_APY + EN;
    static constexpr int O_BPY = O_AVY + EN;
    static constexpr int O_BVY = O_BPY + EN;
    static constexpr int O_FB = O_BVY + EN;             // adjoints of Fp, Fu, Gp, Gv
    static constexpr int O_GB = O_FB + 2 * FN;
    static constexpr int O_END = O_GB + 2 * GN;
    static size_t smem_bytes(int) { return (size_t)O_END * 8; }
};
static_assert(AUX_Z == 0 && AUX_C == 1 && AUX_K == 2, "medium adjoint planes are the first three aux planes");

template <int MED, int LIM>
__global__ void __launch_bounds__(ANT, 2)
    step_adjoint_kernel(const StepArgs A, const double* __restrict__ lam_new, double* __restrict__ lam_old,
                        double* __restrict__ g_aux)
{
    using G = AGeo;
    extern __shared__ __align__(128) double sm[];
    double* sp = sm + G::O_Q;
    double* su = sp + G::QPL;
    double* sv = su + G::QPL;
    double* A1 = sm + G::O_A1;
    double* A2 = sm + G::O_A2;
    double* B1 = sm + G::O_B1;
    double* B2 = sm + G::O_B2;
    double* A1b = sm + G::O_A1B;
    double* A2b = sm + G::O_A2B;
    double* B1b = sm + G::O_B1B;
    double* B2b = sm + G::O_B2B;
    double* M1x = sm + G::O_M1X;
    double* M2x = sm + G::O_M2X;
    double* M1y = sm + G::O_M1Y;
    double* M2y = sm + G::O_M2Y;
    double* Cpx = sm + G::O_CPX;
    double* Cux = sm + G::O_CUX;
    double* Cpy = sm + G::O_CPY;
    double* Cvy = sm + G::O_CVY;
    double* Dx = sm + G::O_D;
    double* Ey = sm + G::O_E;
    double* Db = sm + G::O_DB;
    double* Eb = sm + G::O_EB;
    double* apxb = sm + G::O_APX;
    double* auxb = sm + G::O_AUX;
    double* bpxb = sm + G::O_BPX;
    double* buxb = sm + G::O_BUX;
    double* apyb = sm + G::O_APY;
    double* avyb = sm + G::O_AVY;
    double* bpyb = sm + G::O_BPY;
    double* bvyb = sm + G::O_BVY;
    double* Fpb = sm + G::O_FB;
    double* Fub = Fpb + G::FN;
    double* Gpb = sm + G::O_GB;
    double* Gvb = Gpb + G::GN;

    const int tid = threadIdx.x;
    const bool second = A.order == 2;
    const bool trans = A.transverse != 0;
    const double w = (A.transverse == 2 && A.order == 2) ? 1.0 : 0.0;
    double Z0 = 0, c0 = 0, iZs = 0;
    if (MED == 0) {
        Z0 = sqrt(A.K0 * A.rho0);
        c0 = sqrt(A.K0 / A.rho0);
        iZs = 1.0 / (Z0 + Z0);
    }

    for (int t = blockIdx.x; t < A.ntiles; t += gridDim.x) {
        const TileDev T = A.tiles[t];
        const PatchDev P = A.patches[T.patch];
        const int tx = T.tx, ty = T.ty, x0 = T.x0, y0 = T.y0;
        const int W = P.nx + 4;
        const long long WH = (long long)W * (P.ny + 4);
        const double dt = __ldg(A.dt + P.run) * P.dtscale;
        const double lx = dt * P.dxinv, ly = dt * P.dyinv;
        const double* aux = MED ? A.aux + P.aoff : nullptr;
        // medium plane k of tile-local cell (i, j): aux planes, or the uniform medium's values
        auto AX = [&](int k, int i, int j) -> double {
            if (MED) return __ldg(aux + k * WH + (long long)(y0 + j + 2) * W + (x0 + i + 2));
            switch (k) {
            case AUX_Z: return Z0;
            case AUX_C: return c0;
            case AUX_K: return A.K0;
            case AUX_C2: return c0 * c0;
            case AUX_IXS: case AUX_IYS: return iZs;
            default: return 1.0;
            }
        };
        auto CI = [](int i, int j) { return (i + 2) + (j + 2) * G::SW; };
        auto XE = [](int a, int r) { return (a + 1) + (r + 1) * G::XEW; };
        auto YE = [](int c, int b) { return (c + 1) + (b + 1) * G::YEW; };
        auto XL = [](int a, int r) { return a + (r + 1) * G::XLW; };
        auto YL = [](int c, int b) { return (c + 1) + b * G::YLW; };
        auto DI = [](int c, int r) { return c + (r + 1) * G::DW; };
        auto EI = [](int c, int r) { return (c + 1) + r * G::EW; };
        // adjoint of medium plane k at tile-local cell (i, j): a cell plane (AUX_Z, AUX_C, AUX_K)
        // or an edge plane (held at the edge's east / north cell); a global reduction
        double* gmed = (MED && g_aux) ? g_aux + P.aoff : nullptr;
        auto medadd = [&](int k, int i, int j, double v) {
            if (MED && nonzero(v)) atomicAdd(gmed + k * WH + (long long)(y0 + j + 2) * W + (x0 + i + 2), v);
        };
        auto edgeadd = medadd;

        // ---------------------------------------------------------------- stage, clear
        {
            const double* src = A.qold + P.qoff;
            for (int k = tid; k < 3 * G::QPL; k += ANT) {
                const int m = k / G::QPL, rem = k - m * G::QPL;
                const int jj = rem / G::SW, ii = rem - jj * G::SW;
                double v = 0.0;
                if (ii < tx + 4 && jj < ty + 4) v = __ldg(src + m * WH + (long long)(y0 + jj) * W + (x0 + ii));
                sm[G::O_Q + k] = v;
            }
            // accumulators only: every other work array is written before it is read
            for (int k = tid; k < G::O_M1X - G::O_A1B; k += ANT) sm[G::O_A1B + k] = 0.0;
        }
        __syncthreads();
        if (A.ring && P.ring >= 0) {   // the ghosts the forward step pulled from their source cells
            pull_ghosts<G::SW, G::QPL, ANT>(A, P, sp, x0, y0, tx, ty);
            __syncthreads();
        }

        // ---------------------------------------------------------------- forward recompute
        for (int k = tid; k < (ty + 2) * (tx + 3); k += ANT) {
            const int r = k / (tx + 3) - 1, a = k % (tx + 3) - 1;
            const int iR = CI(a, r);
            const double dp = sp[iR] - sp[iR - 1], du = su[iR] - su[iR - 1];
            const double zr = AX(AUX_Z, a, r), zl = AX(AUX_Z, a - 1, r), is = AX(AUX_IXS, a, r);
            A1[XE(a, r)] = fma(zr, du, -dp) * is;
            A2[XE(a, r)] = fma(zl, du, dp) * is;
        }
        for (int k = tid; k < (ty + 3) * (tx + 2); k += ANT) {
            const int b = k / (tx + 2) - 1, c = k % (tx + 2) - 1;
            const int iR = CI(c, b);
            const double dp = sp[iR] - sp[iR - G::SW], dv = sv[iR] - sv[iR - G::SW];
            const double zr = AX(AUX_Z, c, b), zl = AX(AUX_Z, c, b - 1), is = AX(AUX_IYS, c, b);
            B1[YE(c, b)] = fma(zr, dv, -dp) * is;
            B2[YE(c, b)] = fma(zl, dv, dp) * is;
        }
        __syncthreads();
        if (second) {
            for (int k = tid; k < (ty + 2) * (tx + 1); k += ANT) {
                const int r = k / (tx + 1) - 1, a = k % (tx + 1);
                double da, db;
                const double m1 = LimD<LIM>::f(A1[XE(a, r)], A1[XE(a + 1, r)] * AX(AUX_FX1, a, r), da, db);
                const double m2 = LimD<LIM>::f(A2[XE(a, r)], A2[XE(a - 1, r)] * AX(AUX_FX2, a, r), da, db);
                const double kl = fma(-lx, AX(AUX_C2, a - 1, r), AX(AUX_C, a - 1, r));
                const double kr = fma(-lx, AX(AUX_C2, a, r), AX(AUX_C, a, r));
                const double e1 = kl * m1, e2 = kr * m2;
                M1x[XL(a, r)] = m1;
                M2x[XL(a, r)] = m2;
                Cpx[XL(a, r)] = fma(AX(AUX_Z, a, r), e2, -(AX(AUX_Z, a - 1, r) * e1));
                Cux[XL(a, r)] = e1 + e2;
            }
            for (int k = tid; k < (ty + 1) * (tx + 2); k += ANT) {
                const int b = k / (tx + 2), c = k % (tx + 2) - 1;
                double da, db;
                const double m1 = LimD<LIM>::f(B1[YE(c, b)], B1[YE(c, b + 1)] * AX(AUX_FY1, c, b), da, db);
                const double m2 = LimD<LIM>::f(B2[YE(c, b)], B2[YE(c, b - 1)] * AX(AUX_FY2, c, b), da, db);
                const double kl = fma(-ly, AX(AUX_C2, c, b - 1), AX(AUX_C, c, b - 1));
                const double kr = fma(-ly, AX(AUX_C2, c, b), AX(AUX_C, c, b));
                const double e1 = kl * m1, e2 = kr * m2;
                M1y[YL(c, b)] = m1;
                M2y[YL(c, b)] = m2;
                Cpy[YL(c, b)] = fma(AX(AUX_Z, c, b), e2, -(AX(AUX_Z, c, b - 1) * e1));
                Cvy[YL(c, b)] = e1 + e2;
            }
            __syncthreads();
        }
        if (trans) {
            for (int k = tid; k < (ty + 2) * tx; k += ANT) {   // D: cols [0,tx), rows [-1,ty]
                const int r = k / tx - 1, c = k % tx;
                const double ap = A2[XE(c, r)] + A1[XE(c + 1, r)];
                const double bp = second ? Cpx[XL(c + 1, r)] - Cpx[XL(c, r)] : 0.0;
                Dx[DI(c, r)] = fma(AX(AUX_K, c, r), ap, w * bp);
            }
            for (int k = tid; k < ty * (tx + 2); k += ANT) {   // E: cols [-1,tx], rows [0,ty)
                const int r = k / (tx + 2), c = k % (tx + 2) - 1;
                const double ap = B2[YE(c, r)] + B1[YE(c, r + 1)];
                const double bp = second ? Cpy[YL(c, r + 1)] - Cpy[YL(c, r)] : 0.0;
                Ey[EI(c, r)] = fma(AX(AUX_K, c, r), ap, w * bp);
            }
        }
        __syncthreads();

        // ---------------------------------------------------------------- reverse: update
        // p_new = p + dP - lx (Fp_e - Fp_w) - ly (Gp_n - Gp_s), u_new, v_new likewise
        const double* ln = lam_new + P.qoff;
        auto LAM = [&](int m, int c, int r) -> double {
            if (c < 0 || c >= tx || r < 0 || r >= ty) return 0.0;
            return __ldg(ln + m * WH + (long long)(y0 + r + 2) * W + (x0 + c + 2));
        };
        if (trans) {
            for (int k = tid; k < ty * (tx + 1); k += ANT) {   // x-edge a of row r
                const int r = k / (tx + 1), a = k % (tx + 1);
                Fpb[a + r * (ATX + 1)] = lx * (LAM(0, a, r) - LAM(0, a - 1, r));
                Fub[a + r * (ATX + 1)] = lx * (LAM(1, a, r) - LAM(1, a - 1, r));
            }
            for (int k = tid; k < (ty + 1) * tx; k += ANT) {   // y-edge jj of column c
                const int jj = k / tx, c = k % tx;
                Gpb[c + jj * ATX] = ly * (LAM(0, c, jj) - LAM(0, c, jj - 1));
                Gvb[c + jj * ATX] = ly * (LAM(2, c, jj) - LAM(2, c, jj - 1));
            }
        }
        __syncthreads();

        // ---------------------------------------------------------------- reverse: transverse fluxes
        // Gp = wG (K_hi D_lo - K_lo D_hi), Gv = wG (c_hi D_lo + c_lo D_hi), wG = -lx/2 iys_hi
        if (trans) {
            for (int k = tid; k < (ty + 2) * tx; k += ANT) {   // D-bar of cell (c, r), r in [-1, ty]
                const int r = k / tx - 1, c = k % tx;
                double acc = 0.0;
                const double Kc = AX(AUX_K, c, r), cc = AX(AUX_C, c, r);
                if (r + 1 <= ty) {   // this cell is "lo" of y-edge r+1
                    const int jj = r + 1;
                    const double is = AX(AUX_IYS, c, jj), wG = -0.5 * lx * is;
                    const double gp = Gpb[c + jj * ATX], gv = Gvb[c + jj * ATX];
                    const double khi = AX(AUX_K, c, jj), chi = AX(AUX_C, c, jj);
                    acc += wG * (khi * gp + chi * gv);
                    const double dhi = Dx[DI(c, jj)];
                    // medium: K_lo, c_lo of this cell; K_hi, c_hi, iys of the hi cell
                    medadd(AUX_K, c, r, -wG * dhi * gp);
                    medadd(AUX_C, c, r, wG * dhi * gv);
                }
                if (r >= 0) {        // this cell is "hi" of y-edge r
                    const int jj = r;
                    const double is = AX(AUX_IYS, c, jj), wG = -0.5 * lx * is;
                    const double gp = Gpb[c + jj * ATX], gv = Gvb[c + jj * ATX];
                    const double klo = AX(AUX_K, c, jj - 1), clo = AX(AUX_C, c, jj - 1);
                    acc += wG * (-klo * gp + clo * gv);
                    const double dlo = Dx[DI(c, jj - 1)], dme = Dx[DI(c, jj)];
                    medadd(AUX_K, c, r, wG * dlo * gp);
                    medadd(AUX_C, c, r, wG * dlo * gv);
                    const double gpf = fma(Kc, dlo, -(klo * dme)), gvf = fma(cc, dlo, clo * dme);
                    edgeadd(AUX_IYS, c, r, wG * fma(gpf, gp, gvf * gv));   // is x its adjoint
                }
                Db[DI(c, r)] = acc;
            }
            for (int k = tid; k < ty * (tx + 2); k += ANT) {   // E-bar of cell (c, r), c in [-1, tx]
                const int r = k / (tx + 2), c = k % (tx + 2) - 1;
                double acc = 0.0;
                const double Kc = AX(AUX_K, c, r), cc = AX(AUX_C, c, r);
                if (c + 1 <= tx) {   // "lo" of x-edge c+1
                    const int a = c + 1;
                    const double is = AX(AUX_IXS, a, r), wF = -0.5 * ly * is;
                    const double fp = Fpb[a + r * (ATX + 1)], fu = Fub[a + r * (ATX + 1)];
                    const double khi = AX(AUX_K, a, r), chi = AX(AUX_C, a, r);
                    acc += wF * (khi * fp + chi * fu);
                    const double ehi = Ey[EI(a, r)];
                    medadd(AUX_K, c, r, -wF * ehi * fp);
                    medadd(AUX_C, c, r, wF * ehi * fu);
                }
                if (c >= 0) {        // "hi" of x-edge c
                    const int a = c;
                    const double is = AX(AUX_IXS, a, r), wF = -0.5 * ly * is;
                    const double fp = Fpb[a + r * (ATX + 1)], fu = Fub[a + r * (ATX + 1)];
                    const double klo = AX(AUX_K, a - 1, r), clo = AX(AUX_C, a - 1, r);
                    acc += wF * (-klo * fp + clo * fu);
                    const double elo = Ey[EI(a - 1, r)], eme = Ey[EI(a, r)];
                    medadd(AUX_K, c, r, wF * elo * fp);
                    medadd(AUX_C, c, r, wF * elo * fu);
                    const double fpf = fma(Kc, elo, -(klo * eme)), fuf = fma(cc, elo, clo * eme);
                    edgeadd(AUX_IXS, c, r, wF * fma(fpf, fp, fuf * fu));
                }
                Eb[EI(c, r)] = acc;
            }
        }
        __syncthreads();

        // ---------------------------------------------------------------- reverse: per-cell terms
        // D = K ap + w bp ; interior: dP = -lx (K ap + bp/2) - ly (K apy + bpy/2),
        // dU = -lx (c au + bu/2), dV = -ly (c avy + bvy/2)
        for (int k = tid; k < (ty + 2) * tx; k += ANT) {
            const int r = k / tx - 1, c = k % tx;
            const double Kc = AX(AUX_K, c, r), cc = AX(AUX_C, c, r);
            const double ap = A2[XE(c, r)] + A1[XE(c + 1, r)];
            const double au = A2[XE(c, r)] - A1[XE(c + 1, r)];
            const double db = trans ? Db[DI(c, r)] : 0.0;
            double gap = Kc * db, gbp = w * db, gau = 0.0, gbu = 0.0, gK = ap * db, gc = 0.0;
            if (r >= 0 && r < ty) {
                const double tp = -lx * LAM(0, c, r), tu = -lx * LAM(1, c, r);
                gap += Kc * tp;
                gbp += 0.5 * tp;
                gK += ap * tp;
                gau = cc * tu;
                gbu = 0.5 * tu;
                gc = au * tu;
            }
            apxb[DI(c, r)] = gap;
            auxb[DI(c, r)] = gau;
            bpxb[DI(c, r)] = gbp;
            buxb[DI(c, r)] = gbu;
            medadd(AUX_K, c, r, gK);
            medadd(AUX_C, c, r, gc);
        }
        for (int k = tid; k < ty * (tx + 2); k += ANT) {
            const int r = k / (tx + 2), c = k % (tx + 2) - 1;
            const double Kc = AX(AUX_K, c, r), cc = AX(AUX_C, c, r);
            const double ap = B2[YE(c, r)] + B1[YE(c, r + 1)];
            const double av = B2[YE(c, r)] - B1[YE(c, r + 1)];
            const double eb = trans ? Eb[EI(c, r)] : 0.0;
            double gap = Kc * eb, gbp = w * eb, gav = 0.0, gbv = 0.0, gK = ap * eb, gc = 0.0;
            if (c >= 0 && c < tx) {
                const double tp = -ly * LAM(0, c, r), tv = -ly * LAM(2, c, r);
                gap += Kc * tp;
                gbp += 0.5 * tp;
                gK += ap * tp;
                gav = cc * tv;
                gbv = 0.5 * tv;
                gc = av * tv;
            }
            apyb[EI(c, r)] = gap;
            avyb[EI(c, r)] = gav;
            bpyb[EI(c, r)] = gbp;
            bvyb[EI(c, r)] = gbv;
            medadd(AUX_K, c, r, gK);
            medadd(AUX_C, c, r, gc);
        }
        __syncthreads();

        // ---------------------------------------------------------------- reverse: edge gathers
        // ap(cell c) = A2[c] + A1[c+1], au = A2[c] - A1[c+1]; bp = C[c+1] - C[c]
        for (int k = tid; k < (ty + 2) * (tx + 1); k += ANT) {   // x-edges a in [0, tx]
            const int r = k / (tx + 1) - 1, a = k % (tx + 1);
            double g1 = 0.0, g2 = 0.0, gcp = 0.0, gcu = 0.0;
            if (a - 1 >= 0) {   // cell a-1 holds this edge as its east edge (A1)
                g1 += apxb[DI(a - 1, r)] - auxb[DI(a - 1, r)];
                gcp += bpxb[DI(a - 1, r)];
                gcu += buxb[DI(a - 1, r)];
            }
            if (a < tx) {       // cell a holds it as its west edge (A2)
                g2 += apxb[DI(a, r)] + auxb[DI(a, r)];
                gcp -= bpxb[DI(a, r)];
                gcu -= buxb[DI(a, r)];
            }
            A1b[XE(a, r)] = g1;
            A2b[XE(a, r)] = g2;
            Cpx[XL(a, r)] = gcp;   // the forward corrections are dead: reuse for their adjoints
            Cux[XL(a, r)] = gcu;
        }
        for (int k = tid; k < (ty + 1) * (tx + 2); k += ANT) {   // y-edges b in [0, ty]
            const int b = k / (tx + 2), c = k % (tx + 2) - 1;
            double g1 = 0.0, g2 = 0.0, gcp = 0.0, gcv = 0.0;
            if (b - 1 >= 0) {
                g1 += apyb[EI(c, b - 1)] - avyb[EI(c, b - 1)];
                gcp += bpyb[EI(c, b - 1)];
                gcv += bvyb[EI(c, b - 1)];
            }
            if (b < ty) {
                g2 += apyb[EI(c, b)] + avyb[EI(c, b)];
                gcp -= bpyb[EI(c, b)];
                gcv -= bvyb[EI(c, b)];
            }
            B1b[YE(c, b)] = g1;
            B2b[YE(c, b)] = g2;
            Cpy[YL(c, b)] = gcp;
            Cvy[YL(c, b)] = gcv;
        }
        __syncthreads();

        // ---------------------------------------------------------------- reverse: limiter, correction
        // Cp = Z_R e2 - Z_L e1, Cu = e1 + e2, e = kappa m, kappa = c - l c^2,
        // m1 = lim(A1[a], A1[a+1] f1), m2 = lim(A2[a], A2[a-1] f2)
        if (second) {
            for (int k = tid; k < (ty + 2) * (tx + 1); k += ANT) {
                const int r = k / (tx + 1) - 1, a = k % (tx + 1);
                const double gcp = Cpx[XL(a, r)], gcu = Cux[XL(a, r)];
                const double zr = AX(AUX_Z, a, r), zl = AX(AUX_Z, a - 1, r);
                const double kl = fma(-lx, AX(AUX_C2, a - 1, r), AX(AUX_C, a - 1, r));
                const double kr = fma(-lx, AX(AUX_C2, a, r), AX(AUX_C, a, r));
                const double m1 = M1x[XL(a, r)], m2 = M2x[XL(a, r)];
                const double ge2 = fma(zr, gcp, gcu), ge1 = fma(-zl, gcp, gcu);
                const double gkl = m1 * ge1, gkr = m2 * ge2;
                // kappa = c - l c^2: d kappa / dc = 1 - 2 l c (the c^2 plane folded into c)
                if (MED) {
                    medadd(AUX_C, a - 1, r, gkl * fma(-2.0 * lx, AX(AUX_C, a - 1, r), 1.0));
                    medadd(AUX_C, a, r, gkr * fma(-2.0 * lx, AX(AUX_C, a, r), 1.0));
                }
                const double gm1 = kl * ge1, gm2 = kr * ge2;
                const double f1 = AX(AUX_FX1, a, r), f2 = AX(AUX_FX2, a, r);
                const double up1 = A1[XE(a + 1, r)], up2 = A2[XE(a - 1, r)];
                double da, db;
                // own edge: plain update (only this thread touches the slot here); the upwind
                // edge's share goes to this edge's M slot (read above, dead now) for a gather
                LimD<LIM>::f(A1[XE(a, r)], up1 * f1, da, db);
                A1b[XE(a, r)] += da * gm1;
                const double dg1 = db * gm1;
                M1x[XL(a, r)] = f1 * dg1;        // to A1b of edge a+1
                const double gf1 = up1 * dg1;
                LimD<LIM>::f(A2[XE(a, r)], up2 * f2, da, db);
                A2b[XE(a, r)] += da * gm2;
                const double dg2 = db * gm2;
                M2x[XL(a, r)] = f2 * dg2;        // to A2b of edge a-1
                const double gf2 = up2 * dg2;
                if (MED) {
                    edgeadd(AUX_FX1, a, r, gf1);
                    edgeadd(AUX_FX2, a, r, gf2);
                    medadd(AUX_Z, a, r, kr * m2 * gcp);
                    medadd(AUX_Z, a - 1, r, -(kl * m1 * gcp));
                }
            }
            for (int k = tid; k < (ty + 1) * (tx + 2); k += ANT) {
                const int b = k / (tx + 2), c = k % (tx + 2) - 1;
                const double gcp = Cpy[YL(c, b)], gcv = Cvy[YL(c, b)];
                const double zr = AX(AUX_Z, c, b), zl = AX(AUX_Z, c, b - 1);
                const double kl = fma(-ly, AX(AUX_C2, c, b - 1), AX(AUX_C, c, b - 1));
                const double kr = fma(-ly, AX(AUX_C2, c, b), AX(AUX_C, c, b));
                const double m1 = M1y[YL(c, b)], m2 = M2y[YL(c, b)];
                const double ge2 = fma(zr, gcp, gcv), ge1 = fma(-zl, gcp, gcv);
                const double gkl = m1 * ge1, gkr = m2 * ge2;
                if (MED) {
                    medadd(AUX_C, c, b - 1, gkl * fma(-2.0 * ly, AX(AUX_C, c, b - 1), 1.0));
                    medadd(AUX_C, c, b, gkr * fma(-2.0 * ly, AX(AUX_C, c, b), 1.0));
                }
                const double gm1 = kl * ge1, gm2 = kr * ge2;
                const double f1 = AX(AUX_FY1, c, b), f2 = AX(AUX_FY2, c, b);
                const double up1 = B1[YE(c, b + 1)], up2 = B2[YE(c, b - 1)];
                double da, db;
                LimD<LIM>::f(B1[YE(c, b)], up1 * f1, da, db);
                B1b[YE(c, b)] += da * gm1;
                const double dg1 = db * gm1;
                M1y[YL(c, b)] = f1 * dg1;        // to B1b of edge b+1
                const double gf1 = up1 * dg1;
                LimD<LIM>::f(B2[YE(c, b)], up2 * f2, da, db);
                B2b[YE(c, b)] += da * gm2;
                const double dg2 = db * gm2;
                M2y[YL(c, b)] = f2 * dg2;        // to B2b of edge b-1
                const double gf2 = up2 * dg2;
                if (MED) {
                    edgeadd(AUX_FY1, c, b, gf1);
                    edgeadd(AUX_FY2, c, b, gf2);
                    medadd(AUX_Z, c, b, kr * m2 * gcp);
                    medadd(AUX_Z, c, b - 1, -(kl * m1 * gcp));
                }
            }
            __syncthreads();
        }

        // ---------------------------------------------------------------- reverse: normal Riemann
        // a1 = (Z_R du - dp) is, a2 = (Z_L du + dp) is
        // per edge: the adjoints of dp and du, stored in the edge's A1b / A2b slots for the
        // per-cell gather below
        for (int k = tid; k < (ty + 2) * (tx + 3); k += ANT) {
            const int r = k / (tx + 3) - 1, a = k % (tx + 3) - 1;
            double g1 = A1b[XE(a, r)], g2 = A2b[XE(a, r)];
            if (second) {
                if (a >= 1) g1 += M1x[XL(a - 1, r)];
                if (a <= tx - 1) g2 += M2x[XL(a + 1, r)];
            }
            if (!nonzero(g1) && !nonzero(g2)) {
                A1b[XE(a, r)] = 0.0;
                A2b[XE(a, r)] = 0.0;
                continue;
            }
            const int iR = CI(a, r);
            const double dp = sp[iR] - sp[iR - 1], du = su[iR] - su[iR - 1];
            const double zr = AX(AUX_Z, a, r), zl = AX(AUX_Z, a - 1, r), is = AX(AUX_IXS, a, r);
            const double n1 = fma(zr, du, -dp), n2 = fma(zl, du, dp);
            const double gn1 = is * g1, gn2 = is * g2;
            A1b[XE(a, r)] = gn2 - gn1;              // adjoint of dp = p_a - p_{a-1}
            A2b[XE(a, r)] = fma(zr, gn1, zl * gn2); // adjoint of du
            if (MED) {
                edgeadd(AUX_IXS, a, r, fma(n1, gn1, n2 * gn2));   // is x its adjoint
                medadd(AUX_Z, a, r, du * gn1);
                medadd(AUX_Z, a - 1, r, du * gn2);
            }
        }
        for (int k = tid; k < (ty + 3) * (tx + 2); k += ANT) {
            const int b = k / (tx + 2) - 1, c = k % (tx + 2) - 1;
            double g1 = B1b[YE(c, b)], g2 = B2b[YE(c, b)];
            if (second) {
                if (b >= 1) g1 += M1y[YL(c, b - 1)];
                if (b <= ty - 1) g2 += M2y[YL(c, b + 1)];
            }
            if (!nonzero(g1) && !nonzero(g2)) {
                B1b[YE(c, b)] = 0.0;
                B2b[YE(c, b)] = 0.0;
                continue;
            }
            const int iR = CI(c, b);
            const double dp = sp[iR] - sp[iR - G::SW], dv = sv[iR] - sv[iR - G::SW];
            const double zr = AX(AUX_Z, c, b), zl = AX(AUX_Z, c, b - 1), is = AX(AUX_IYS, c, b);
            const double n1 = fma(zr, dv, -dp), n2 = fma(zl, dv, dp);
            const double gn1 = is * g1, gn2 = is * g2;
            B1b[YE(c, b)] = gn2 - gn1;
            B2b[YE(c, b)] = fma(zr, gn1, zl * gn2);
            if (MED) {
                edgeadd(AUX_IYS, c, b, fma(n1, gn1, n2 * gn2));
                medadd(AUX_Z, c, b, dv * gn1);
                medadd(AUX_Z, c, b - 1, dv * gn2);
            }
        }
        __syncthreads();

        // ---------------------------------------------------------------- flush to global
        {
            // cell (i, j) of the staged block, i in [-2, tx+1], j in [-2, ty+1]: it is the right
            // cell of x-edge i and the left cell of x-edge i+1 (edges a in [-1, tx+1] on rows
            // [-1, ty]), likewise for the y-edges (b in [-1, ty+1] on columns [-1, tx])
            double* lo = lam_old + P.qoff;
            const int w4 = tx + 4, n4 = w4 * (ty + 4);
            auto gx = [&](const double* arr, int a, int r) -> double {
                return (a >= -1 && a <= tx + 1 && r >= -1 && r <= ty) ? arr[XE(a, r)] : 0.0;
            };
            auto gy = [&](const double* arr, int c, int b) -> double {
                return (b >= -1 && b <= ty + 1 && c >= -1 && c <= tx) ? arr[YE(c, b)] : 0.0;
            };
            for (int k = tid; k < n4; k += ANT) {
                const int j = k / w4 - 2, i = k % w4 - 2;
                double p = gx(A1b, i, j) - gx(A1b, i + 1, j) + gy(B1b, i, j) - gy(B1b, i, j + 1);
                double u = gx(A2b, i, j) - gx(A2b, i + 1, j);
                double v = gy(B2b, i, j) - gy(B2b, i, j + 1);
                p += LAM(0, i, j);
                u += LAM(1, i, j);
                v += LAM(2, i, j);
                const int gx = x0 + i, gy = y0 + j;
                if (A.ring && P.ring >= 0 && (gx < 0 || gx >= P.nx || gy < 0 || gy >= P.ny)) {
                    // a ghost of the box that the forward took from a cell of the level (same-level
                    // copy or physical boundary): its adjoint goes straight to that cell, with the
                    // wall sign flips; interpolated ghosts (source -1) keep theirs
                    const longlong2 e = A.ring[P.ring + ring_index(gx + 2, gy + 2, P.nx, P.ny)];
                    if (e.x >= 0) {
                        const long long pl = e.y & ((1LL << kRingFlagShift) - 1);
                        const int fl = (int)(e.y >> kRingFlagShift);
                        if (nonzero(p)) atomicAdd(lam_old + e.x, p);
                        if (nonzero(u)) atomicAdd(lam_old + e.x + pl, flip_sign(u, fl & 1));
                        if (nonzero(v)) atomicAdd(lam_old + e.x + 2 * pl, flip_sign(v, (fl >> 1) & 1));
                        continue;
                    }
                }
                const long long o = (long long)(gy + 2) * W + (gx + 2);
                if (nonzero(p)) atomicAdd(lo + o, p);
                if (nonzero(u)) atomicAdd(lo + WH + o, u);
                if (nonzero(v)) atomicAdd(lo + 2 * WH + o, v);
            }
        }
        __syncthreads();   // shared memory is reused by the next tile
    }
}

template <int MED>
void (*adj_kernel(int limiter))(const StepArgs, const double*, double*, double*)
{
    switch (limiter) {
    case CLAW_LIM_NONE: return step_adjoint_kernel<MED, CLAW_LIM_NONE>;
    case CLAW_LIM_MINMOD: return step_adjoint_kernel<MED, CLAW_LIM_MINMOD>;
    case CLAW_LIM_SUPERBEE: return step_adjoint_kernel<MED, CLAW_LIM_SUPERBEE>;
    case CLAW_LIM_VANLEER: return step_adjoint_kernel<MED, CLAW_LIM_VANLEER>;
    case CLAW_LIM_MC: return step_adjoint_kernel<MED, CLAW_LIM_MC>;
    }
    return nullptr;
}

// kernel with its shared-memory attribute set, and its resident CTAs per SM (cached per device)
template <int MED>
cudaError_t prepare_adj(int limiter, void (**fn)(const StepArgs, const double*, double*, double*), int* per_sm)
{
    constexpr int kDev = 64;
    static int cached[kDev][5] = {};
    *fn = adj_kernel<MED>(limiter);
    if (!*fn || limiter < 0 || limiter > 4) return cudaErrorInvalidValue;
    int dev = 0;
    cudaError_t ed = cudaGetDevice(&dev);
    if (ed != cudaSuccess) return ed;
    if (dev < 0 || dev >= kDev) return cudaErrorInvalidDevice;
    int* c = cached[dev];
    const size_t smem = AGeo::smem_bytes(MED);
    if (!c[limiter]) {
        cudaError_t e = cudaFuncSetAttribute((const void*)*fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int n = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, *fn, ANT, smem);
        if (e != cudaSuccess) return e;
        c[limiter] = n > 0 ? n : 1;
    }
    *per_sm = c[limiter];
    return cudaSuccess;
}

template <int MED>
cudaError_t launch_adj_med(const StepArgs& a, const double* lam_new, double* lam_old, double* g_aux, int limiter,
                           int nsm, cudaStream_t s)
{
    void (*fn)(const StepArgs, const double*, double*, double*) = nullptr;
    int per_sm = 1;
    cudaError_t e = prepare_adj<MED>(limiter, &fn, &per_sm);
    if (e != cudaSuccess) return e;
    const int grid = a.ntiles < per_sm * nsm ? a.ntiles : per_sm * nsm;
    if (grid <= 0) return cudaSuccess;
    fn<<<grid, ANT, AGeo::smem_bytes(MED), s>>>(a, lam_new, lam_old, g_aux);
    return cudaGetLastError();
}

}  // namespace

int adjoint_tile() { return ATX; }

cudaError_t launch_step_adjoint(const StepArgs& a, const double* lam_new, double* lam_old, double* g_aux, int medium,
                                int limiter, int nsm, cudaStream_t s)
{
    return medium ? launch_adj_med<1>(a, lam_new, lam_old, g_aux, limiter, nsm, s)
                  : launch_adj_med<0>(a, lam_new, lam_old, nullptr, limiter, nsm, s);
}

}  // namespace claw

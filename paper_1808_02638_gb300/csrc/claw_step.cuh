// claw_step.cuh -- the fused, persistent level-step kernel (sm_103a, FP64).
//
// One launch advances every tile of every box of a level (Eq. wave_form_2d_2nd_order, Sec. 2.1):
//   Q^{n+1} = Q - dt/dx (A+dQ_{i-1/2} + A-dQ_{i+1/2}) - dt/dy (B+dQ_{j-1/2} + B-dQ_{j+1/2})
//               - dt/dx (F~_{i+1/2} - F~_{i-1/2}) - dt/dy (G~_{j+1/2} - G~_{j-1/2})
// for the acoustics system of Sec. 4.1 with the wave-propagation Riemann solver, limiter,
// correction flux and transverse splitting of LeVeque (2002), the reference Sec. 2.1 defers to.
//
// Design (GB300 first, not the paper's per-patch launches of Sec. 3.1):
//  * persistent CTAs walk a size-sorted tile table; the (tx+4) x (ty+4) x 3 input tile with its
//    two ghost layers is staged into shared memory by a tensor-memory-accelerator bulk copy
//    (double-buffered: the next tile streams in while this one is computed) or by coalesced
//    loads;
//  * every edge is solved once per tile; waves and fluctuations never leave shared memory;
//    only Q^{n+1} is written back;
//  * the path is bound by the FP64 pipe (1/64 of FP32 on this part), so the arithmetic is
//    arranged to minimise FP64 instructions: the transverse split is applied once per cell
//    to the summed x-fluctuation (it is linear), constant coefficients fold into per-tile
//    constants, limiters are division free (phi(b/a) a), wave speeds are reduced on the
//    integer pipe as bit patterns;
//  * the CFL reduction (Sec. 2.4, 3.2.2) is a warp-shuffle / shared-memory max per tile folded
//    by the CTA, with one 64-bit atomic max per CTA and run on the run's device scalar.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "claw_interp.cuh"

namespace claw {

// ------------------------------------------------------------------------- limiters
// Lim<L>::f(a, b) = phi(b / a) * a for the wave strength a at an edge and the projected
// strength b of the same family at the upwind edge; 0 when a b <= 0 (also covers a = 0, where
// the wave vanishes).
//
// FP64 is 1/64 of the FP32 rate on this part, so minmod, superbee and MC run on the integer
// pipe: for non-negative doubles the bit patterns order like the values, so min / max of
// magnitudes are 64-bit integer min / max, and doubling or halving a magnitude adds or
// subtracts 1 in the exponent field.  MC's sum |a| + |b| is the IEEE-754 sum rounded to
// nearest even, formed on the integer pipe as well (add_mag), so none of the three issues an
// FP64 instruction.  The exponent shifts are exact for magnitudes >= 2^-1021; below that the
// result (itself below 2^-1020 in magnitude) may differ from the IEEE evaluation of the same
// formula by less than 2^-1020.  van Leer needs a quotient: one correctly rounded reciprocal
// and two products instead of a division (four roundings: within a relative 4 * 2^-53 of
// 2ab / (a + b)).
namespace lim_bits {
constexpr long long MAG = 0x7fffffffffffffffLL;
constexpr long long SIGN = (long long)0x8000000000000000ULL;
constexpr long long ONE_EXP = 1LL << 52;   // +1 in the exponent field: x2
__device__ __forceinline__ long long bits(double x) { return __double_as_longlong(x); }
__device__ __forceinline__ double val(long long b) { return __longlong_as_double(b); }
// a b > 0: same sign bit and both magnitudes non-zero
__device__ __forceinline__ bool same_sign_nonzero(long long ia, long long ib, long long ma, long long mb)
{
    return ((ia ^ ib) >= 0) & (ma != 0) & (mb != 0);
}
// The bit pattern of x + y for non-negative doubles x, y given by their bit patterns: the
// exact sum rounded to nearest, ties to even (IEEE 754, Sec. 4.3.1 and 6.3 of the 2008
// standard), on the integer pipe.  The smaller significand is aligned to the larger with three
// extra low bits (guard, round and a sticky OR of every bit shifted out), the significands are
// added, a carry out renormalises by one place (its lost bit joins the sticky bit), and the
// rounding increment may carry into the exponent field, which is how the significand overflow
// and the step from subnormal to normal come out right.  Subnormals take exponent 1 without the
// hidden bit.  Overflow gives +inf; an infinite or NaN operand gives +inf or that NaN (quieted).
__device__ __forceinline__ long long add_mag(long long x, long long y)
{
    constexpr long long FRAC = (1LL << 52) - 1, HID = 1LL << 52, INF = 0x7ff0000000000000LL;
    const long long hi = x > y ? x : y, lo = x > y ? y : x;
    const int eh = (int)(hi >> 52), el = (int)(lo >> 52);
    if (eh == 2047) return (hi & FRAC) ? (hi | (1LL << 51)) : hi;
    const int Eh = eh ? eh : 1, El = el ? el : 1;
    const int d = Eh - El < 57 ? Eh - El : 57;   // Fl < 2^56: a shift by 57 already leaves only the sticky bit
    const long long Fh = ((hi & FRAC) | (eh ? HID : 0)) << 3;
    const long long Fl = ((lo & FRAC) | (el ? HID : 0)) << 3;
    const long long al = (Fl >> d) | (long long)((Fl & ((1LL << d) - 1)) != 0);
    long long S = Fh + al;
    int E = Eh;
    if (S >> 56) {
        S = (S >> 1) | (S & 1);
        ++E;
    }
    const long long m = S >> 3;
    const int r = (int)(S & 7);
    const long long res = ((long long)(E - 1) << 52) + m + (long long)((r > 4) | ((r == 4) & (int)(m & 1)));
    return res >= INF ? INF : res;
}
}  // namespace lim_bits

// fc(a, b, code) returns f(a, b) and the branch the value took (LimCode), for the tape of a
// recording step; on the integer pipe like f.
template <int L> struct Lim;
template <> struct Lim<CLAW_LIM_NONE> {
    template <bool = false>
    static __device__ __forceinline__ double f(double a, double) { return a; }
    template <bool = false>
    static __device__ __forceinline__ double fc(double a, double, int& code)
    {
        code = LIMC_A;
        return a;
    }
};
template <> struct Lim<CLAW_LIM_MINMOD> {   // max(0, min(1, theta)): sign(a) min(|a|, |b|)
    template <bool = false>
    static __device__ __forceinline__ double f(double a, double b)
    {
        using namespace lim_bits;
        const long long ia = bits(a), ib = bits(b), ma = ia & MAG, mb = ib & MAG;
        const long long m = ma < mb ? ma : mb;
        return same_sign_nonzero(ia, ib, ma, mb) ? val(m | (ia & SIGN)) : 0.0;
    }
    template <bool = false>
    static __device__ __forceinline__ double fc(double a, double b, int& code)
    {
        using namespace lim_bits;
        const long long ia = bits(a), ib = bits(b), ma = ia & MAG, mb = ib & MAG;
        const bool nz = same_sign_nonzero(ia, ib, ma, mb);
        code = !nz ? LIMC_ZERO : (ma < mb ? LIMC_A : LIMC_B);
        return nz ? val((ma < mb ? ma : mb) | (ia & SIGN)) : 0.0;
    }
};
template <> struct Lim<CLAW_LIM_SUPERBEE> {   // max(0, min(1, 2 theta), min(2, theta))
    template <bool = false>
    static __device__ __forceinline__ double f(double a, double b)
    {   // sign(a) max(min(|a|, 2|b|), min(2|a|, |b|))
        using namespace lim_bits;
        const long long ia = bits(a), ib = bits(b), ma = ia & MAG, mb = ib & MAG;
        const long long a2 = ma + ONE_EXP, b2 = mb + ONE_EXP;
        const long long m1 = ma < b2 ? ma : b2, m2 = a2 < mb ? a2 : mb;
        const long long m = m1 > m2 ? m1 : m2;
        return same_sign_nonzero(ia, ib, ma, mb) ? val(m | (ia & SIGN)) : 0.0;
    }
    template <bool = false>
    static __device__ __forceinline__ double fc(double a, double b, int& code)
    {
        using namespace lim_bits;
        const long long ia = bits(a), ib = bits(b), ma = ia & MAG, mb = ib & MAG;
        const long long a2 = ma + ONE_EXP, b2 = mb + ONE_EXP;
        const bool first_a = ma < b2, second_a2 = a2 < mb;
        const long long m1 = first_a ? ma : b2, m2 = second_a2 ? a2 : mb;
        const bool nz = same_sign_nonzero(ia, ib, ma, mb);
        code = !nz ? LIMC_ZERO : (m1 > m2 ? (first_a ? LIMC_A : LIMC_2B) : (second_a2 ? LIMC_2A : LIMC_B));
        return nz ? val((m1 > m2 ? m1 : m2) | (ia & SIGN)) : 0.0;
    }
};
template <> struct Lim<CLAW_LIM_VANLEER> {   // (theta + |theta|) / (1 + |theta|): 2ab / (a + b)
    template <bool = false>
    static __device__ __forceinline__ double f(double a, double b)
    {   // a (b r) with r = 1 / ((a + b) / 2); |b r| <= 2 as a and b share their sign
        using namespace lim_bits;
        const long long ia = bits(a), ib = bits(b);
        const long long hs = (bits(a + b) & MAG) - ONE_EXP;   // |a + b| / 2, exact above 2^-1021
        // below that the result is under 2^-1020 in magnitude: 0 (r would overflow)
        if (!same_sign_nonzero(ia, ib, ia & MAG, ib & MAG) || hs < ONE_EXP) return 0.0;
        return a * (b * __drcp_rn(val(hs | (ia & SIGN))));
    }
    template <bool = false>
    static __device__ __forceinline__ double fc(double a, double b, int& code)
    {
        const double m = f(a, b);
        code = lim_bits::bits(m) & lim_bits::MAG ? LIMC_SMOOTH : LIMC_ZERO;
        return m;
    }
};
template <> struct Lim<CLAW_LIM_MC> {   // max(0, min((1 + theta)/2, 2, 2 theta))
    // FPSUM: the sum on the FP64 pipe instead (the same bits)
    template <bool FPSUM = false>
    static __device__ __forceinline__ double f(double a, double b)
    {   // sign(a) min((|a| + |b|) / 2, 2 |a|, 2 |b|) = sign(a) min(s / 2, 2 min(|a|, |b|))
        using namespace lim_bits;
        const long long ia = bits(a), ib = bits(b), ma = ia & MAG, mb = ib & MAG;
        const long long t2 = (ma < mb ? ma : mb) + ONE_EXP;
        long long sh = (FPSUM ? bits(val(ma) + val(mb)) : add_mag(ma, mb)) - ONE_EXP;
        sh = sh > 0 ? sh : 0;   // a subnormal sum would wrap below zero
        const long long m = sh < t2 ? sh : t2;
        return same_sign_nonzero(ia, ib, ma, mb) ? val(m | (ia & SIGN)) : 0.0;
    }
    template <bool FPSUM = false>
    static __device__ __forceinline__ double fc(double a, double b, int& code)
    {
        using namespace lim_bits;
        const long long ia = bits(a), ib = bits(b), ma = ia & MAG, mb = ib & MAG;
        const long long t2 = (ma < mb ? ma : mb) + ONE_EXP;
        long long sh = (FPSUM ? bits(val(ma) + val(mb)) : add_mag(ma, mb)) - ONE_EXP;
        sh = sh > 0 ? sh : 0;
        const bool nz = same_sign_nonzero(ia, ib, ma, mb);
        code = !nz ? LIMC_ZERO : (sh < t2 ? LIMC_HALF : (ma < mb ? LIMC_2A : LIMC_2B));
        return nz ? val((sh < t2 ? sh : t2) | (ia & SIGN)) : 0.0;
    }
};

// a limited strength with its branch in the three lowest mantissa bits (a relative change
// below 2^-49; exact zeros stay zero)
__device__ __forceinline__ double tag_code(double m, int code)
{
    return __longlong_as_double((__double_as_longlong(m) & ~7LL) | (long long)code);
}

// ------------------------------------------------------------------------- tile geometry
template <int TX, int TY> struct Geo {
    static constexpr int SW = TX + 4, SH = TY + 4, QPL = SW * SH;  // staged q plane
    static constexpr int XEW = TX + 3, XEH = TY + 2;               // x-edges a in [-1,TX+1], rows [-1,TY]
    static constexpr int YEW = TX + 2, YEH = TY + 3;               // y-edges b in [-1,TY+1], cols [-1,TX]
    static constexpr int XLW = TX + 1, XLH = TY + 2;               // limited x-edges a in [0,TX]
    static constexpr int YLW = TX + 2, YLH = TY + 1;               // limited y-edges b in [0,TY]
    static constexpr int DW = TX, DH = TY + 2;                     // D: cols [0,TX), rows [-1,TY]
    static constexpr int EW = TX + 2, EH = TY;                     // E: cols [-1,TX], rows [0,TY)
    static constexpr int QBYTES = 3 * QPL * 8;
    // shared-memory carve (in doubles), q buffers first (128-byte aligned)
    static constexpr int QSTRIDE = (3 * QPL + 15) / 16 * 16;
    // rows a tile hands to the tile above it in a column walk (top rows of each array):
    // x-edge strengths 2 rows, y-edge strengths 3, limited x-edges 2, limited y-edges 1, D 1
    static constexpr int C_A = 0, C_B = 4 * XEW, C_S = C_B + 6 * YEW, C_SY = C_S + 4 * XLW,
                         C_D = C_SY + 2 * YLW, NCARRY = C_D + DW;
    static constexpr int NWORK = 2 * XEW * XEH + 2 * YEW * YEH + 2 * XLW * XLH + 2 * YLW * YLH +
                                 DW * DH + EW * EH;
    // q buffers, work arrays, 64 bytes of barriers, then (column walks only) the carried rows
    static size_t smem_bytes(int nbuf, bool walk = false)
    {
        return (size_t)(nbuf * QSTRIDE + NWORK) * 8 + 64 + (walk ? (size_t)NCARRY * 8 : 0);
    }
};

// The tiles [*begin, *end) of CTA b of `grid` in a column walk: the contiguous range whose
// cumulative cost (cum[i] = cost of tiles [0, i), cum[n] the total) starts at or after b / grid
// of the total.  The ranges of all CTAs partition [0, n).
__device__ __forceinline__ int walk_start(const long long* cum, int n, int b, int grid)
{
    const long long target = (long long)b * __ldg(cum + n) / grid;   // b < 2^20, cum[n] < 2^40
    int lo = 0, hi = n;   // first i in [0, n] with cum[i] >= target
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(cum + mid) < target) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// ------------------------------------------------------------------------- PTX helpers
__device__ __forceinline__ unsigned smem_u32(const void* p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void fence_barrier_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// 3-D tiled bulk tensor copy global -> shared completing on an mbarrier.  Coordinates are
// (x, y, plane) in elements; x * 8 bytes is a multiple of 16 (x is even by construction).
__device__ __forceinline__ void tma_load_3d(void* dst, const void* tmap, int x, int y, int z,
                                            unsigned long long* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(tmap), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// bounded wait: gives up after `polls` polls and reports it; never spins without a limit
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity,
                                                  unsigned polls = kWaitPolls)
{
    for (unsigned it = 0; it < polls; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ bool not_finite(double x)
{
    return ((unsigned)(__double_as_longlong(x) >> 32) & 0x7ff00000u) == 0x7ff00000u;
}

// max of non-negative doubles on the integer pipe (bit patterns order like the values)
__device__ __forceinline__ unsigned long long umax64(unsigned long long a, unsigned long long b)
{
    return a > b ? a : b;
}

// fused Eq. cfl, run by thread 0 of every CTA as its last action: the last CTA to finish sees
// every CTA's speed maximum (each published its atomics before its fence and its count), checks
// the CFL number of the step just taken, sets the next dt, resets the maxima and re-arms the
// counter.  No CTA waits on another.
__device__ __forceinline__ void finish_cta(const StepArgs& A)
{
    if (!A.dtupd) return;
    __threadfence();
    const unsigned prev = atomicAdd(A.done, 1u);
    if (prev != gridDim.x - 1) return;
    __threadfence();
    for (int r = 0; r < A.nruns; ++r) {
        const double s = *reinterpret_cast<volatile double*>(A.smax + r);
        const double used = *reinterpret_cast<volatile double*>(A.dt_out + r);
        if (s * used > A.minh[r] * (1.0 + 1e-12)) atomicOr(A.err, ERR_CFL);
        if (s > 0.0) A.dt_out[r] = A.cflv[r] * A.minh[r] / s;
        A.smax[r] = 0.0;
    }
    __threadfence();
    *reinterpret_cast<volatile unsigned*>(A.done) = 0u;
}

// The fill jobs of a launch, run by its CTAs from A.step_grid on: one thread per (ghost cell,
// component), striding over the jobs' cells together, each value as the ghost-fill kernel
// computes it.  The cells written are ghosts that no tile of the launch reads or writes.
template <int NT>
__device__ __forceinline__ void fill_jobs(const StepArgs& A)
{
    const long long n0 = 3LL * A.fills[0].n;
    const long long n = n0 + (A.nfill > 1 ? 3LL * A.fills[1].n : 0LL);
    const long long stride = (long long)(gridDim.x - A.step_grid) * NT;
    for (long long k = (long long)(blockIdx.x - A.step_grid) * NT + threadIdx.x; k < n; k += stride) {
        const bool second = k >= n0;
        const InterpCell* cells = second ? A.fills[1].cells : A.fills[0].cells;
        double* q = second ? A.fills[1].q : A.fills[0].q;
        const double* cold = second ? A.fills[1].cold : A.fills[0].cold;
        const double* cnew = second ? A.fills[1].cnew : A.fills[0].cnew;
        const double tau = second ? A.fills[1].tau : A.fills[0].tau;
        const long long kk = second ? k - n0 : k;
        const int c = (int)(kk / 3), m = (int)(kk - 3LL * c);
        const InterpCell C = cells[c];
        q[C.dst + m * C.dplane] = interp_value(C, m, cold, cnew, tau);
    }
}

// Same-level and physical-boundary ghosts of a staged tile, taken from their source cells in
// q_old (the box's ghost ring table) instead of the pool's own ghost cells: only the frame of
// width two around the tile can hold ghosts of its box.  Ghosts interpolated from the coarser
// level are evaluated from the coarse states in the instantiations with INTERP (the same
// arithmetic as the ghost-fill kernel; a separate instantiation, as the code alone costs the
// other kernels registers), else keep the staged value.  The caller separates this from the
// staging and from the tile's first reads with barriers.
template <int SW, int QPL, int NT, bool INTERP = false>
__device__ __forceinline__ void pull_ghosts(const StepArgs& A, const PatchDev& P, double* sq, int x0, int y0, int tx,
                                            int ty)
{
    const int w = tx + 4, nf = 4 * (tx + ty + 4);
    for (int k = (int)threadIdx.x; k < nf; k += NT) {
        int xs, ys;
        if (k < 4 * w) {   // rows 0, 1, ty+2, ty+3 of the staged tile
            const int r = k / w;
            xs = k - r * w;
            ys = r < 2 ? r : ty + r;
        } else {           // columns 0, 1, tx+2, tx+3 of rows 2 .. ty+1
            const int kk = k - 4 * w, c = kk & 3;
            ys = 2 + (kk >> 2);
            xs = c < 2 ? c : tx + c;
        }
        const int ri = ring_index(x0 + xs, y0 + ys, P.nx, P.ny);
        if (ri < 0) continue;
        const longlong2 e = __ldg(&A.ring[P.ring + ri]);
        if (e.x < 0) {   // interpolated from the coarser level
            if (INTERP) {
                const InterpCell C = A.interp[P.interp + (int)(-1 - e.x)];
                const int i = xs + ys * SW;
                sq[i] = interp_value(C, 0, A.cold, A.cnew, A.tau);
                sq[QPL + i] = interp_value(C, 1, A.cold, A.cnew, A.tau);
                sq[2 * QPL + i] = interp_value(C, 2, A.cold, A.cnew, A.tau);
            }
            continue;
        }
        const long long sp = e.y & ((1LL << kRingFlagShift) - 1);
        const double* src = A.qold + e.x;
        const unsigned fl = (unsigned)(e.y >> kRingFlagShift);
        // wall sign flips as sign-bit xors (integer pipe, not an FP64 negation)
        const unsigned long long sb = (unsigned long long)(fl & 1u) << 63;
        const unsigned long long sc = (unsigned long long)((fl >> 1) & 1u) << 63;
        const double a = __ldg(src);
        const unsigned long long b = (unsigned long long)__double_as_longlong(__ldg(src + sp));
        const unsigned long long c = (unsigned long long)__double_as_longlong(__ldg(src + 2 * sp));
        const int i = xs + ys * SW;
        sq[i] = a;
        sq[QPL + i] = __longlong_as_double((long long)(b ^ sb));
        sq[2 * QPL + i] = __longlong_as_double((long long)(c ^ sc));
    }
    // these generic writes precede later bulk copies (async proxy) into the same buffer
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// ------------------------------------------------------------------------- the kernel
// MED: 0 uniform medium (rho0, K0), 1 cell-wise aux planes.
// STAGE: 0 cooperative loads, 1 tensor bulk copies (double buffered: the next tile streams in
// during the whole of this one), 2 tensor bulk copies into one buffer (the next tile is requested
// once this one's state has been read, in phase D) with registers capped for three CTAs per SM.
// PULL: 1 same-level and boundary ghosts are taken from their source cells (a separate
// instantiation: the mere presence of the pull code slowed the other kernels by up to 11 %);
// 2 those and the ghosts interpolated from the coarser level, evaluated in the step.
// REC (cell-wise medium): also write the step's intermediates to the tape A.tape (TapePlane);
// each padded cell's entries come from the one tile that owns the cell (its interior, plus the
// box's ghost frame next to it), so the tape is the same whatever the tiling.
// Registers: the one-buffer staging is capped for three CTAs per SM; the 128-thread tiles for
// five (the shared memory of five fits an SM), except those evaluating interpolated ghosts.
template <int MED, int LIM, int TX, int TY, int NT, int STAGE, int PULL, bool REC = false>
__global__ void __launch_bounds__(NT, STAGE == 2 ? 3 : (NT == 128 && !REC ? 5 : 1))
    step_kernel(const StepArgs A)
{
    static_assert(!REC || MED == 1, "the tape records the cell-wise step");
    // (REC kernels never walk: column walks are built for the uniform medium only)
    using G = Geo<TX, TY>;
    constexpr int NBUF = STAGE == 1 ? 2 : 1;
    constexpr int NPER = (TX * TY + NT - 1) / NT;
    if (A.step_grid && blockIdx.x >= A.step_grid) {   // a fill CTA: no tiles, no shared memory
        fill_jobs<NT>(A);
        if (threadIdx.x == 0) finish_cta(A);
        return;
    }
    // the CTAs that step tiles
    const int nstep = A.step_grid ? A.step_grid : (int)gridDim.x;
    extern __shared__ __align__(128) double smem[];
    double* qbuf = smem;                            // NBUF x QSTRIDE
    double* A1x = smem + NBUF * G::QSTRIDE;         // x-edge wave strengths, family 1 / 2
    double* A2x = A1x + G::XEW * G::XEH;
    double* B1y = A2x + G::XEW * G::XEH;            // y-edge wave strengths
    double* B2y = B1y + G::YEW * G::YEH;
    double* Sx = B2y + G::YEW * G::YEH;             // limited x-edges: const: M2-M1 / var: C_p
    double* Px = Sx + G::XLW * G::XLH;              //                  const: M1+M2 / var: C_u
    double* Sy = Px + G::XLW * G::XLH;
    double* Py = Sy + G::YLW * G::YLH;
    double* Dx = Py + G::YLW * G::YLH;              // x-fluctuation pressure into each cell
    double* Ey = Dx + G::DW * G::DH;                // y-fluctuation pressure into each cell
    unsigned long long* bar = reinterpret_cast<unsigned long long*>(Ey + G::EW * G::EH);
    // rows carried to the next tile of a column walk: allocated only for launches that walk
    double* Cy = reinterpret_cast<double*>(bar) + 8;
    __shared__ unsigned long long s_tmax[2];   // per-tile speed max, double-buffered by tile parity
    __shared__ int s_flag;
    __shared__ int s_range[2];                 // this CTA's tiles in a column walk
    __shared__ double s_k[16];                 // per-tile constants, written by thread 0
    __shared__ double s_med[3];                // uniform medium Z0, c0, 1 / Z0, written by thread 0

    const int tid = threadIdx.x;
    if (tid == 0) {
        s_tmax[0] = s_tmax[1] = 0ull;
        s_flag = 0;
        if (MED == 0) {   // square roots and a division: thread 0 alone (all threads cost ~0.9 FP64 per cell)
            s_med[0] = sqrt(A.K0 * A.rho0);
            s_med[1] = sqrt(A.K0 / A.rho0);
            s_med[2] = 1.0 / s_med[0];
        }
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
    // Column walk (A.tcum set): the CTA takes a contiguous range of tiles, and a tile flagged
    // TILE_CARRY that follows its lower neighbour in the same range takes the rows the two share
    // (edges of the rows between them) from that neighbour instead of recomputing them: the
    // neighbour is the tile directly below in the same box or (uniform medium) in the same-level
    // box below, whose shared rows hold the same values.  Otherwise the CTA strides over all
    // tiles by the grid.
    // Only the uniform medium walks (the host builds column walks for no other kind), so the
    // cell-wise kernels carry none of this code.
    const int t_begin = s_range[0], t_end = s_range[1];
    const int t_step = A.tcum ? 1 : nstep;
    const bool walk = MED == 0 && A.tcum != nullptr;

    const CUtensorMap* tmaps = reinterpret_cast<const CUtensorMap*>(A.tmaps);
    int my_flag = 0;
    // thread 0 folds the tile maxima of consecutive tiles of the same run and flushes one
    // 64-bit atomic max per run change (speeds are >= 0: bit patterns order like values)
    int cur_run = -1;
    unsigned long long cur_max = 0ull;
    auto flush = [&]() {
        if (cur_run >= 0 && cur_max)
            atomicMax(reinterpret_cast<unsigned long long*>(A.smax) + cur_run, cur_max);
    };
    // uniform medium constants (once per CTA)
    double Z0 = 0, c0 = 0, iZ = 0;
    if (MED == 0) {
        Z0 = s_med[0];
        c0 = s_med[1];
        iZ = s_med[2];
    }

    auto issue = [&](int t, int b) {
        const TileDev T = A.tiles[t];
        mbar_expect_tx(&bar[b], (unsigned)G::QBYTES);
        tma_load_3d(qbuf + b * G::QSTRIDE, &tmaps[T.patch], T.x0, T.y0, 0, &bar[b]);
    };
    if (STAGE && tid == 0 && t_begin < t_end) issue(t_begin, 0);

    int it = 0;
    for (int t = t_begin; t < t_end; t += t_step, ++it) {
        const int b = STAGE == 1 ? (it & 1) : 0;
        const TileDev T = A.tiles[t];
        // carry: this tile's lowest rows come from the previous tile; hand: the next one takes
        // this tile's top rows
        const bool carry = walk && t > t_begin && (T.flags & TILE_CARRY);
        const bool hand = walk && t + 1 < t_end && (A.tiles[t + 1].flags & TILE_CARRY);
        const PatchDev P = A.patches[T.patch];
        const int tx = T.tx, ty = T.ty, x0 = T.x0, y0 = T.y0;
        const int W = P.nx + 4;
        const long long WH = (long long)W * (P.ny + 4);
        double* sq = qbuf + b * G::QSTRIDE;
        double* sp = sq;
        double* su = sq + G::QPL;
        double* sv = sq + 2 * G::QPL;

        if (STAGE) {
            const int tn = t + t_step;
            if (STAGE == 1 && tid == 0 && tn < t_end) issue(tn, b ^ 1);
            // each buffer's barrier completes once per use: every other tile with two buffers,
            // every tile with one
            const unsigned par = STAGE == 1 ? (unsigned)((it >> 1) & 1) : (unsigned)(it & 1);
            bool ok = mbar_wait_bounded(&bar[b], par, A.wait_polls);
            if (__syncthreads_or(!ok)) {   // the copy is late or lost: report and stop this CTA
                if (tid == 0) {
                    atomicOr(A.err, ERR_TIMEOUT);
                    // no copy may land in this CTA's shared memory after it exits: wait, with the
                    // full bound, for this tile's own copy and for the prefetch of the next one
                    mbar_wait_bounded(&bar[b], par);
                    if (STAGE == 1 && tn < t_end)
                        mbar_wait_bounded(&bar[b ^ 1], (unsigned)(((it + 1) >> 1) & 1));
                    finish_cta(A);   // keeps the completion count consistent
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
            pull_ghosts<G::SW, G::QPL, NT, PULL == 2>(A, P, sq, x0, y0, tx, ty);
            __syncthreads();
        }

        // ---------------------------------------------------------------- per-tile constants
        // Computed once per tile by thread 0 (every thread doing it cost several FP64 slots per
        // cell); first read after the barrier that ends phase A, last read in phase D, which
        // the end-of-tile barrier separates from the next tile's write.
        const bool second = A.order == 2 && LIM >= 0;
        const bool trans = A.transverse != 0;
        const bool cw = A.transverse == 2 && A.order == 2;   // correction rides the transverse split
        if (tid == 0) {
            const double dt = __ldg(A.dt + P.run) * P.dtscale;
            const double lx = dt * P.dxinv, ly = dt * P.dyinv;
            s_k[12] = lx;
            s_k[13] = ly;
            s_k[14] = -0.5 * lx;
            s_k[15] = -0.5 * ly;
            if (MED == 0) {
                // the centre part 2 kT (D + E) of the transverse pressure update folds into the
                // normal-update coefficients (D = ap + kDx bp, E likewise); phase D adds the rest
                const double kapx = c0 * (1.0 - lx * c0), kapy = c0 * (1.0 - ly * c0);
                const double kDx = cw ? 1.0 - lx * c0 : 0.0, kDy = cw ? 1.0 - ly * c0 : 0.0;
                const double kT = trans ? 0.125 * lx * ly * c0 * A.K0 : 0.0;
                s_k[0] = fma(-0.5 * lx, A.K0, 2.0 * kT);              // cpa
                s_k[1] = fma(-0.25 * lx * kapx, Z0, 2.0 * kT * kDx);  // cpb
                s_k[2] = -0.5 * lx * c0;                              // cua
                s_k[3] = -0.25 * lx * kapx;                           // cub
                s_k[4] = fma(-0.5 * ly, A.K0, 2.0 * kT);              // cpay
                s_k[5] = fma(-0.25 * ly * kapy, Z0, 2.0 * kT * kDy);  // cpby
                s_k[6] = -0.5 * ly * c0;                              // cva
                s_k[7] = -0.25 * ly * kapy;                           // cvb
                s_k[8] = kDx;
                s_k[9] = kDy;
                s_k[10] = -kT;
                s_k[11] = trans ? 0.125 * lx * ly * c0 * c0 : 0.0;   // kU
            }
        }
        // medium access (MED == 1): aux plane k of the cell at tile-local (i, j)
        const double* aux = MED ? A.aux + P.aoff : nullptr;
        auto AX = [&](int k, int i, int j) -> double {
            return __ldg(aux + k * WH + (long long)(y0 + j + 2) * W + (x0 + i + 2));
        };
        // recording: the tile owns its interior and, at a box side, the two ghost layers there
        const int olx = x0 == 0 ? -2 : 0, ohx = x0 + tx == P.nx ? tx + 2 : tx;
        const int oly = y0 == 0 ? -2 : 0, ohy = y0 + ty == P.ny ? ty + 2 : ty;
        double* tape = REC ? A.tape + P.aoff : nullptr;
        auto rec = [&](int k, int i, int j, double v) {
            if (REC && i >= olx && i < ohx && j >= oly && j < ohy)
                tape[k * WH + (long long)(y0 + j + 2) * W + (x0 + i + 2)] = v;
        };

        // ---------------------------------------------------------------- phase A: normal Riemann
        // carried rows land in the lowest rows of the arrays, which this phase does not write
        // (the previous tile's last reads of them were behind its end-of-tile barrier)
        if (carry) {
            for (int k = tid; k < G::NCARRY; k += NT) {
                double* dst;
                if (k < G::C_B) dst = k < 2 * G::XEW ? A1x + k : A2x + (k - 2 * G::XEW);
                else if (k < G::C_S) dst = k < G::C_B + 3 * G::YEW ? B1y + (k - G::C_B) : B2y + (k - G::C_B - 3 * G::YEW);
                else if (k < G::C_SY) dst = k < G::C_S + 2 * G::XLW ? Sx + (k - G::C_S) : Px + (k - G::C_S - 2 * G::XLW);
                else if (k < G::C_D) dst = k < G::C_SY + G::YLW ? Sy + (k - G::C_SY) : Py + (k - G::C_SY - G::YLW);
                else dst = Dx + (k - G::C_D);
                *dst = Cy[k];
            }
        }
        // first rows computed here: with a carry, the rows below come from the previous tile
        const int rx0 = carry ? 1 : -1;   // x-edges and limited x-edges: rows [rx0, ty]
        const int by0 = carry ? 2 : -1;   // y-edges: b in [by0, ty + 1]
        const int ly0 = carry ? 1 : 0;    // limited y-edges: b in [ly0, ty]
        // x-edge a (between cells a-1 and a) on rows r in [-1, ty]
        {
            const int w = tx + 3, n = (ty + 1 - rx0) * w;
            for (int k = tid; k < n; k += NT) {
                const int r = k / w + rx0, a = k - (r - rx0) * w - 1;
                const int iR = (a + 2) + (r + 2) * G::SW;
                const double dp = sp[iR] - sp[iR - 1];
                const double du = su[iR] - su[iR - 1];
                double a1, a2;
                if (MED == 0) {   // 2 alpha: du -/+ dp / Z
                    a1 = fma(-dp, iZ, du);
                    a2 = fma(dp, iZ, du);
                } else {
                    const double zr = AX(AUX_Z, a, r), zl = AX(AUX_Z, a - 1, r), is = AX(AUX_IXS, a, r);
                    a1 = fma(zr, du, -dp) * is;
                    a2 = fma(zl, du, dp) * is;
                    rec(TAPE_A1, a, r, a1);
                    rec(TAPE_A2, a, r, a2);
                }
                A1x[(r + 1) * G::XEW + (a + 1)] = a1;
                A2x[(r + 1) * G::XEW + (a + 1)] = a2;
            }
        }
        // y-edge b (between rows b-1 and b) on columns c in [-1, tx]
        {
            const int w = tx + 2, n = (ty + 2 - by0) * w;
            for (int k = tid; k < n; k += NT) {
                const int bb = k / w + by0, c = k - (bb - by0) * w - 1;
                const int iR = (c + 2) + (bb + 2) * G::SW;
                const double dp = sp[iR] - sp[iR - G::SW];
                const double dv = sv[iR] - sv[iR - G::SW];
                double b1, b2;
                if (MED == 0) {
                    b1 = fma(-dp, iZ, dv);
                    b2 = fma(dp, iZ, dv);
                } else {
                    const double zr = AX(AUX_Z, c, bb), zl = AX(AUX_Z, c, bb - 1), is = AX(AUX_IYS, c, bb);
                    b1 = fma(zr, dv, -dp) * is;
                    b2 = fma(zl, dv, dp) * is;
                    rec(TAPE_B1, c, bb, b1);
                    rec(TAPE_B2, c, bb, b2);
                }
                B1y[(bb + 1) * G::YEW + (c + 1)] = b1;
                B2y[(bb + 1) * G::YEW + (c + 1)] = b2;
            }
        }
        // wave speeds seen by this tile (ring [-1,tx] x [-1,ty]): integer max of bit patterns,
        // warp shuffle, shared atomic
        if (MED == 0) {
            if (tid == 0) s_tmax[it & 1] = (unsigned long long)__double_as_longlong(c0);
        } else {
            unsigned long long m = 0ull;
            const int w = tx + 2, n = (ty + 2) * w;
            for (int k = tid; k < n; k += NT) {
                const int r = k / w - 1, c = k - (r + 1) * w - 1;
                m = umax64(m, (unsigned long long)__double_as_longlong(AX(AUX_C, c, r)));
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) m = umax64(m, __shfl_xor_sync(0xffffffffu, m, o));
            if ((tid & 31) == 0 && m) atomicMax(&s_tmax[it & 1], m);
        }
        __syncthreads();

        // ---------------------------------------------------------------- phase B: limiter, correction
        const double lx = s_k[12], ly = s_k[13];
        if (second) {
            {
                const int w = tx + 1, n = (ty + 1 - rx0) * w;
                for (int k = tid; k < n; k += NT) {
                    const int r = k / w + rx0, a = k - (r - rx0) * w;
                    const int e = (r + 1) * G::XEW + (a + 1);
                    const double a1 = A1x[e], a2 = A2x[e];
                    double m1, m2;
                    if (MED == 0) {
                        m1 = Lim<LIM>::f(a1, A1x[e + 1]);   // left-going: upwind edge a+1
                        m2 = Lim<LIM>::f(a2, A2x[e - 1]);   // right-going: upwind edge a-1
                        Sx[(r + 1) * G::XLW + a] = m2 - m1;
                        Px[(r + 1) * G::XLW + a] = m1 + m2;
                    } else {
                        if (REC) {
                            int c1, c2;
                            m1 = Lim<LIM>::template fc<true>(a1, A1x[e + 1] * AX(AUX_FX1, a, r), c1);
                            m2 = Lim<LIM>::template fc<true>(a2, A2x[e - 1] * AX(AUX_FX2, a, r), c2);
                            rec(TAPE_M1, a, r, tag_code(m1, c1));
                            rec(TAPE_M2, a, r, tag_code(m2, c2));
                        } else {
                            m1 = Lim<LIM>::template f<true>(a1, A1x[e + 1] * AX(AUX_FX1, a, r));
                            m2 = Lim<LIM>::template f<true>(a2, A2x[e - 1] * AX(AUX_FX2, a, r));
                        }
                        const double kl = fma(-lx, AX(AUX_C2, a - 1, r), AX(AUX_C, a - 1, r));
                        const double kr = fma(-lx, AX(AUX_C2, a, r), AX(AUX_C, a, r));
                        const double e1 = kl * m1, e2 = kr * m2;
                        Sx[(r + 1) * G::XLW + a] = fma(AX(AUX_Z, a, r), e2, -(AX(AUX_Z, a - 1, r) * e1));
                        Px[(r + 1) * G::XLW + a] = e1 + e2;
                    }
                }
            }
            {
                const int w = tx + 2, n = (ty + 1 - ly0) * w;
                for (int k = tid; k < n; k += NT) {
                    const int bb = k / w + ly0, c = k - (bb - ly0) * w - 1;
                    const int e = (bb + 1) * G::YEW + (c + 1);
                    const double b1 = B1y[e], b2 = B2y[e];
                    double m1, m2;
                    if (MED == 0) {
                        m1 = Lim<LIM>::f(b1, B1y[e + G::YEW]);
                        m2 = Lim<LIM>::f(b2, B2y[e - G::YEW]);
                        Sy[bb * G::YLW + (c + 1)] = m2 - m1;
                        Py[bb * G::YLW + (c + 1)] = m1 + m2;
                    } else {
                        if (REC) {
                            int c1, c2;
                            m1 = Lim<LIM>::template fc<true>(b1, B1y[e + G::YEW] * AX(AUX_FY1, c, bb), c1);
                            m2 = Lim<LIM>::template fc<true>(b2, B2y[e - G::YEW] * AX(AUX_FY2, c, bb), c2);
                            rec(TAPE_N1, c, bb, tag_code(m1, c1));
                            rec(TAPE_N2, c, bb, tag_code(m2, c2));
                        } else {
                            m1 = Lim<LIM>::template f<true>(b1, B1y[e + G::YEW] * AX(AUX_FY1, c, bb));
                            m2 = Lim<LIM>::template f<true>(b2, B2y[e - G::YEW] * AX(AUX_FY2, c, bb));
                        }
                        const double kl = fma(-ly, AX(AUX_C2, c, bb - 1), AX(AUX_C, c, bb - 1));
                        const double kr = fma(-ly, AX(AUX_C2, c, bb), AX(AUX_C, c, bb));
                        const double e1 = kl * m1, e2 = kr * m2;
                        Sy[bb * G::YLW + (c + 1)] = fma(AX(AUX_Z, c, bb), e2, -(AX(AUX_Z, c, bb - 1) * e1));
                        Py[bb * G::YLW + (c + 1)] = e1 + e2;
                    }
                }
            }
            __syncthreads();
        }

        // ---------------------------------------------------------------- phase C: per-cell terms
        // uniform medium, with a = 2 alpha and M = phi(theta) a:
        //   x-normal update  dp = -(lx K/2) ap - (lx kap Z/4) bp,  du = -(lx c/2) au - (lx kap/4) bu
        //   (dp also carries the centre term 2 kT D of the transverse update)
        //   ap = A2_w + A1_e, au = A2_w - A1_e, bp = S_e - S_w, bu = P_e - P_w,  kap = c (1 - lx c)
        //   x-fluctuation pressure into the cell D = (K/2) (ap + (1 - lx c) bp)
        // cell-wise medium: D = K ap + bp,  x-normal (K ap + bp/2, c au + bu/2)
        double cpa = 0, cpb = 0, cua = 0, cub = 0, cpay = 0, cpby = 0, cva = 0, cvb = 0, kDx = 0, kDy = 0;
        if (MED == 0) {
            cpa = s_k[0];
            cpb = s_k[1];
            cua = s_k[2];
            cub = s_k[3];
            cpay = s_k[4];
            cpby = s_k[5];
            cva = s_k[6];
            cvb = s_k[7];
            kDx = s_k[8];
            kDy = s_k[9];
        }
        // dP, dU, dV: Q plus the normal updates (the transverse terms are added in phase D)
        double dP[NPER], dU[NPER], dV[NPER];
#pragma unroll
        for (int n = 0; n < NPER; ++n) {
            dP[n] = dU[n] = dV[n] = 0.0;
            const int ci = tid + n * NT;
            const int c = ci % TX, r = ci / TX;
            if (ci >= TX * TY || c >= tx || r >= ty) continue;
            const int iq = (c + 2) + (r + 2) * G::SW;
            const int ex = (r + 1) * G::XEW + (c + 1);
            const int ey = (r + 1) * G::YEW + (c + 1);
            const double apx = A2x[ex] + A1x[ex + 1], aux_ = A2x[ex] - A1x[ex + 1];
            const double apy = B2y[ey] + B1y[ey + G::YEW], avy = B2y[ey] - B1y[ey + G::YEW];
            double bpx = 0, bux = 0, bpy = 0, bvy = 0;
            if (second) {
                bpx = Sx[(r + 1) * G::XLW + c + 1] - Sx[(r + 1) * G::XLW + c];
                bux = Px[(r + 1) * G::XLW + c + 1] - Px[(r + 1) * G::XLW + c];
                bpy = Sy[(r + 1) * G::YLW + c + 1] - Sy[r * G::YLW + c + 1];
                bvy = Py[(r + 1) * G::YLW + c + 1] - Py[r * G::YLW + c + 1];
            }
            if (MED == 0) {
                if (trans) {
                    Dx[(r + 1) * G::DW + c] = fma(kDx, bpx, apx);
                    Ey[r * G::EW + c + 1] = fma(kDy, bpy, apy);
                }
                dP[n] = fma(cpa, apx, fma(cpb, bpx, fma(cpay, apy, fma(cpby, bpy, sp[iq]))));
                dU[n] = fma(cua, aux_, fma(cub, bux, su[iq]));
                dV[n] = fma(cva, avy, fma(cvb, bvy, sv[iq]));
            } else {
                const double Kc = AX(AUX_K, c, r), cc = AX(AUX_C, c, r);
                if (trans) {
                    const double dd = cw ? fma(Kc, apx, bpx) : Kc * apx;
                    const double ee = cw ? fma(Kc, apy, bpy) : Kc * apy;
                    Dx[(r + 1) * G::DW + c] = dd;
                    Ey[r * G::EW + c + 1] = ee;
                    rec(TAPE_D, c, r, dd);
                    rec(TAPE_E, c, r, ee);
                }
                const double tpx = fma(0.5, bpx, Kc * apx), tux = fma(0.5, bux, cc * aux_);
                const double tpy = fma(0.5, bpy, Kc * apy), tvy = fma(0.5, bvy, cc * avy);
                dP[n] = fma(-lx, tpx, fma(-ly, tpy, sp[iq]));
                dU[n] = fma(-lx, tux, su[iq]);
                dV[n] = fma(-ly, tvy, sv[iq]);
            }
        }
        // D on the ghost rows -1, ty and E on the ghost columns -1, tx (transverse only)
        if (trans) {
            const int n = 2 * (tx + ty);
            for (int k = tid + (carry ? tx : 0); k < n; k += NT) {   // row -1 is carried
                if (k < 2 * tx) {
                    const int c = k % tx, r = (k < tx) ? -1 : ty;
                    const int ex = (r + 1) * G::XEW + (c + 1);
                    const double apx = A2x[ex] + A1x[ex + 1];
                    const double bpx = second ? Sx[(r + 1) * G::XLW + c + 1] - Sx[(r + 1) * G::XLW + c] : 0.0;
                    double d;
                    if (MED == 0) d = fma(kDx, bpx, apx);
                    else {
                        const double Kc = AX(AUX_K, c, r);
                        d = cw ? fma(Kc, apx, bpx) : Kc * apx;
                        rec(TAPE_D, c, r, d);
                    }
                    Dx[(r + 1) * G::DW + c] = d;
                } else {
                    const int kk = k - 2 * tx;
                    const int r = kk % ty, c = (kk < ty) ? -1 : tx;
                    const int ey = (r + 1) * G::YEW + (c + 1);
                    const double apy = B2y[ey] + B1y[ey + G::YEW];
                    const double bpy = second ? Sy[(r + 1) * G::YLW + c + 1] - Sy[r * G::YLW + c + 1] : 0.0;
                    double e;
                    if (MED == 0) e = fma(kDy, bpy, apy);
                    else {
                        const double Kc = AX(AUX_K, c, r);
                        e = cw ? fma(Kc, apy, bpy) : Kc * apy;
                        rec(TAPE_E, c, r, e);
                    }
                    Ey[r * G::EW + c + 1] = e;
                }
            }
        }
        // hand the top rows of the edge arrays to the next tile (none of them is written from
        // here to the end of the tile, but phase C2 reuses the strength arrays)
        if (hand) {
            for (int k = tid; k < G::C_D; k += NT) {
                const double* src;
                if (k < G::C_B) src = k < 2 * G::XEW ? A1x + ty * G::XEW + k : A2x + ty * G::XEW + (k - 2 * G::XEW);
                else if (k < G::C_S)
                    src = k < G::C_B + 3 * G::YEW ? B1y + ty * G::YEW + (k - G::C_B)
                                                  : B2y + ty * G::YEW + (k - G::C_B - 3 * G::YEW);
                else if (k < G::C_SY)
                    src = k < G::C_S + 2 * G::XLW ? Sx + ty * G::XLW + (k - G::C_S)
                                                  : Px + ty * G::XLW + (k - G::C_S - 2 * G::XLW);
                else src = k < G::C_SY + G::YLW ? Sy + ty * G::YLW + (k - G::C_SY) : Py + ty * G::YLW + (k - G::C_SY - G::YLW);
                Cy[k] = *src;
            }
        }
        __syncthreads();

        // ---------------------------------------------------------------- phase C2 (cell-wise medium):
        // transverse fluxes at the y-edges (from D) and the x-edges (from E); written over the
        // wave-strength arrays, which are dead now
        double* Gp = B1y;
        double* Gv = B2y;
        double* Fp = A1x;
        double* Fu = A2x;
        if (MED == 1 && trans) {
            {   // y-edge jj in [0, ty] of column c in [0, tx): lo = (c, jj-1), hi = (c, jj)
                const int n = (ty + 1) * tx;
                for (int k = tid; k < n; k += NT) {
                    const int jj = k / tx, c = k - jj * tx;
                    const double dlo = Dx[jj * G::DW + c], dhi = Dx[(jj + 1) * G::DW + c];
                    const double w = s_k[14] * AX(AUX_IYS, c, jj);
                    const double khi = AX(AUX_K, c, jj), klo = AX(AUX_K, c, jj - 1);
                    const double chi = AX(AUX_C, c, jj), clo = AX(AUX_C, c, jj - 1);
                    Gp[jj * TX + c] = w * fma(khi, dlo, -(klo * dhi));
                    Gv[jj * TX + c] = w * fma(chi, dlo, clo * dhi);
                }
            }
            {   // x-edge a in [0, tx] of row r in [0, ty): lo = (a-1, r), hi = (a, r)
                const int w1 = tx + 1, n = ty * w1;
                for (int k = tid; k < n; k += NT) {
                    const int r = k / w1, a = k - r * w1;
                    const double elo = Ey[r * G::EW + a], ehi = Ey[r * G::EW + a + 1];
                    const double w = s_k[15] * AX(AUX_IXS, a, r);
                    const double khi = AX(AUX_K, a, r), klo = AX(AUX_K, a - 1, r);
                    const double chi = AX(AUX_C, a, r), clo = AX(AUX_C, a - 1, r);
                    Fp[r * (TX + 1) + a] = w * fma(khi, elo, -(klo * ehi));
                    Fu[r * (TX + 1) + a] = w * fma(chi, elo, clo * ehi);
                }
            }
            __syncthreads();
        }

        // ---------------------------------------------------------------- phase D: update, store
        // one staging buffer: the tile's state was last read in phase C (behind the barrier
        // above), so the next tile's copy can land while this one finishes
        if (STAGE == 2 && tid == 0 && t + t_step < t_end) issue(t + t_step, 0);
        double kT = 0, kU = 0;
        if (MED == 0 && trans) {
            kT = s_k[10];
            kU = s_k[11];
        }
        // D of row ty - 1 becomes the next tile's row -1 (final since the barrier ending phase C)
        if (hand)
            for (int k = tid; k < G::DW; k += NT) Cy[G::C_D + k] = Dx[ty * G::DW + k];
        double* dst = A.qnew + P.qoff;
#pragma unroll
        for (int n = 0; n < NPER; ++n) {
            const int ci = tid + n * NT;
            const int c = ci % TX, r = ci / TX;
            if (ci >= TX * TY || c >= tx || r >= ty) continue;
            double p = dP[n], u = dU[n], v = dV[n];
            if (trans) {
                if (MED == 0) {
                    const double dn = Dx[(r + 2) * G::DW + c], ds = Dx[r * G::DW + c];
                    const double ee = Ey[r * G::EW + c + 2], ew = Ey[r * G::EW + c];
                    p = fma(kT, (dn + ds) + (ee + ew), p);   // kT holds -kT; 2 kT (dc + ec) is in p
                    u = fma(kU, ee - ew, u);
                    v = fma(kU, dn - ds, v);
                } else {
                    const double fpe = Fp[r * (TX + 1) + c + 1], fpw = Fp[r * (TX + 1) + c];
                    const double gpn = Gp[(r + 1) * TX + c], gps = Gp[r * TX + c];
                    p = fma(-lx, fpe - fpw, fma(-ly, gpn - gps, p));
                    u = fma(-lx, Fu[r * (TX + 1) + c + 1] - Fu[r * (TX + 1) + c], u);
                    v = fma(-ly, Gv[(r + 1) * TX + c] - Gv[r * TX + c], v);
                }
            }
            if (not_finite(p) | not_finite(u) | not_finite(v)) my_flag |= ERR_NAN;
            const long long o = (long long)(y0 + r + 2) * W + (x0 + c + 2);
            dst[o] = p;
            dst[WH + o] = u;
            dst[2 * WH + o] = v;
        }
        __syncthreads();   // the staged tile and work arrays are reused by the next tile
        if (tid == 0) {
            const unsigned long long m = s_tmax[it & 1];
            s_tmax[it & 1] = 0ull;   // next written two tiles later, after two more barriers
            if (P.run != cur_run) {
                flush();
                cur_run = P.run;
                cur_max = m;
            } else {
                cur_max = umax64(cur_max, m);
            }
        }
    }

    // ---------------------------------------------------------------- CFL and error flags
    if (tid == 0) flush();
    if (my_flag) atomicOr(&s_flag, my_flag);
    __syncthreads();
    if (tid == 0 && s_flag) atomicOr(A.err, s_flag);
    if (tid == 0) finish_cta(A);
}

}  // namespace claw

namespace claw {

// kernel pointer and dynamic shared memory of one configuration
struct StepKernel {
    void (*fn)(const StepArgs);
    size_t smem;        // dynamic shared memory of a launch that strides over the tiles
    int nt;
    size_t smem_walk;   // ... of a launch that walks tile columns (the carried rows added)
};

template <int MED, int LIM, int TX, int TY, int NT, int STAGE, int PULL, bool REC = false>
StepKernel step_kernel_entry()
{
    StepKernel k;
    k.fn = step_kernel<MED, LIM, TX, TY, NT, STAGE, PULL, REC>;
    k.smem = Geo<TX, TY>::smem_bytes(STAGE == 1 ? 2 : 1);
    k.nt = NT;
    k.smem_walk = MED == 1 ? k.smem : Geo<TX, TY>::smem_bytes(STAGE == 1 ? 2 : 1, true);
    return k;
}

// all tile shapes and stagings of one medium and limiter
// tile shapes x thread counts x stagings of one medium and limiter (nt = 0: the default)
template <int MED, int LIM, int PULL, bool REC = false>
StepKernel step_kernel_select(int tx, int ty, int nt, int staging)
{
    if (tx == 32 && ty == 32 && (nt == 0 || nt == 256))
        return staging ? step_kernel_entry<MED, LIM, 32, 32, 256, 1, PULL, REC>()
                       : step_kernel_entry<MED, LIM, 32, 32, 256, 0, PULL, REC>();
    if (tx == 32 && ty == 32 && nt == 512)
        return staging ? step_kernel_entry<MED, LIM, 32, 32, 512, 1, PULL, REC>()
                       : step_kernel_entry<MED, LIM, 32, 32, 512, 0, PULL, REC>();
    if (tx == 32 && ty == 16 && (nt == 0 || nt == 256)) {
        if (staging == 2) return step_kernel_entry<MED, LIM, 32, 16, 256, 2, PULL, REC>();
        return staging ? step_kernel_entry<MED, LIM, 32, 16, 256, 1, PULL, REC>()
                       : step_kernel_entry<MED, LIM, 32, 16, 256, 0, PULL, REC>();
    }
    if (tx == 16 && ty == 16 && (nt == 0 || nt == 128))
        return staging ? step_kernel_entry<MED, LIM, 16, 16, 128, 1, PULL, REC>()
                       : step_kernel_entry<MED, LIM, 16, 16, 128, 0, PULL, REC>();
    return StepKernel{nullptr, 0, 0, 0};
}

template <int MED, int PULL, bool REC = false>
StepKernel step_kernel_for(int lim, int tx, int ty, int nt, int staging)
{
    switch (lim) {
    case CLAW_LIM_NONE: return step_kernel_select<MED, CLAW_LIM_NONE, PULL, REC>(tx, ty, nt, staging);
    case CLAW_LIM_MINMOD: return step_kernel_select<MED, CLAW_LIM_MINMOD, PULL, REC>(tx, ty, nt, staging);
    case CLAW_LIM_SUPERBEE: return step_kernel_select<MED, CLAW_LIM_SUPERBEE, PULL, REC>(tx, ty, nt, staging);
    case CLAW_LIM_VANLEER: return step_kernel_select<MED, CLAW_LIM_VANLEER, PULL, REC>(tx, ty, nt, staging);
    case CLAW_LIM_MC: return step_kernel_select<MED, CLAW_LIM_MC, PULL, REC>(tx, ty, nt, staging);
    }
    return StepKernel{nullptr, 0, 0, 0};
}

// one translation unit per kernel family (pull: the instantiations taking pulled ghosts)
StepKernel step_kernel_uniform(int lim, int tx, int ty, int nt, int staging);
StepKernel step_kernel_uniform_pull(int lim, int tx, int ty, int nt, int staging);
StepKernel step_kernel_cellwise(int lim, int tx, int ty, int nt, int staging);
StepKernel step_kernel_cellwise_pull(int lim, int tx, int ty, int nt, int staging);
StepKernel step_kernel_uniform_interp(int lim, int tx, int ty, int nt, int staging);
StepKernel step_kernel_cellwise_interp(int lim, int tx, int ty, int nt, int staging);
StepKernel step_kernel_cellwise_record(int lim, int tx, int ty, int nt, int staging);
StepKernel step_kernel_cellwise_record_fill(int lim, int tx, int ty, int nt, int staging);
StepKernel step_kernel_swe(int lim, int tx, int ty, int nt, int staging);
StepKernel step_kernel_swe_pull(int lim, int tx, int ty, int nt, int staging);

}  // namespace claw

// claw_ghost.cu -- ghost fill (Sec. 2.2: physical boundary, same-level copy, coarse-to-fine
// space-time interpolation), "updating" average (Sec. 2.2-2.3), per-cell medium planes, the
// first-step CFL max and the device time-step rule (Eq. cfl), with their reverse modes.
// These are light, memory-bound kernels; the host builds compact task tables once per regrid
// (claw_set_level) so that each launch is a flat loop over tasks.
#include <cuda_runtime.h>

#include "claw_interp.cuh"

namespace claw {

static inline int div_up(long long a, int b) { return (int)((a + b - 1) / b); }

// ------------------------------------------------------------------------ same-level copy
// Block k copies the rectangles [start[k], start[k+1]) (the host groups consecutive
// rectangles, at most 32 rows each, into blocks of about 256 cells).  The block stages
// its rectangles in shared memory with the running element count, and every thread takes
// kCopyBatch elements of the flattened range with all loads issued before the stores (the
// copy is latency-bound: one dependent load-store pair per thread would leave HBM idle).
constexpr int kCopyThreads = 128;
constexpr int kCopyChunk = 32;
constexpr int kCopyBatch = 8;

struct CopyChunk {
    CopyRect r[kCopyChunk];
    int end[kCopyChunk];   // inclusive prefix of ncomp * w * h
    int n, total;
};

__device__ __forceinline__ void stage_chunk(CopyChunk& c, const CopyRect* __restrict__ rects, int r0, int n,
                                            int ncomp)
{
    const int tid = threadIdx.x;
    if (tid < n) c.r[tid] = rects[r0 + tid];
    __syncthreads();
    if (tid < 32) {   // warp-inclusive scan of the element counts
        int v = tid < n ? ncomp * c.r[tid].w * c.r[tid].h : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, v, o);
            if (tid >= o) v += u;
        }
        c.end[tid] = v;
        if (tid == 31) {
            c.total = v;
            c.n = n;
        }
    }
    __syncthreads();
}

// element k of the staged chunk -> (rectangle, component, x, y)
__device__ __forceinline__ void locate(const CopyChunk& c, int k, int& ri, int& m, int& x, int& y)
{
    ri = 0;
    while (c.end[ri] <= k) ++ri;
    const CopyRect& R = c.r[ri];
    const int e0 = k - (ri ? c.end[ri - 1] : 0);
    const int cells = R.w * R.h;
    m = e0 / cells;
    const int e = e0 - m * cells;
    y = e / R.w;
    x = e - y * R.w;
}

__device__ __forceinline__ bool negated(int flags, int m)
{
    return (m == 1 && (flags & 1)) || (m == 2 && (flags & 2));
}

__global__ void __launch_bounds__(kCopyThreads) fill_copy_kernel(const CopyRect* __restrict__ rects,
                                                                 const int* __restrict__ start,
                                                                 double* __restrict__ q, int ncomp)
{
    __shared__ CopyChunk c;
    const int r_lo = start[blockIdx.x], r_hi = start[blockIdx.x + 1];
    for (int r0 = r_lo; r0 < r_hi; r0 += kCopyChunk) {
        stage_chunk(c, rects, r0, min(kCopyChunk, r_hi - r0), ncomp);
        for (int base = 0; base < c.total; base += kCopyThreads * kCopyBatch) {
            double v[kCopyBatch];
            long long dst[kCopyBatch];
#pragma unroll
            for (int j = 0; j < kCopyBatch; ++j) {
                const int k = base + j * kCopyThreads + (int)threadIdx.x;
                dst[j] = -1;
                if (k < c.total) {
                    int ri, m, x, y;
                    locate(c, k, ri, m, x, y);
                    const CopyRect& R = c.r[ri];
                    const double s = q[R.src + m * R.splane + (long long)y * R.sy + (long long)x * R.sx];
                    v[j] = negated(R.flags, m) ? -s : s;
                    dst[j] = R.dst + m * R.dplane + (long long)y * R.dpitch + x;
                }
            }
#pragma unroll
            for (int j = 0; j < kCopyBatch; ++j)
                if (dst[j] >= 0) q[dst[j]] = v[j];
        }
        __syncthreads();   // the chunk is restaged
    }
}

// reverse: ghost adjoint flows into its source, then the ghost adjoint is cleared.  Sources
// are interior cells and several ghosts may share one (extrapolation), hence the atomics.
__global__ void __launch_bounds__(kCopyThreads) fill_copy_adjoint_kernel(const CopyRect* __restrict__ rects,
                                                                         const int* __restrict__ start,
                                                                         double* __restrict__ lam, int ncomp)
{
    __shared__ CopyChunk c;
    const int r_lo = start[blockIdx.x], r_hi = start[blockIdx.x + 1];
    for (int r0 = r_lo; r0 < r_hi; r0 += kCopyChunk) {
        stage_chunk(c, rects, r0, min(kCopyChunk, r_hi - r0), ncomp);
        for (int k = threadIdx.x; k < c.total; k += kCopyThreads) {
            int ri, m, x, y;
            locate(c, k, ri, m, x, y);
            const CopyRect& R = c.r[ri];
            const long long d = R.dst + m * R.dplane + (long long)y * R.dpitch + x;
            double g = lam[d];
            lam[d] = 0.0;
            if (negated(R.flags, m)) g = -g;
            if (g != 0.0) atomicAdd(&lam[R.src + m * R.splane + (long long)y * R.sy + (long long)x * R.sx], g);
        }
        __syncthreads();
    }
}

cudaError_t launch_fill_copy(const CopyRect* r, const int* start, int nblocks, double* q, cudaStream_t s, int ncomp)
{
    if (nblocks <= 0) return cudaSuccess;
    fill_copy_kernel<<<nblocks, kCopyThreads, 0, s>>>(r, start, q, ncomp);
    return cudaGetLastError();
}

cudaError_t launch_fill_copy_adjoint(const CopyRect* r, const int* start, int nblocks, double* lam, cudaStream_t s,
                                     int ncomp)
{
    if (nblocks <= 0) return cudaSuccess;
    fill_copy_adjoint_kernel<<<nblocks, kCopyThreads, 0, s>>>(r, start, lam, ncomp);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------ interpolation
__device__ __forceinline__ double sgn_of(int flags, int m) { return interp_sign(flags, m); }

// thread per (fine ghost cell, component)
__global__ void fill_interp_kernel(const InterpCell* __restrict__ cells, int n, double* __restrict__ q,
                                   const double* __restrict__ cold, const double* __restrict__ cnew,
                                   double tau)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= 3 * n) return;
    const int i = k / 3, m = k - 3 * i;
    const InterpCell C = cells[i];
    q[C.dst + m * C.dplane] = interp_value(C, m, cold, cnew, tau);
}

__global__ void fill_interp_adjoint_kernel(const InterpCell* __restrict__ cells, int n,
                                           double* __restrict__ lam, double* __restrict__ lco,
                                           double* __restrict__ lcn, const double* __restrict__ cold,
                                           const double* __restrict__ cnew, double tau)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= 3 * n) return;
    const int i = k / 3, m = k - 3 * i;
    const InterpCell C = cells[i];
    double Q[5], G[5] = {0, 0, 0, 0, 0};
    interp_coarse(C, m, cold, cnew, tau, Q);
    const long long d = C.dst + m * C.dplane;
    const double g = sgn_of(C.flags, m) * lam[d];
    lam[d] = 0.0;
    G[0] = g;
    // minmod branches as in the forward kernel
    double a = Q[2] - Q[0], b = Q[0] - Q[1];
    if (a * b > 0.0) {
        if (fabs(a) < fabs(b)) { G[2] += C.xi * g; G[0] -= C.xi * g; }
        else { G[0] += C.xi * g; G[1] -= C.xi * g; }
    }
    a = Q[4] - Q[0];
    b = Q[0] - Q[3];
    if (a * b > 0.0) {
        if (fabs(a) < fabs(b)) { G[4] += C.eta * g; G[0] -= C.eta * g; }
        else { G[0] += C.eta * g; G[3] -= C.eta * g; }
    }
#pragma unroll
    for (int s = 0; s < 5; ++s) {
        if (G[s] == 0.0) continue;
        const long long o = C.src[s] + m * C.splane[s];
        const double gs = sgn_of(C.sflags[s], m) * G[s];
        if (lco) atomicAdd(&lco[o], (1.0 - tau) * gs);
        if (lcn) atomicAdd(&lcn[o], tau * gs);
    }
}

cudaError_t launch_fill_interp(const InterpCell* c, int n, double* q, const double* cold,
                               const double* cnew, double tau, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    fill_interp_kernel<<<div_up(3LL * n, 256), 256, 0, s>>>(c, n, q, cold, cnew, tau);
    return cudaGetLastError();
}

cudaError_t launch_fill_interp_adjoint(const InterpCell* c, int n, double* lam, double* lco,
                                       double* lcn, const double* cold, const double* cnew,
                                       double tau, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    fill_interp_adjoint_kernel<<<div_up(3LL * n, 256), 256, 0, s>>>(c, n, lam, lco, lcn, cold, cnew, tau);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------ averaging
// block per rectangle, thread per (coarse cell, component); the r x r children are summed
// row by row and divided by r^2
__global__ void average_kernel(const AvgRect* __restrict__ rects, int ratio, const double* __restrict__ qf,
                               double* __restrict__ qc)
{
    const AvgRect R = rects[blockIdx.x];
    const int cells = R.w * R.h;
    const double rr = (double)(ratio * ratio);
    for (int k = threadIdx.x; k < 3 * cells; k += blockDim.x) {
        const int m = k / cells, e = k - m * cells;
        const int y = e / R.w, x = e - y * R.w;
        const double* f = qf + R.fsrc + m * R.fplane + (long long)y * ratio * R.fpitch + (long long)x * ratio;
        double s = 0.0;
        for (int b = 0; b < ratio; ++b)
            for (int a = 0; a < ratio; ++a) s += f[(long long)b * R.fpitch + a];
        qc[R.cdst + m * R.cplane + (long long)y * R.cpitch + x] = s / rr;
    }
}

__global__ void average_adjoint_kernel(const AvgRect* __restrict__ rects, int ratio, double* __restrict__ lf,
                                       double* __restrict__ lc)
{
    const AvgRect R = rects[blockIdx.x];
    const int cells = R.w * R.h;
    const double rr = (double)(ratio * ratio);
    for (int k = threadIdx.x; k < 3 * cells; k += blockDim.x) {
        const int m = k / cells, e = k - m * cells;
        const int y = e / R.w, x = e - y * R.w;
        const long long c = R.cdst + m * R.cplane + (long long)y * R.cpitch + x;
        const double g = lc[c] / rr;
        lc[c] = 0.0;
        double* f = lf + R.fsrc + m * R.fplane + (long long)y * ratio * R.fpitch + (long long)x * ratio;
        for (int b = 0; b < ratio; ++b)
            for (int a = 0; a < ratio; ++a) f[(long long)b * R.fpitch + a] += g;
    }
}

cudaError_t launch_average(const AvgRect* r, int n, int ratio, const double* qf, double* qc, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    average_kernel<<<n, 256, 0, s>>>(r, ratio, qf, qc);
    return cudaGetLastError();
}

cudaError_t launch_average_adjoint(const AvgRect* r, int n, int ratio, double* lf, double* lc, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    average_adjoint_kernel<<<n, 256, 0, s>>>(r, ratio, lf, lc);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------ medium planes
// block per box, thread per cell of the padded box
__global__ void medium_aux_kernel(const PatchDev* __restrict__ patches, const double* __restrict__ rho,
                                  const double* __restrict__ K, double* __restrict__ aux)
{
    const PatchDev P = patches[blockIdx.x];
    const int W = P.nx + 4, H = P.ny + 4;
    const int j0 = blockIdx.y * kBoxRows, j1 = min(H, j0 + kBoxRows);
    if (j0 >= H) return;
    const long long WH = (long long)W * H;
    const long long co = P.aoff / CLAW_NAUX;
    const double* r = rho + co;
    const double* k = K + co;
    double* a = aux + P.aoff;
    for (int e = j0 * W + threadIdx.x; e < j1 * W; e += blockDim.x) {
        const int j = e / W, i = e - j * W;
        const double z = sqrt(k[e] * r[e]), c = sqrt(k[e] / r[e]);
        a[AUX_Z * WH + e] = z;
        a[AUX_C * WH + e] = c;
        a[AUX_K * WH + e] = k[e];
        a[AUX_C2 * WH + e] = c * c;
        double ixs = 0, fx1 = 0, fx2 = 0, iys = 0, fy1 = 0, fy2 = 0;
        if (i > 0) {
            const double zw = sqrt(k[e - 1] * r[e - 1]);
            const double zz = fma(zw, z, 1.0);
            ixs = 1.0 / (zw + z);
            fx1 = zz / fma(zw, zw, 1.0);
            fx2 = zz / fma(z, z, 1.0);
        }
        if (j > 0) {
            const double zs = sqrt(k[e - W] * r[e - W]);
            const double zz = fma(zs, z, 1.0);
            iys = 1.0 / (zs + z);
            fy1 = zz / fma(zs, zs, 1.0);
            fy2 = zz / fma(z, z, 1.0);
        }
        a[AUX_IXS * WH + e] = ixs;
        a[AUX_FX1 * WH + e] = fx1;
        a[AUX_FX2 * WH + e] = fx2;
        a[AUX_IYS * WH + e] = iys;
        a[AUX_FY1 * WH + e] = fy1;
        a[AUX_FY2 * WH + e] = fy2;
    }
}

// chain rule through the planes above; each cell gathers from the planes that read it
// (itself, and the edges to its east and north), so no atomics are needed
__global__ void medium_aux_adjoint_kernel(const PatchDev* __restrict__ patches, const double* __restrict__ rho,
                                          const double* __restrict__ K, const double* __restrict__ ga,
                                          double* __restrict__ g_rho, double* __restrict__ g_K)
{
    const PatchDev P = patches[blockIdx.x];
    const int W = P.nx + 4, H = P.ny + 4;
    const int j0 = blockIdx.y * kBoxRows, j1 = min(H, j0 + kBoxRows);
    if (j0 >= H) return;
    const long long WH = (long long)W * H;
    const long long co = P.aoff / CLAW_NAUX;
    const double* r = rho + co;
    const double* k = K + co;
    const double* g = ga + P.aoff;
    for (int e = j0 * W + threadIdx.x; e < j1 * W; e += blockDim.x) {
        const int j = e / W, i = e - j * W;
        const double z = sqrt(k[e] * r[e]), c = sqrt(k[e] / r[e]);
        // dZ/dK = Z/(2K), dZ/drho = Z/(2 rho), dc/dK = c/(2K), dc/drho = -c/(2 rho)
        double gz = g[AUX_Z * WH + e];
        double gc = g[AUX_C * WH + e] + 2.0 * c * g[AUX_C2 * WH + e];
        double gk = g[AUX_K * WH + e];
        // edge to the west / south of this cell (this cell is the "right" cell)
        auto edge_right = [&](int ip, int po, int p1, int p2, int e2) {
            const double zw = sqrt(k[e2] * r[e2]);
            const double zz = fma(zw, z, 1.0), s = zw + z;
            const double d1 = fma(zw, zw, 1.0), d2 = fma(z, z, 1.0);
            // ixs = 1/s ; fx1 = zz/d1 ; fx2 = zz/d2  -> derivatives w.r.t. z (this cell); the ixs
            // plane holds ixs times its adjoint: d(1/s)/dz x adjoint = -(1/s^2) (s x plane) = -plane / s
            gz += -g[ip * WH + e] / s + g[p1 * WH + e] * (zw / d1) +
                  g[p2 * WH + e] * (zw / d2 - zz * 2.0 * z / (d2 * d2));
            (void)po;
        };
        auto edge_left = [&](int ip, int p1, int p2, int e2) {
            // the cell to the east / north owns the edge; this cell is its "left" cell
            const double zr = sqrt(k[e2] * r[e2]);
            const double zz = fma(z, zr, 1.0), s = z + zr;
            const double d1 = fma(z, z, 1.0), d2 = fma(zr, zr, 1.0);
            gz += -g[ip * WH + e2] / s + g[p1 * WH + e2] * (zr / d1 - zz * 2.0 * z / (d1 * d1)) +
                  g[p2 * WH + e2] * (zr / d2);
        };
        if (i > 0) edge_right(AUX_IXS, 0, AUX_FX1, AUX_FX2, e - 1);
        if (j > 0) edge_right(AUX_IYS, 0, AUX_FY1, AUX_FY2, e - W);
        if (i + 1 < W) edge_left(AUX_IXS, AUX_FX1, AUX_FX2, e + 1);
        if (j + 1 < H) edge_left(AUX_IYS, AUX_FY1, AUX_FY2, e + W);
        g_K[co + e] += gk + gz * z / (2.0 * k[e]) + gc * c / (2.0 * k[e]);
        g_rho[co + e] += gz * z / (2.0 * r[e]) - gc * c / (2.0 * r[e]);
    }
}

static inline dim3 box_rows_grid(int n, int max_rows)
{
    return dim3((unsigned)n, (unsigned)((max_rows + kBoxRows - 1) / kBoxRows));
}

// ------------------------------------------------------------------------ packed interiors
// block (box b0 + x, chunk y of kBoxRows interior rows): the chunk's 3 x rows x nx cells between
// the box's padded planes and its packed planes (3 planes of nx x ny at poff[b])
__global__ void pack_kernel(const PatchDev* __restrict__ patches, const long long* __restrict__ poff, int b0,
                            double* __restrict__ q, double* __restrict__ packed, int unpack)
{
    const int b = b0 + (int)blockIdx.x;
    const PatchDev P = patches[b];
    const int r0 = blockIdx.y * kBoxRows;
    if (r0 >= P.ny) return;
    const int rows = min(P.ny, r0 + kBoxRows) - r0;
    const int W = P.nx + 4;
    const long long WH = (long long)W * (P.ny + 4), NN = (long long)P.nx * P.ny;
    const long long base = poff[b];
    const int per = rows * P.nx, n = 3 * per;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const int m = k / per, e = k - m * per;
        const int r = r0 + e / P.nx, i = e % P.nx;
        const long long qo = P.qoff + m * WH + (long long)(r + 2) * W + (i + 2);
        const long long po = base + m * NN + (long long)r * P.nx + i;
        if (unpack) q[qo] = packed[po];
        else packed[po] = q[qo];
    }
}

cudaError_t launch_pack(const PatchDev* p, const long long* poff, int b0, int b1, int max_rows, double* q,
                        double* packed, int unpack, cudaStream_t s)
{
    if (b1 <= b0) return cudaSuccess;
    pack_kernel<<<box_rows_grid(b1 - b0, max_rows), 256, 0, s>>>(p, poff, b0, q, packed, unpack);
    return cudaGetLastError();
}

cudaError_t launch_medium_aux(const PatchDev* p, int n, int max_rows, const double* rho, const double* K,
                              double* aux, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    medium_aux_kernel<<<box_rows_grid(n, max_rows), 128, 0, s>>>(p, rho, K, aux);
    return cudaGetLastError();
}

cudaError_t launch_medium_aux_adjoint(const PatchDev* p, int n, int max_rows, const double* rho, const double* K,
                                      const double* g_aux, double* g_rho, double* g_K, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    medium_aux_adjoint_kernel<<<box_rows_grid(n, max_rows), 128, 0, s>>>(p, rho, K, g_aux, g_rho, g_K);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------ CFL
// block per (box, chunk of rows): max c over the ring [-1, nx] x [-1, ny] (integer max of the
// bit patterns), one 64-bit atomic max per warp on the run's scalar (zeroed by the host first)
__global__ void cfl_max_kernel(const PatchDev* __restrict__ patches, int medium, double c0,
                               const double* __restrict__ aux, unsigned long long* __restrict__ smax)
{
    const PatchDev P = patches[blockIdx.x];
    unsigned long long m = 0ull;
    const int r0 = blockIdx.y * kBoxRows, r1 = min(P.ny + 2, r0 + kBoxRows);   // ring rows, from -1
    if (r0 >= P.ny + 2) return;
    if (medium == 0) {
        m = (unsigned long long)__double_as_longlong(c0);
    } else {
        const int W = P.nx + 4;
        const double* c = aux + P.aoff + AUX_C * (long long)W * (P.ny + 4);
        const int w = P.nx + 2, n = w * (r1 - r0);
        for (int k = threadIdx.x; k < n; k += blockDim.x) {
            const int r = r0 + k / w, i = k % w;
            const unsigned long long v = (unsigned long long)__double_as_longlong(c[(r + 1) * W + (i + 1)]);
            m = v > m ? v : m;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long v = __shfl_xor_sync(0xffffffffu, m, o);
        m = v > m ? v : m;
    }
    if ((threadIdx.x & 31) == 0 && m) atomicMax(smax + P.run, m);
}

cudaError_t launch_cfl_max(const PatchDev* p, int n, int max_rows, int medium, double c0, const double* aux,
                           double* smax, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    cfl_max_kernel<<<box_rows_grid(n, max_rows), 128, 0, s>>>(p, medium, c0, aux,
                                                            reinterpret_cast<unsigned long long*>(smax));
    return cudaGetLastError();
}

// the same ring for shallow water: max of |u| + sqrt(g h), |v| + sqrt(g h) from the state
__global__ void cfl_max_state_kernel(const PatchDev* __restrict__ patches, double grav,
                                     const double* __restrict__ q, unsigned long long* __restrict__ smax)
{
    const PatchDev P = patches[blockIdx.x];
    unsigned long long m = 0ull;
    const int r0 = blockIdx.y * kBoxRows, r1 = min(P.ny + 2, r0 + kBoxRows);
    if (r0 >= P.ny + 2) return;
    const int W = P.nx + 4;
    const long long WH = (long long)W * (P.ny + 4);
    const double* b = q + P.qoff;
    const int w = P.nx + 2, n = w * (r1 - r0);
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const int r = r0 + k / w, i = k % w;
        const long long o = (long long)(r + 1) * W + (i + 1);
        const double h = b[o];
        const double c = sqrt(grav * h);
        const double su = fabs(b[WH + o] / h) + c, sv = fabs(b[2 * WH + o] / h) + c;
        const unsigned long long vu = (unsigned long long)__double_as_longlong(su);
        const unsigned long long vv = (unsigned long long)__double_as_longlong(sv);
        m = vu > m ? vu : m;
        m = vv > m ? vv : m;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long v = __shfl_xor_sync(0xffffffffu, m, o);
        m = v > m ? v : m;
    }
    if ((threadIdx.x & 31) == 0 && m) atomicMax(smax + P.run, m);
}

cudaError_t launch_cfl_max_state(const PatchDev* p, int n, int max_rows, double grav, const double* q,
                                 double* smax, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    cfl_max_state_kernel<<<box_rows_grid(n, max_rows), 128, 0, s>>>(p, grav, q,
                                                                  reinterpret_cast<unsigned long long*>(smax));
    return cudaGetLastError();
}

// ------------------------------------------------------------------------ time step (Eq. cfl)
__global__ void dt_update_kernel(const double* __restrict__ minh, const double* __restrict__ cfl, int nruns,
                                 double* __restrict__ smax, double* __restrict__ dt, int* __restrict__ err)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nruns) return;
    const double s = smax[r];
    const double used = dt[r];
    // CFL number of the step just taken (Sec. 2.4): nu = s dt / dx must not exceed 1
    if (s * used > minh[r] * (1.0 + 1e-12)) atomicOr(err, ERR_CFL);
    if (s > 0.0) dt[r] = cfl[r] * minh[r] / s;
    smax[r] = 0.0;
}

cudaError_t launch_dt_update(const double* minh, const double* cfl, int nruns, double* smax, double* dt,
                             int* err, cudaStream_t s)
{
    dt_update_kernel<<<div_up(nruns, 128), 128, 0, s>>>(minh, cfl, nruns, smax, dt, err);
    return cudaGetLastError();
}

}  // namespace claw

// claw_regrid.cu -- device parts of regridding (Sec. 2.2): the refinement flags of a level and the
// copy of old fine values into a new fine pool.  Clustering runs on the host (claw_api.cu); the
// interpolation of new fine cells from the coarse level reuses the ghost interpolation kernel.
#include <cuda_runtime.h>

#include "claw_internal.h"

namespace claw {
namespace {

// thread per interior cell (block: box x row chunk): flagged when some component differs from a
// face neighbour by more than tol (ghosts of q filled)
__global__ void flag_kernel(const FlagBox* __restrict__ boxes, const double* __restrict__ q, double tol,
                            unsigned char* __restrict__ flags)
{
    const FlagBox B = boxes[blockIdx.x];
    const int j0 = blockIdx.y * kBoxRows, j1 = min(B.ny, j0 + kBoxRows);
    if (j0 >= B.ny) return;
    const int W = B.nx + 4;
    const long long WH = (long long)W * (B.ny + 4);
    for (int k = threadIdx.x; k < (j1 - j0) * B.nx; k += blockDim.x) {
        const int j = j0 + k / B.nx, i = k % B.nx;
        const long long o = B.qoff + (long long)(j + 2) * W + (i + 2);
        bool f = false;
        for (int m = 0; m < 3; ++m) {
            const double* p = q + o + m * WH;
            const double c = p[0];
            f |= fabs(p[1] - c) > tol;
            f |= fabs(p[-1] - c) > tol;
            f |= fabs(p[W] - c) > tol;
            f |= fabs(p[-W] - c) > tol;
        }
        flags[B.goff + (long long)j * B.pitch + i] = f ? 1 : 0;
    }
}

__global__ void rect_copy_kernel(const RectCopy* __restrict__ c, const double* __restrict__ src,
                                 double* __restrict__ dst)
{
    const RectCopy C = c[blockIdx.x];
    const int cells = C.w * C.h;
    for (int k = threadIdx.x; k < 3 * cells; k += blockDim.x) {
        const int m = k / cells, e = k - m * cells;
        const int y = e / C.w, x = e - y * C.w;
        dst[C.dst + m * C.dplane + (long long)y * C.dpitch + x] = src[C.src + m * C.splane + (long long)y * C.spitch + x];
    }
}

__device__ __forceinline__ double minmod2(double a, double b)
{
    if (!(a * b > 0.0)) return 0.0;
    return fabs(a) < fabs(b) ? a : b;
}

// conservative space interpolation (minmod-limited slopes) of each fine cell of a run from its
// coarse cell and the four face neighbours, read from the coarse box's padded planes (ghosts filled)
__global__ void interp_runs_kernel(const InterpRun* __restrict__ runs, const double* __restrict__ qc,
                                   double* __restrict__ qf)
{
    const InterpRun R = runs[blockIdx.x];
    for (int k = threadIdx.x; k < 3 * R.n; k += blockDim.x) {
        const int m = k / R.n, t = k - m * R.n;
        const int gi = R.gi0 + t;
        const int I = gi >= 0 ? gi / R.r : -((-gi + R.r - 1) / R.r);
        const int J = R.gj >= 0 ? R.gj / R.r : -((-R.gj + R.r - 1) / R.r);
        const double* c = qc + R.cbase + m * R.cplane + (long long)(J - R.cjlo + 2) * R.cpitch + (I - R.cilo + 2);
        const double q0 = c[0];
        const double sx = minmod2(c[1] - q0, q0 - c[-1]);
        const double sy = minmod2(c[R.cpitch] - q0, q0 - c[-R.cpitch]);
        const double xi = ((double)(gi - I * R.r) + 0.5) / R.r - 0.5;
        const double eta = ((double)(R.gj - J * R.r) + 0.5) / R.r - 0.5;
        qf[R.dst + m * R.dplane + t] = q0 + xi * sx + eta * sy;
    }
}

}  // namespace

cudaError_t launch_flags(const FlagBox* boxes, int nb, int max_rows, const double* q, double tol,
                         unsigned char* flags, cudaStream_t s)
{
    if (nb <= 0) return cudaSuccess;
    flag_kernel<<<dim3((unsigned)nb, (unsigned)((max_rows + kBoxRows - 1) / kBoxRows)), 128, 0, s>>>(boxes, q, tol,
                                                                                                      flags);
    return cudaGetLastError();
}

cudaError_t launch_rect_copy(const RectCopy* c, int n, const double* src, double* dst, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    rect_copy_kernel<<<n, 128, 0, s>>>(c, src, dst);
    return cudaGetLastError();
}

cudaError_t launch_interp_runs(const InterpRun* r, int n, const double* qc, double* qf, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    interp_runs_kernel<<<n, 128, 0, s>>>(r, qc, qf);
    return cudaGetLastError();
}

}  // namespace claw

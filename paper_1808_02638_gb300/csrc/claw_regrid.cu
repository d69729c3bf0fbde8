// claw_regrid.cu -- device parts of regridding (Sec. 2.2): the refinement flags of a level and the
// transfer into a new fine pool (old fine values where an old box had them, conservative
// interpolation from the coarse level elsewhere).  Clustering runs on the host
// (claw_clustering.cu).
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

__device__ __forceinline__ double minmod2(double a, double b)
{
    if (!(a * b > 0.0)) return 0.0;
    return fabs(a) < fabs(b) ? a : b;
}

// each cell of box b (block: box x row chunk) writes the box's index into the run's grid
__global__ void paint_kernel(const XferBox* __restrict__ boxes, const long long* __restrict__ goff,
                             const int* __restrict__ pitch, int* __restrict__ grid)
{
    const XferBox B = boxes[blockIdx.x];
    const int j0 = blockIdx.y * kBoxRows, j1 = min(B.ny, j0 + kBoxRows);
    if (j0 >= B.ny) return;
    int* g = grid + goff[B.run] + (long long)B.jlo * pitch[B.run] + B.ilo;
    for (int k = threadIdx.x; k < (j1 - j0) * B.nx; k += blockDim.x) {
        const int j = j0 + k / B.nx, i = k % B.nx;
        g[(long long)j * pitch[B.run] + i] = (int)blockIdx.x;
    }
}

// every cell of a new fine box: the old fine box's value where one covered the cell, else the
// conservative space interpolation (minmod-limited slopes) from its coarse cell and the four face
// neighbours, read from the coarse box's padded planes (ghosts filled)
__global__ void transfer_kernel(const XferBox* __restrict__ nb, const XferBox* __restrict__ ob,
                                const XferBox* __restrict__ cb, int r, XferGrids g, const double* __restrict__ q_old,
                                const double* __restrict__ qc, double* __restrict__ q_new, int* __restrict__ err)
{
    const XferBox B = nb[blockIdx.x];
    const int j0 = blockIdx.y * kBoxRows, j1 = min(B.ny, j0 + kBoxRows);
    if (j0 >= B.ny) return;
    const long long dplane = (long long)(B.nx + 4) * (B.ny + 4);
    for (int k = threadIdx.x; k < (j1 - j0) * B.nx; k += blockDim.x) {
        const int j = j0 + k / B.nx, i = k % B.nx;
        const int gi = B.ilo + i, gj = B.jlo + j;
        double* dst = q_new + B.qoff + (long long)(j + 2) * (B.nx + 4) + (i + 2);
        const int o = g.fgrid[g.fgoff[B.run] + (long long)gj * g.fpitch[B.run] + gi];
        if (o >= 0) {
            const XferBox O = ob[o];
            const long long splane = (long long)(O.nx + 4) * (O.ny + 4);
            const double* src = q_old + O.qoff + (long long)(gj - O.jlo + 2) * (O.nx + 4) + (gi - O.ilo + 2);
            for (int m = 0; m < 3; ++m) dst[m * dplane] = src[m * splane];
            continue;
        }
        const int I = gi / r, J = gj / r;   // level indices are non-negative
        const int c = g.cgrid[g.cgoff[B.run] + (long long)J * g.cpitch[B.run] + I];
        if (c < 0) {   // not properly nested: reported, the cell left as it is
            atomicOr(err, 1);
            continue;
        }
        const XferBox C = cb[c];
        const int cp = C.nx + 4;
        const long long cplane = (long long)cp * (C.ny + 4);
        const double xi = ((double)(gi - I * r) + 0.5) / r - 0.5;
        const double eta = ((double)(gj - J * r) + 0.5) / r - 0.5;
        for (int m = 0; m < 3; ++m) {
            const double* p = qc + C.qoff + m * cplane + (long long)(J - C.jlo + 2) * cp + (I - C.ilo + 2);
            const double q0 = p[0];
            const double sx = minmod2(p[1] - q0, q0 - p[-1]);
            const double sy = minmod2(p[cp] - q0, q0 - p[-cp]);
            dst[m * dplane] = fma(eta, sy, fma(xi, sx, q0));
        }
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

cudaError_t launch_regrid_transfer(const XferBox* nb, int n_new, const XferBox* ob, int n_old, const XferBox* cb,
                                   int n_coarse, int max_rows, int ratio, const XferGrids& g, long long fcells,
                                   long long ccells, const double* q_old, const double* q_coarse, double* q_new,
                                   int* err, cudaStream_t s)
{
    if (n_new <= 0) return cudaSuccess;
    const unsigned chunks = (unsigned)((max_rows + kBoxRows - 1) / kBoxRows);
    cudaError_t e = cudaMemsetAsync(g.fgrid, 0xff, (size_t)fcells * sizeof(int), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(g.cgrid, 0xff, (size_t)ccells * sizeof(int), s);
    if (e != cudaSuccess) return e;
    if (n_old > 0) paint_kernel<<<dim3((unsigned)n_old, chunks), 128, 0, s>>>(ob, g.fgoff, g.fpitch, g.fgrid);
    if (n_coarse > 0) paint_kernel<<<dim3((unsigned)n_coarse, chunks), 128, 0, s>>>(cb, g.cgoff, g.cpitch, g.cgrid);
    transfer_kernel<<<dim3((unsigned)n_new, chunks), 128, 0, s>>>(nb, ob, cb, ratio, g, q_old, q_coarse, q_new, err);
    return cudaGetLastError();
}

}  // namespace claw

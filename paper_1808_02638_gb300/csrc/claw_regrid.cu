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

__global__ void cell_copy_kernel(const CellCopy* __restrict__ c, int n, const double* __restrict__ src,
                                 double* __restrict__ dst)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const CellCopy C = c[k];
    for (int m = 0; m < 3; ++m) dst[C.dst + m * C.dplane] = src[C.src + m * C.splane];
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

cudaError_t launch_cell_copy(const CellCopy* c, int n, const double* src, double* dst, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    cell_copy_kernel<<<(n + 127) / 128, 128, 0, s>>>(c, n, src, dst);
    return cudaGetLastError();
}

}  // namespace claw

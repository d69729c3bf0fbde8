// claw_noalloc.cu -- claw_level_step_noalloc: the fused level-step for a single box without
// any device allocation.
//
// The regular entry points keep their tile and patch tables in device memory that
// claw_set_level allocates.  Some callers cannot allocate device memory at the point where
// they want to step: code running while a stream is being captured into a CUDA graph (an
// allocation there breaks the capture), code embedded in a host application that hands
// every byte of device memory to its own pool allocator, or a real-time loop that cannot
// afford the implicit device synchronisation of cudaMalloc / cudaFree.  This entry point
// serves them: its scratch (the patch descriptor, the tile table and an error word) lives in
// a fixed file-scope device array, so a call only launches kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "claw_internal.h"

namespace claw {
namespace {

// Scratch of every call on a device: 256 KiB (16367 tiles), held by every device that loads the library
// until the process exits.  Layout: [0, 64) error word, [64, 256) the box descriptor,
// [256, end) the tile table.
constexpr size_t kScratchBytes = 256 * 1024;
constexpr size_t kHeader = 256;
constexpr int kTile = 32;
constexpr int kMaxTiles = (int)((kScratchBytes - kHeader) / sizeof(TileDev));
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

static_assert(sizeof(PatchDev) <= kHeader - 64, "box descriptor must fit the header");

// device address of the scratch array on each device, looked up once per device
void* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

cudaError_t scratch_address(int dev, void** out)
{
    std::lock_guard<std::mutex> g(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        // the array's name is a host-side stand-in: only this call yields the device address
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

// writes the box descriptor and the tile table and clears the error word: the array keeps
// the previous call's contents, so nothing in it is trusted without being rewritten here
__global__ void noalloc_setup_kernel(unsigned char* s, int nx, int ny, double dxinv, double dyinv, int ntx,
                                     int ntiles)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k == 0) {
        *reinterpret_cast<int*>(s) = 0;
        PatchDev* P = reinterpret_cast<PatchDev*>(s + 64);
        P->qoff = 0;
        P->aoff = 0;
        P->nx = nx;
        P->ny = ny;
        P->run = 0;
        P->ring = -1;
        P->dxinv = dxinv;
        P->dyinv = dyinv;
        P->dtscale = 1.0;
    }
    if (k < ntiles) {
        TileDev* T = reinterpret_cast<TileDev*>(s + kHeader) + k;
        const int bx = k % ntx, by = k / ntx;
        T->patch = 0;
        T->x0 = (short)(bx * kTile);
        T->y0 = (short)(by * kTile);
        T->tx = (short)min(kTile, nx - bx * kTile);
        T->ty = (short)min(kTile, ny - by * kTile);
        T->flags = 0;
    }
}

}  // namespace
}  // namespace claw

using namespace claw;

extern "C" int claw_level_step_noalloc(int32_t nx, int32_t ny, double dx, double dy, int32_t limiter, int32_t order,
                                       int32_t transverse, double rho0, double K0, const double* q_old,
                                       double* q_new, const double* aux, const double* dt, double* smax,
                                       void* stream)
{
    if (nx < 1 || ny < 1 || nx > 4096 || ny > 4096 || !(dx > 0) || !(dy > 0) || limiter < 0 || limiter > 4 ||
        order < 1 || order > 2 || transverse < 0 || transverse > 2 || !q_old || !q_new || !dt || !smax ||
        q_old == q_new)
        return CLAW_EINVAL;
    if (!aux && !(rho0 > 0 && K0 > 0)) return CLAW_EINVAL;
    const int ntx = (nx + kTile - 1) / kTile, nty = (ny + kTile - 1) / kTile;
    if ((long long)ntx * nty > kMaxTiles) return CLAW_EINVAL;   // beyond the fixed scratch
    const int ntiles = ntx * nty;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return CLAW_ECUDA;
    void* sp = nullptr;
    if (scratch_address(dev, &sp) != cudaSuccess) return CLAW_ECUDA;
    unsigned char* s = static_cast<unsigned char*>(sp);
    cudaStream_t st = (cudaStream_t)stream;
    noalloc_setup_kernel<<<(ntiles + 255) / 256, 256, 0, st>>>(s, nx, ny, 1.0 / dx, 1.0 / dy, ntx, ntiles);
    if (cudaGetLastError() != cudaSuccess) return CLAW_ECUDA;
    int nsm = 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return CLAW_ECUDA;
    const int medium = aux ? 1 : 0;
    const int per_sm = step_max_ctas_per_sm(medium, limiter, kTile, kTile, 0, 0);
    if (per_sm <= 0) return CLAW_ECUDA;
    StepArgs a;
    a.patches = reinterpret_cast<const PatchDev*>(s + 64);
    a.tiles = reinterpret_cast<const TileDev*>(s + kHeader);
    a.tmaps = nullptr;
    a.ntiles = ntiles;
    a.qold = q_old;
    a.qnew = q_new;
    a.aux = aux;
    a.dt = dt;
    a.smax = smax;
    a.err = reinterpret_cast<int*>(s);
    a.order = order;
    a.transverse = transverse;
    a.rho0 = rho0;
    a.K0 = K0;
    const int grid = std::min(ntiles, per_sm * nsm);
    return launch_step(a, medium, limiter, kTile, kTile, 0, 0, grid, st) == cudaSuccess ? CLAW_OK : CLAW_ECUDA;
}

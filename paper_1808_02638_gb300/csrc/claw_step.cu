// Dispatch of the fused level-step kernels (instantiated in claw_step_uniform.cu,
// claw_step_cellwise.cu and claw_step_swe.cu).
#include <algorithm>
#include <mutex>
#include <set>

#include "claw_step.cuh"

namespace claw {

static StepKernel pick(int kind, int limiter, int tx, int ty, int nt, int staging, bool pull, bool rec = false,
                       bool interp = false)
{
    if (interp) {   // acoustics only; shallow water takes the interpolation launch first (claw_api.cu)
        if (!pull || rec) return StepKernel{nullptr, 0, 0};
        if (kind == KIND_UNIFORM) return step_kernel_uniform_interp(limiter, tx, ty, nt, staging);
        if (kind == KIND_CELLWISE) return step_kernel_cellwise_interp(limiter, tx, ty, nt, staging);
        return StepKernel{nullptr, 0, 0};
    }
    if (rec) {
        if (kind != KIND_CELLWISE) return StepKernel{nullptr, 0, 0};
        return pull ? step_kernel_cellwise_record(limiter, tx, ty, nt, staging)
                    : step_kernel_cellwise_record_fill(limiter, tx, ty, nt, staging);
    }
    switch (kind) {
    case KIND_UNIFORM:
        return pull ? step_kernel_uniform_pull(limiter, tx, ty, nt, staging)
                    : step_kernel_uniform(limiter, tx, ty, nt, staging);
    case KIND_CELLWISE:
        return pull ? step_kernel_cellwise_pull(limiter, tx, ty, nt, staging)
                    : step_kernel_cellwise(limiter, tx, ty, nt, staging);
    case KIND_SWE:
        return pull ? step_kernel_swe_pull(limiter, tx, ty, nt, staging) : step_kernel_swe(limiter, tx, ty, nt, staging);
    }
    return StepKernel{nullptr, 0, 0};
}

static cudaError_t prepare(const StepKernel& k)
{
    // opt in to the dynamic shared memory once per kernel and device
    static std::mutex mu;
    static std::set<std::pair<const void*, int>> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> g(mu);
    auto key = std::make_pair((const void*)k.fn, dev);
    if (done.count(key)) return cudaSuccess;
    e = cudaFuncSetAttribute((const void*)k.fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)std::max(k.smem, k.smem_walk));
    if (e == cudaSuccess) done.insert(key);
    return e;
}

int step_max_ctas_per_sm(int kind, int limiter, int tx, int ty, int nt, int staging, bool pull, bool rec, bool interp,
                         bool walk)
{
    StepKernel k = pick(kind, limiter, tx, ty, nt, staging, pull, rec, interp);
    if (!k.fn || prepare(k) != cudaSuccess) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, (const void*)k.fn, k.nt, walk ? k.smem_walk : k.smem) !=
        cudaSuccess)
        return 0;
    return n;
}

cudaError_t launch_step(const StepArgs& a, int kind, int limiter, int tx, int ty, int nt, int staging,
                        int grid, cudaStream_t s, int spare)
{
    StepKernel k = pick(kind, limiter, tx, ty, nt, staging, a.ring != nullptr, a.tape != nullptr, a.interp != nullptr);
    if (!k.fn) return cudaErrorInvalidValue;
    cudaError_t e = prepare(k);
    if (e != cudaSuccess) return e;
    long long items = 0;   // (ghost cell, component) pairs of the fill jobs
    for (int j = 0; j < a.nfill; ++j) items += 3LL * a.fills[j].n;
    if (items > 0) {
        // one pair per thread where `spare` CTAs allow, else those CTAs stride over them
        StepArgs b = a;
        b.step_grid = grid;
        const int extra = (int)std::min<long long>((items + k.nt - 1) / k.nt, std::max(spare, 1));
        k.fn<<<grid + extra, k.nt, a.tcum ? k.smem_walk : k.smem, s>>>(b);
    } else {
        k.fn<<<grid, k.nt, a.tcum ? k.smem_walk : k.smem, s>>>(a);
    }
    return cudaGetLastError();
}

template <int L>
__global__ void limiter_eval_kernel(long long n, const double* a, const double* b, double* out)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = Lim<L>::f(__ldg(a + i), __ldg(b + i));
}

cudaError_t launch_limiter_eval(int limiter, long long n, const double* a, const double* b, double* out,
                                cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    const int grid = (int)std::min<long long>((n + 255) / 256, 4096);
    switch (limiter) {
    case CLAW_LIM_NONE: limiter_eval_kernel<CLAW_LIM_NONE><<<grid, 256, 0, s>>>(n, a, b, out); break;
    case CLAW_LIM_MINMOD: limiter_eval_kernel<CLAW_LIM_MINMOD><<<grid, 256, 0, s>>>(n, a, b, out); break;
    case CLAW_LIM_SUPERBEE: limiter_eval_kernel<CLAW_LIM_SUPERBEE><<<grid, 256, 0, s>>>(n, a, b, out); break;
    case CLAW_LIM_VANLEER: limiter_eval_kernel<CLAW_LIM_VANLEER><<<grid, 256, 0, s>>>(n, a, b, out); break;
    case CLAW_LIM_MC: limiter_eval_kernel<CLAW_LIM_MC><<<grid, 256, 0, s>>>(n, a, b, out); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace claw

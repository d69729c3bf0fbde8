// Instantiations of the fused level-step for a uniform medium (rho0, K0).
#include "claw_step.cuh"

namespace claw {
StepKernel step_kernel_uniform(int lim, int tx, int ty, int nt, int staging)
{
    return step_kernel_for<0, 0>(lim, tx, ty, nt, staging);
}
}  // namespace claw

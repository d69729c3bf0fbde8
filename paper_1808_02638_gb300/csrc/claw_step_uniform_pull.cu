// Instantiations of the fused level-step for a uniform medium that take pulled ghosts.
#include "claw_step.cuh"

namespace claw {
StepKernel step_kernel_uniform_pull(int lim, int tx, int ty, int nt, int staging)
{
    return step_kernel_for<0, 1>(lim, tx, ty, nt, staging);
}
}  // namespace claw

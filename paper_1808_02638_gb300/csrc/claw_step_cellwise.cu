// Instantiations of the fused level-step for a cell-wise medium (aux planes).
#include "claw_step.cuh"

namespace claw {
StepKernel step_kernel_cellwise(int lim, int tx, int ty, int nt, int staging)
{
    return step_kernel_for<1, 0>(lim, tx, ty, nt, staging);
}
}  // namespace claw

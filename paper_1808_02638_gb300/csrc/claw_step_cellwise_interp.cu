// Instantiations of the fused level-step (cell-wise medium) that pull the same-level and boundary ghosts
// and evaluate the ghosts interpolated from the coarser level inside the step.
#include "claw_step.cuh"

namespace claw {
StepKernel step_kernel_cellwise_interp(int lim, int tx, int ty, int nt, int staging)
{
    return step_kernel_for<1, 2>(lim, tx, ty, nt, staging);
}
}  // namespace claw

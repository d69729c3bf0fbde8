// Instantiations of the fused level-step (uniform medium) that pull the same-level and boundary ghosts
// and evaluate the ghosts interpolated from the coarser level inside the step.
#include "claw_step.cuh"

namespace claw {
StepKernel step_kernel_uniform_interp(int lim, int tx, int ty, int nt, int staging)
{
    return step_kernel_for<0, 2>(lim, tx, ty, nt, staging);
}
}  // namespace claw

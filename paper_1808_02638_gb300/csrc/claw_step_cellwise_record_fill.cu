// Instantiations of the recording level-step (cell-wise medium) that read every ghost from the
// pool (filled by the ghost-copy launch first), for levels that step without pulled ghosts.
#include "claw_step.cuh"

namespace claw {
StepKernel step_kernel_cellwise_record_fill(int lim, int tx, int ty, int nt, int staging)
{
    return step_kernel_for<1, 0, true>(lim, tx, ty, nt, staging);
}
}  // namespace claw

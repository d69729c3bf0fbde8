// Instantiations of the recording level-step (cell-wise medium, pulled ghosts): the step that
// also writes its intermediates to the tape the tape-driven adjoint reads.
#include "claw_step.cuh"

namespace claw {
StepKernel step_kernel_cellwise_record(int lim, int tx, int ty, int nt, int staging)
{
    return step_kernel_for<1, 1, true>(lim, tx, ty, nt, staging);
}
}  // namespace claw

// claw_adjoint.cu -- reverse mode of the fused level-step (filled in below).
#include "claw_internal.h"

namespace claw {
cudaError_t launch_step_adjoint(const StepArgs&, double*, double*, int, int, int, int, int, cudaStream_t)
{
    return cudaErrorNotSupported;
}
}  // namespace claw

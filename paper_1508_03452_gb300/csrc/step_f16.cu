// step_f16.cu -- instantiation of the fused time step for CfgF16.
#include "step_impl.cuh"

namespace lb {
template cudaError_t launch_step<CfgF16>(const StepArgs<CfgF16>&, cudaStream_t);
}  // namespace lb

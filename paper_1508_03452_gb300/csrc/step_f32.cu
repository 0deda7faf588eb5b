// step_f32.cu -- instantiation of the fused time step for CfgF32.
#include "step_impl.cuh"

namespace lb {
template cudaError_t launch_step<CfgF32>(const StepArgs<CfgF32>&, cudaStream_t);
}  // namespace lb

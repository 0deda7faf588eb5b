// step_f64.cu -- instantiation of the fused time step for CfgF64.
#include "step_impl.cuh"

namespace lb {
template cudaError_t launch_step<CfgF64>(const StepArgs<CfgF64>&, cudaStream_t);
}  // namespace lb

// step_f32.cu -- instantiation of the fused time step for CfgF32.
#include "step_impl.cuh"

namespace lb {
template cudaError_t launch_step<CfgF32>(const StepArgs<CfgF32>&, cudaStream_t, const TileMaps*);
template cudaError_t launch_step_batch<CfgF32>(const unsigned char*, const int4*, int, int, int, bool, int, bool,
                                                  cudaStream_t);
template int batch_blocks_per_sm<CfgF32>(bool, int, bool);
}  // namespace lb

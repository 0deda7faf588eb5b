// step_f16.cu -- instantiation of the fused time step for CfgF16.
#include "step_impl.cuh"

namespace lb {
template cudaError_t launch_step<CfgF16>(const StepArgs<CfgF16>&, cudaStream_t, const TileLaunch*);
template cudaError_t launch_step_batch<CfgF16>(const unsigned char*, const int4*, int, int, int, bool, int, bool,
                                                  cudaStream_t);
template int batch_blocks_per_sm<CfgF16>(bool, int, bool);
template cudaError_t launch_step_persistent<CfgF16>(const unsigned char*, size_t, int, const int4*, int, int, int, int,
                                                     bool, int, bool, unsigned int*, int*, unsigned long long,
                                                     cudaStream_t);
template int persistent_blocks_per_sm<CfgF16>(bool, int, bool);
}  // namespace lb

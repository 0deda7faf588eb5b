// step_f32.cu -- instantiation of the fused time step for CfgF32.
#include "step_impl.cuh"

namespace lb {
template cudaError_t launch_step<CfgF32>(const StepArgs<CfgF32>&, cudaStream_t, const TileLaunch*);
template cudaError_t launch_step_batch<CfgF32>(const unsigned char*, const int4*, int, int, int, bool, int, bool,
                                                  cudaStream_t);
template int batch_blocks_per_sm<CfgF32>(bool, int, bool);
template cudaError_t launch_step_persistent<CfgF32>(const unsigned char*, size_t, int, const int4*, int, int, int, int,
                                                     bool, int, bool, unsigned int*, int*, unsigned long long,
                                                     cudaStream_t);
template int persistent_blocks_per_sm<CfgF32>(bool, int, bool);

// A grid barrier that waits for one arrival more than the grid has when
// `unreachable`: the check that the persistent launch's bounded wait gives up
// and raises its status bit instead of spinning on.
__global__ void barrier_selftest_kernel(unsigned int* counter, int* status, int unreachable,
                                        unsigned long long wait_ns)
{
    grid_barrier(counter, gridDim.x + (unreachable ? 1u : 0u), status, wait_ns);
}

cudaError_t launch_barrier_selftest(int blocks, unsigned int* counter, int* status, int unreachable,
                                    unsigned long long wait_ns, cudaStream_t stream)
{
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(64);
    cfg.stream = stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, barrier_selftest_kernel, counter, status, unreachable, wait_ns);
}
}  // namespace lb

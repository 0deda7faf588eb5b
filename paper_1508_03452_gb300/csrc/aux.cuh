// aux.cuh -- declarations shared by the host API and the auxiliary kernels.
#pragma once

#include "common.cuh"
#include "tma.cuh"

namespace lb {

// one buffer set (current state) of one run
template <class Cfg>
struct PopView {
    typename Cfg::pop* fg;  // f and g in the group order of fg_elem
    typename Cfg::hpop* h;  // h in the pair order of h_elem
    typename Cfg::prim* prim;
    int nx, ny, nz;
    int64_t stride;
    int periodic[3];
    HalfScale hs;
};

// device float64 input fields of lbrmhd_init_fields (E may be NULL)
struct InitInputs {
    const double* n;
    const double* p;
    const double* u;
    const double* B;
    const double* E;
};

// absolute reference rest equilibrium populations (added back on output)
struct RefPops {
    double f[19], g[19], h[25];
};

struct RefState {
    double n_r, eps_r, p_r;
};

constexpr int NPART = 9;
constexpr int NMEANS = 23;  // entries of the reference-state means
constexpr int kMeansThreads = 256, kMeansBlocks = 608;
constexpr int kDiagThreads = 256;

// block-wide reduction of NPART float64 values (index 6 is a max, the others
// sums); thread 0 writes dst[blockIdx.x * NPART + j]
__device__ __forceinline__ void block_reduce_partials(double* v, double* dst)
{
    __shared__ double sh[kDiagThreads / 32][NPART];
    for (int j = 0; j < NPART; ++j)
        for (int o = 16; o > 0; o >>= 1) {
            const double other = __shfl_down_sync(0xffffffffu, v[j], o);
            v[j] = (j == 6) ? fmax(v[j], other) : v[j] + other;
        }
    const int w = threadIdx.x / 32, lane = threadIdx.x % 32;
    if (lane == 0)
        for (int j = 0; j < NPART; ++j) sh[w][j] = v[j];
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int j = 0; j < NPART; ++j) {
            double acc = sh[0][j];
            for (int ww = 1; ww < (int)(blockDim.x / 32); ++ww) acc = (j == 6) ? fmax(acc, sh[ww][j]) : acc + sh[ww][j];
            dst[(int64_t)blockIdx.x * NPART + j] = acc;
        }
    }
}

// one step of one run; `tl` (or NULL) describes the run's tiled launch for its
// input buffer, which lets 2-D periodic runs take the TMA tile kernel
template <class Cfg>
cudaError_t launch_step(const StepArgs<Cfg>& A, cudaStream_t stream, const TileLaunch* tl);
template <class Cfg>
cudaError_t launch_step_batch(const unsigned char* d_args, const int4* d_tiles, int ntiles, int bx, int grid,
                              bool is3d, int seed, bool open, cudaStream_t stream);
template <class Cfg>
int batch_blocks_per_sm(bool is3d, int seed, bool open);
// nsteps steps of every run of one kernel variant in one cooperative launch
// (grid-wide barrier between steps; *counter zero on entry)
template <class Cfg>
cudaError_t launch_step_persistent(const unsigned char* d_args, size_t parity_bytes, int in0, const int4* d_tiles,
                                   int ntiles, int bx, int nsteps, int grid, bool is3d, int seed, bool open,
                                   unsigned int* counter, int* status, unsigned long long wait_ns,
                                   cudaStream_t stream);
template <class Cfg>
int persistent_blocks_per_sm(bool is3d, int seed, bool open);
// a cooperative grid of `blocks` blocks meeting at a grid barrier that never
// completes when `unreachable` (the bounded wait's self-test)
cudaError_t launch_barrier_selftest(int blocks, unsigned int* counter, int* status, int unreachable,
                                    unsigned long long wait_ns, cudaStream_t stream);
template <class Cfg>
cudaError_t launch_null(const PopView<Cfg>& V, int y_lo, int y_hi, const typename Cfg::prim* ez0, double B0,
                        double* scratch, int64_t scratch_doubles, double* out, cudaStream_t s);
// device stride of the per-run argument records of the batched kernel
template <class Cfg>
constexpr size_t batch_args_stride()
{
    return (sizeof(StepArgs<Cfg>) + 15) / 16 * 16;
}
template <class Cfg>
cudaError_t launch_init(const PopView<Cfg>& V, const InitInputs& in, const Phys<double>& k, int* bad, cudaStream_t s);
cudaError_t launch_means(const InitInputs& in, int64_t N, double* partial, double* out, cudaStream_t s);
template <class Cfg>
cudaError_t launch_boundaries(const PopView<Cfg>& V, const Phys<typename Cfg::real>& k, const int* bc, int layers,
                              const double* drive_uv, cudaStream_t s);
// the drive velocity of every (x, y) column (2 float64 each) for a driven run
cudaError_t launch_drive_profile(int nx, int ny, double u0, double* uv, cudaStream_t s);
template <class Cfg>
cudaError_t launch_moments(const PopView<Cfg>& V, const Phys<double>& k, double* out, cudaStream_t s);
// primitive component P (a P_ index) of every cell into out (N values of the primitive type)
template <class Cfg>
cudaError_t launch_prim_component(const PopView<Cfg>& V, int P, typename Cfg::prim* out, cudaStream_t s);
// max |u|^2 of a state into out[0], out[1] = 0 (body-force cut-off)
template <class Cfg>
cudaError_t launch_umax_state(const PopView<Cfg>& V, double* out, cudaStream_t s);
// after a step of a run with a cut-off: u[0] = u[1], u[1] = 0
cudaError_t launch_umax_roll(double* u, cudaStream_t s);
// E of a state into the two history planes of the relaxed initialisation
template <class Cfg>
cudaError_t launch_relax_history(const PopView<Cfg>& V, double* e, cudaStream_t s);
template <class Cfg>
cudaError_t launch_populations(const PopView<Cfg>& V, const RefPops& ref, double* f, double* g, double* h,
                               cudaStream_t s);
template <class Cfg>
cudaError_t launch_diag(const PopView<Cfg>& V, const Phys<double>& k, const RefState& r, double* partial,
                        int64_t max_blocks, double* out, cudaStream_t s);

}  // namespace lb

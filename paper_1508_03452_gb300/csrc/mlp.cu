// mlp.cu -- training and standalone inference kernels of the learned recovery
// seed (see mlp.cuh), and their C-ABI entry points.
//
// Training runs in float32 on the CUDA cores: one warp per sample (two
// neurons per lane). Each warp accumulates its own gradient copy in shared
// memory (the lanes of a warp update disjoint entries, so no atomics); a block
// sums its warps' copies in warp order and the blocks' partial sums are added
// in block order, so a gradient (and a training run) is bit-reproducible. Samples are
// rows of 24 float32: 20 features then 4 targets (beta, eps / T^00 - 1).
// Loss: mean over samples of the squared error summed over the 4 outputs.
#include <cuda_runtime.h>
#include <stdint.h>

#include "lbrmhd.h"
#include "mlp.cuh"

namespace lb {

constexpr int MLP_ROW = MLP_IN + MLP_OUT;
static_assert(MLP_NPARAM == LBRMHD_MLP_NPARAM && MLP_IN == LBRMHD_MLP_NFEAT && MLP_ROW == LBRMHD_MLP_ROW,
              "network layout differs from the C ABI");
constexpr int kTrainWarps = 4;
constexpr int kTrainSmem = (kTrainWarps * MLP_NPARAM + kTrainWarps * 6 * MLP_H + kTrainWarps) * 4;

__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t x)
{
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

// Per-block loss and gradient of `count` samples. Sample j of the batch is
// row (sample_seed ? hash(sample_seed, j) mod n : first + j).
__global__ void __launch_bounds__(32 * kTrainWarps) mlp_grad_kernel(const float* __restrict__ P,
                                                                    const float* __restrict__ data, int64_t n,
                                                                    int64_t first, int64_t count, uint64_t sample_seed,
                                                                    float* __restrict__ partial, float inv_count)
{
    // dynamic shared memory: per-warp gradient copies, then per-warp
    // activations (x, h1, h2, h3) and deltas (2 x 64), then per-warp loss
    extern __shared__ float smem_f[];
    const int w = threadIdx.x / 32, lane = threadIdx.x % 32;
    float* sG = smem_f + w * MLP_NPARAM;
    float* sh = smem_f + kTrainWarps * MLP_NPARAM + w * 6 * MLP_H;
    float* sl = smem_f + kTrainWarps * MLP_NPARAM + kTrainWarps * 6 * MLP_H;
    for (int i = threadIdx.x; i < kTrainWarps * MLP_NPARAM; i += blockDim.x) smem_f[i] = 0.0f;
    if (lane == 0) sl[w] = 0.0f;
    __syncthreads();
    // parameters are read through the read-only cache
    const float* W1 = P + MLP_W1;
    const float* b1 = P + MLP_B1;
    const float* W2 = P + MLP_W2;
    const float* b2 = P + MLP_B2;
    const float* W3 = P + MLP_W3;
    const float* b3 = P + MLP_B3;
    const float* W4 = P + MLP_W4;
    const float* b4 = P + MLP_B4;
    float* x = sh;
    float* h1 = sh + MLP_H;
    float* h2 = sh + 2 * MLP_H;
    float* h3 = sh + 3 * MLP_H;
    float* d3 = sh + 4 * MLP_H;
    float* d2 = sh + 5 * MLP_H;
    const int64_t gw = (int64_t)blockIdx.x * kTrainWarps + w, nw = (int64_t)gridDim.x * kTrainWarps;
    for (int64_t j = gw; j < count; j += nw) {
        const int64_t row = sample_seed ? (int64_t)(splitmix64(sample_seed ^ (uint64_t)j * 0x2545F4914F6CDD1Dull) %
                                                    (uint64_t)n)
                                        : first + j;
        const float* s = data + row * MLP_ROW;
        if (lane < MLP_IN) x[lane] = s[lane];
        __syncwarp();
        // forward
        for (int q = 0; q < 2; ++q) {
            const int o = lane + 32 * q;
            float a = b1[o];
            for (int k = 0; k < MLP_IN; ++k) a += W1[o * MLP_IN + k] * x[k];
            h1[o] = fmaxf(a, 0.0f);
        }
        __syncwarp();
        for (int q = 0; q < 2; ++q) {
            const int o = lane + 32 * q;
            float a = b2[o];
            for (int k = 0; k < MLP_H; ++k) a += W2[o * MLP_H + k] * h1[k];
            h2[o] = fmaxf(a, 0.0f);
        }
        __syncwarp();
        for (int q = 0; q < 2; ++q) {
            const int o = lane + 32 * q;
            float a = b3[o];
            for (int k = 0; k < MLP_H; ++k) a += W3[o * MLP_H + k] * h2[k];
            h3[o] = fmaxf(a, 0.0f);
        }
        __syncwarp();
        float dy[MLP_OUT];
        float loss = 0.0f;
        for (int o = 0; o < MLP_OUT; ++o) {
            float a = b4[o];
            for (int k = 0; k < MLP_H; ++k) a += W4[o * MLP_H + k] * h3[k];
            const float e = a - s[MLP_IN + o];
            loss += e * e;
            dy[o] = 2.0f * e * inv_count;
        }
        if (lane == 0) sl[w] += loss * inv_count;
        // backward: output layer
        for (int q = 0; q < 2; ++q) {
            const int k = lane + 32 * q;
            float g = 0.0f;
            for (int o = 0; o < MLP_OUT; ++o) {
                sG[MLP_W4 + o * MLP_H + k] += dy[o] * h3[k];
                g += W4[o * MLP_H + k] * dy[o];
            }
            d3[k] = h3[k] > 0.0f ? g : 0.0f;
        }
        if (lane < MLP_OUT) sG[MLP_B4 + lane] += dy[lane];
        __syncwarp();
        // layer 3
        for (int q = 0; q < 2; ++q) {
            const int o = lane + 32 * q;
            sG[MLP_B3 + o] += d3[o];
            for (int k = 0; k < MLP_H; ++k) sG[MLP_W3 + o * MLP_H + k] += d3[o] * h2[k];
        }
        for (int q = 0; q < 2; ++q) {
            const int k = lane + 32 * q;
            float g = 0.0f;
            for (int o = 0; o < MLP_H; ++o) g += W3[o * MLP_H + k] * d3[o];
            d2[k] = h2[k] > 0.0f ? g : 0.0f;
        }
        __syncwarp();
        // layer 2
        for (int q = 0; q < 2; ++q) {
            const int o = lane + 32 * q;
            sG[MLP_B2 + o] += d2[o];
            for (int k = 0; k < MLP_H; ++k) sG[MLP_W2 + o * MLP_H + k] += d2[o] * h1[k];
        }
        for (int q = 0; q < 2; ++q) {
            const int k = lane + 32 * q;
            float g = 0.0f;
            for (int o = 0; o < MLP_H; ++o) g += W2[o * MLP_H + k] * d2[o];
            d3[k] = h1[k] > 0.0f ? g : 0.0f;  // reuse d3 as the layer-1 delta
        }
        __syncwarp();
        // layer 1
        for (int q = 0; q < 2; ++q) {
            const int o = lane + 32 * q;
            sG[MLP_B1 + o] += d3[o];
            for (int k = 0; k < MLP_IN; ++k) sG[MLP_W1 + o * MLP_IN + k] += d3[o] * x[k];
        }
        __syncwarp();
    }
    __syncthreads();
    float* out = partial + (int64_t)blockIdx.x * (MLP_NPARAM + 1);
    for (int i = threadIdx.x; i < MLP_NPARAM; i += blockDim.x) {
        float g = 0.0f;
        for (int q = 0; q < kTrainWarps; ++q) g += smem_f[q * MLP_NPARAM + i];
        out[i] = g;
    }
    if (threadIdx.x == 0) {
        float l = 0.0f;
        for (int q = 0; q < kTrainWarps; ++q) l += sl[q];
        out[MLP_NPARAM] = l;
    }
}

// sums the per-block partials in block order: grad[i] (and loss at index NPARAM)
__global__ void mlp_reduce_kernel(const float* __restrict__ partial, int nblocks, float* __restrict__ grad)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > MLP_NPARAM) return;
    float s = 0.0f;
    for (int b = 0; b < nblocks; ++b) s += partial[(int64_t)b * (MLP_NPARAM + 1) + i];
    grad[i] = s;
}

// Adam: m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2, p -= lr mhat / (sqrt(vhat) + eps)
__global__ void mlp_adam_kernel(float* __restrict__ P, float* __restrict__ m, float* __restrict__ v,
                                const float* __restrict__ g, float lr, float b1, float b2, float eps, float c1,
                                float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= MLP_NPARAM) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    P[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// float32 parameters -> bf16 inference blob in fragment order (zero padding)
__global__ void mlp_pack_kernel(const float* __restrict__ P, unsigned char* __restrict__ blob)
{
    __nv_bfloat16* W = reinterpret_cast<__nv_bfloat16*>(blob);
    float* bias = reinterpret_cast<float*>(blob + MLPD_NBF16 * 2);
    const int total = MLP_H * MLP_K1 + 2 * MLP_H * MLP_H + 8 * MLP_H + MLPD_NBIAS;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        // i enumerates (layer, r, k) in row-major order, then the biases
        if (i < MLP_H * MLP_K1) {
            const int r = i / MLP_K1, k = i % MLP_K1;
            W[MLPD_W1 + mlpd_frag_index(r, k, MLP_K1)] =
                __float2bfloat16_rn(k < MLP_IN ? P[MLP_W1 + r * MLP_IN + k] : 0.0f);
        } else if (i < MLP_H * MLP_K1 + MLP_H * MLP_H) {
            const int j = i - MLP_H * MLP_K1, r = j / MLP_H, k = j % MLP_H;
            W[MLPD_W2 + mlpd_frag_index(r, k, MLP_H)] = __float2bfloat16_rn(P[MLP_W2 + r * MLP_H + k]);
        } else if (i < MLP_H * MLP_K1 + 2 * MLP_H * MLP_H) {
            const int j = i - MLP_H * MLP_K1 - MLP_H * MLP_H, r = j / MLP_H, k = j % MLP_H;
            W[MLPD_W3 + mlpd_frag_index(r, k, MLP_H)] = __float2bfloat16_rn(P[MLP_W3 + r * MLP_H + k]);
        } else if (i < MLP_H * MLP_K1 + 2 * MLP_H * MLP_H + 8 * MLP_H) {
            const int j = i - MLP_H * MLP_K1 - 2 * MLP_H * MLP_H, r = j / MLP_H, k = j % MLP_H;
            W[MLPD_W4 + mlpd_frag_index(r, k, MLP_H)] =
                __float2bfloat16_rn(r < MLP_OUT ? P[MLP_W4 + r * MLP_H + k] : 0.0f);
        } else {
            const int j = i - (MLP_H * MLP_K1 + 2 * MLP_H * MLP_H + 8 * MLP_H);
            float val = 0.0f;
            if (j < 64) val = P[MLP_B1 + j];
            else if (j < 128) val = P[MLP_B2 + j - 64];
            else if (j < 192) val = P[MLP_B3 + j - 128];
            else if (j < 192 + MLP_OUT) val = P[MLP_B4 + j - 192];
            bias[j] = val;
        }
    }
}

// standalone inference with the same tensor-core device code as the step
// kernel (128 threads = 128 samples per block; tail lanes use a zero row)
__global__ void __launch_bounds__(128) mlp_infer_kernel(const unsigned char* __restrict__ blob,
                                                        const float* __restrict__ feat, int64_t n,
                                                        float* __restrict__ out)
{
    __shared__ __align__(16) __nv_bfloat16 act[128 * MLP_HS];
    __shared__ float out_f[128 * 8];
    const int tid = threadIdx.x;
    const int64_t s = (int64_t)blockIdx.x * 128 + tid;
    __nv_bfloat16* row = act + tid * MLP_HS;
    for (int j = 0; j < 32; j += 2) {
        const float a = (s < n && j < MLP_IN) ? feat[s * MLP_IN + j] : 0.0f;
        const float b = (s < n && j + 1 < MLP_IN) ? feat[s * MLP_IN + j + 1] : 0.0f;
        *reinterpret_cast<__nv_bfloat162*>(row + j) = __floats2bfloat162_rn(a, b);
    }
    __syncwarp();
    mlp_forward_warp(act, blob, out_f);
    if (s < n)
        for (int o = 0; o < MLP_OUT; ++o) out[s * MLP_OUT + o] = out_f[tid * 8 + o];
}

}  // namespace lb

namespace {
bool train_configured()
{
    static bool ok = cudaFuncSetAttribute(lb::mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          lb::kTrainSmem) == cudaSuccess;
    return ok;
}

int g_train_blocks(int64_t count)
{
    const int64_t per = 4 * lb::kTrainWarps;  // samples per block and pass
    int64_t b = (count + per - 1) / per;
    return (int)(b < 1 ? 1 : (b > 1216 ? 1216 : b));
}
}  // namespace

extern "C" {

int lbrmhd_mlp_nparams(void) { return lb::MLP_NPARAM; }

int lbrmhd_mlp_blob_bytes(void) { return lb::MLPD_BYTES; }

int lbrmhd_mlp_pack(const float* d_params, void* d_blob, void* stream)
{
    if (!d_params || !d_blob) return LBRMHD_ERR_BAD_ARG;
    lb::mlp_pack_kernel<<<32, 256, 0, (cudaStream_t)stream>>>(d_params, (unsigned char*)d_blob);
    return cudaGetLastError() == cudaSuccess ? LBRMHD_OK : LBRMHD_ERR_CUDA;
}

int lbrmhd_mlp_infer(const void* d_blob, const float* d_features, int64_t n, float* d_out, void* stream)
{
    if (!d_blob || !d_features || !d_out || n < 0) return LBRMHD_ERR_BAD_ARG;
    if (n == 0) return LBRMHD_OK;
    lb::mlp_infer_kernel<<<(unsigned)((n + 127) / 128), 128, 0, (cudaStream_t)stream>>>(
        (const unsigned char*)d_blob, d_features, n, d_out);
    return cudaGetLastError() == cudaSuccess ? LBRMHD_OK : LBRMHD_ERR_CUDA;
}

int lbrmhd_mlp_grad(const float* d_params, const float* d_data, int64_t n, float* d_grad, void* stream)
{
    if (!d_params || !d_data || !d_grad || n < 1) return LBRMHD_ERR_BAD_ARG;
    const int nb = g_train_blocks(n);
    float* partial = nullptr;
    if (cudaMalloc(&partial, (size_t)nb * (lb::MLP_NPARAM + 1) * sizeof(float)) != cudaSuccess) return LBRMHD_ERR_OOM;
    cudaStream_t s = (cudaStream_t)stream;
    if (!train_configured()) {
        cudaFree(partial);
        return LBRMHD_ERR_CUDA;
    }
    lb::mlp_grad_kernel<<<nb, 32 * lb::kTrainWarps, lb::kTrainSmem, s>>>(d_params, d_data, n, 0, n, 0, partial,
                                                                          1.0f / (float)n);
    lb::mlp_reduce_kernel<<<(lb::MLP_NPARAM + 256) / 256, 256, 0, s>>>(partial, nb, d_grad);
    const cudaError_t e1 = cudaGetLastError();
    const cudaError_t e2 = cudaStreamSynchronize(s);
    cudaFree(partial);
    return (e1 == cudaSuccess && e2 == cudaSuccess) ? LBRMHD_OK : LBRMHD_ERR_CUDA;
}

int lbrmhd_mlp_train(float* d_params, float* d_adam, const float* d_data, int64_t n, int steps, int batch, float lr,
                     uint64_t seed, float* d_loss, void* stream)
{
    if (!d_params || !d_adam || !d_data || n < 1 || steps < 0 || batch < 1 || !(lr > 0)) return LBRMHD_ERR_BAD_ARG;
    const int nb = g_train_blocks(batch);
    float *partial = nullptr, *grad = nullptr;
    if (cudaMalloc(&partial, (size_t)nb * (lb::MLP_NPARAM + 1) * sizeof(float)) != cudaSuccess) return LBRMHD_ERR_OOM;
    if (cudaMalloc(&grad, (lb::MLP_NPARAM + 1) * sizeof(float)) != cudaSuccess) {
        cudaFree(partial);
        return LBRMHD_ERR_OOM;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (!train_configured()) {
        cudaFree(partial);
        cudaFree(grad);
        return LBRMHD_ERR_CUDA;
    }
    const float b1 = 0.9f, b2 = 0.999f;
    float c1 = 1.0f, c2 = 1.0f;
    for (int t = 0; t < steps; ++t) {
        c1 *= b1;
        c2 *= b2;
        lb::mlp_grad_kernel<<<nb, 32 * lb::kTrainWarps, lb::kTrainSmem, s>>>(
            d_params, d_data, n, 0, batch, lb::splitmix64(seed + (uint64_t)t + 1) | 1ull, partial, 1.0f / (float)batch);
        lb::mlp_reduce_kernel<<<(lb::MLP_NPARAM + 256) / 256, 256, 0, s>>>(partial, nb, grad);
        lb::mlp_adam_kernel<<<(lb::MLP_NPARAM + 255) / 256, 256, 0, s>>>(d_params, d_adam, d_adam + lb::MLP_NPARAM,
                                                                          grad, lr, b1, b2, 1e-8f, 1.0f - c1,
                                                                          1.0f - c2);
        if (d_loss) cudaMemcpyAsync(d_loss + t, grad + lb::MLP_NPARAM, sizeof(float), cudaMemcpyDeviceToDevice, s);
    }
    const cudaError_t e1 = cudaGetLastError();
    const cudaError_t e2 = cudaStreamSynchronize(s);
    cudaFree(partial);
    cudaFree(grad);
    return (e1 == cudaSuccess && e2 == cudaSuccess) ? LBRMHD_OK : LBRMHD_ERR_CUDA;
}

}  // extern "C"

// mlp.cuh -- the learned seed of the primitive recovery: a 20-64-64-64-4 ReLU
// network mapping normalised moments to the velocity (and eps / T^00 - 1).
// It only supplies the starting vector of the Landau eigen-solve; the solve
// itself (and its result) is the method's.
//
// Parameters (float32 master copy, MLP_NPARAM values): W1[64][20] b1[64]
// W2[64][64] b2[64] W3[64][64] b3[64] W4[4][64] b4[4], W[out][in].
//
// Inference inside the step kernel uses warp-level bf16 tensor-core MMA
// (mma.sync m16n8k16, float32 accumulation) on shared-memory tiles: each warp
// owns the 32 cells (rows) of its threads, so no block-wide barrier is needed.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace lb {

constexpr int MLP_IN = 20, MLP_H = 64, MLP_OUT = 4;
constexpr int MLP_W1 = 0, MLP_B1 = MLP_W1 + MLP_H * MLP_IN, MLP_W2 = MLP_B1 + MLP_H,
              MLP_B2 = MLP_W2 + MLP_H * MLP_H, MLP_W3 = MLP_B2 + MLP_H, MLP_B3 = MLP_W3 + MLP_H * MLP_H,
              MLP_W4 = MLP_B3 + MLP_H, MLP_B4 = MLP_W4 + MLP_OUT * MLP_H, MLP_NPARAM = MLP_B4 + MLP_OUT;

// padded bf16 layout for the tensor-core path (row strides chosen so the 8
// rows read by one MMA fragment fall in distinct shared-memory banks)
constexpr int MLP_XS = 40;  // row stride (bf16) of a 32-wide input / W1 row
constexpr int MLP_HS = 72;  // row stride (bf16) of a 64-wide activation / weight row
constexpr int MLPD_W1 = 0, MLPD_W2 = MLPD_W1 + MLP_H * MLP_XS, MLPD_W3 = MLPD_W2 + MLP_H * MLP_HS,
              MLPD_W4 = MLPD_W3 + MLP_H * MLP_HS, MLPD_NBF16 = MLPD_W4 + 8 * MLP_HS;
constexpr int MLPD_NBIAS = 3 * MLP_H + 8;                                // float32 biases after the bf16 block
constexpr int MLPD_BYTES = MLPD_NBF16 * 2 + MLPD_NBIAS * 4;              // device inference blob
constexpr int MLP_ACT_BYTES_PER_CELL = MLP_HS * 2;                       // shared activation row per cell

// normalised features of one cell: T^{mu nu} / T^00 (9), N^a / N^0 (3),
// N^0 / T^00, E_old / sqrt(T^00) (3), B_old / sqrt(T^00) (3), 1
template <class R>
__device__ __forceinline__ void mlp_features(R T00, const R* T0a, const R* Tab /* xx yy zz xy xz yz */, R N0,
                                             const R* Na, const R* E_old, const R* B_old, float* x)
{
    const R it = R(1) / T00;
    const R is = sqrt(it);
    for (int a = 0; a < 3; ++a) x[a] = (float)(T0a[a] * it);
    for (int m = 0; m < 6; ++m) x[3 + m] = (float)(Tab[m] * it);
    const R in = R(1) / N0;
    for (int a = 0; a < 3; ++a) x[9 + a] = (float)(Na[a] * in);
    x[12] = (float)(N0 * it);
    for (int a = 0; a < 3; ++a) {
        x[13 + a] = (float)(E_old[a] * is);
        x[16 + a] = (float)(B_old[a] * is);
    }
    x[19] = 1.0f;
}

__device__ __forceinline__ uint32_t ld_b32(const __nv_bfloat16* p) { return *reinterpret_cast<const uint32_t*>(p); }
__device__ __forceinline__ uint32_t ldg_b32(const __nv_bfloat16* p) { return __ldg(reinterpret_cast<const unsigned int*>(p)); }

__device__ __forceinline__ void mma_bf16(float* d, const uint32_t* a, const uint32_t* b)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// One dense layer for the 32 rows owned by this warp: act[r][0..NOUT) =
// f(act[r][0..K) . W^T + bias), in place (all reads of a row block finish
// before its writes). `row0` is the warp's first row; `ldin` / `ldw` strides.
template <int K, int NOUT, bool RELU, bool TO_FLOAT>
__device__ __forceinline__ void mlp_layer(__nv_bfloat16* act, int ld, const __nv_bfloat16* W, int ldw,
                                          const float* bias, int row0, float* out_f)
{
    const int lane = threadIdx.x & 31, gid = lane >> 2, tig = lane & 3;
    constexpr int NT = NOUT / 8, KT = K / 16;
    float acc[2][NT][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < NT; ++nt)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[mt][nt][j] = 0.0f;
#pragma unroll
    for (int kt = 0; kt < KT; ++kt) {
        uint32_t a[2][4];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
            const __nv_bfloat16* r0 = act + (row0 + 16 * mt + gid) * ld + 16 * kt + 2 * tig;
            const __nv_bfloat16* r1 = r0 + 8 * ld;
            a[mt][0] = ld_b32(r0);
            a[mt][1] = ld_b32(r1);
            a[mt][2] = ld_b32(r0 + 8);
            a[mt][3] = ld_b32(r1 + 8);
        }
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
            const __nv_bfloat16* w = W + (8 * nt + gid) * ldw + 16 * kt + 2 * tig;
            const uint32_t b[2] = {ldg_b32(w), ldg_b32(w + 8)};
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) mma_bf16(acc[mt][nt], a[mt], b);
        }
    }
    __syncwarp();
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < NT; ++nt)
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                const int r = row0 + 16 * mt + gid + 8 * hh;
                const int col = 8 * nt + 2 * tig;
                float v0 = acc[mt][nt][2 * hh] + __ldg(bias + col);
                float v1 = acc[mt][nt][2 * hh + 1] + __ldg(bias + col + 1);
                if (RELU) {
                    v0 = fmaxf(v0, 0.0f);
                    v1 = fmaxf(v1, 0.0f);
                }
                if (TO_FLOAT) {
                    out_f[r * 8 + col] = v0;
                    out_f[r * 8 + col + 1] = v1;
                } else {
                    *reinterpret_cast<__nv_bfloat162*>(act + r * ld + col) = __floats2bfloat162_rn(v0, v1);
                }
            }
    __syncwarp();
}

// Forward pass for the 32 cells of this warp (all 32 lanes must be present).
// `act` (shared) holds per cell row the 20 bf16 features followed by zero
// padding up to 32; on return out_f[r * 8 + j], j < 4, holds the outputs.
// `wts` is the device inference blob in global memory (bf16 weights then
// float32 biases), read through the read-only cache.
__device__ __forceinline__ void mlp_forward_warp(__nv_bfloat16* act, const unsigned char* __restrict__ wts,
                                                 float* out_f)
{
    const __nv_bfloat16* W = reinterpret_cast<const __nv_bfloat16*>(wts);
    const float* bias = reinterpret_cast<const float*>(wts + MLPD_NBF16 * 2);
    const int row0 = (threadIdx.x + threadIdx.y * blockDim.x) & ~31;
    mlp_layer<32, 64, true, false>(act, MLP_HS, W + MLPD_W1, MLP_XS, bias, row0, nullptr);
    mlp_layer<64, 64, true, false>(act, MLP_HS, W + MLPD_W2, MLP_HS, bias + 64, row0, nullptr);
    mlp_layer<64, 64, true, false>(act, MLP_HS, W + MLPD_W3, MLP_HS, bias + 128, row0, nullptr);
    mlp_layer<64, 8, false, true>(act, MLP_HS, W + MLPD_W4, MLP_HS, bias + 192, row0, out_f);
}

}  // namespace lb

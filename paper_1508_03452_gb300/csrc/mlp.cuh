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

// Shared activation rows: 72 bf16 (144 bytes, a multiple of 16 for ldmatrix)
// per cell, so the 8 rows of one 8x8 fragment fall in distinct banks.
constexpr int MLP_HS = 72;
// Device inference blob: bf16 weights in MMA fragment order, then float32
// biases. Layer l (K inputs padded to 32 or 64, N outputs padded to a
// multiple of 8, zero padding) stores, for output row r, k-tile kt (16 wide)
// and lane column group t (0..3), the 4 values W[r][16 kt + 2t + {0, 1, 8, 9}]
// at ((r * K/16 + kt) * 4 + t) * 4: the B fragment of one lane is one 8-byte load.
constexpr int MLP_K1 = 32;  // first-layer inputs, padded
constexpr int MLPD_W1 = 0, MLPD_W2 = MLPD_W1 + MLP_H * MLP_K1, MLPD_W3 = MLPD_W2 + MLP_H * MLP_H,
              MLPD_W4 = MLPD_W3 + MLP_H * MLP_H, MLPD_NBF16 = MLPD_W4 + 8 * MLP_H;
constexpr int MLPD_NBIAS = 3 * MLP_H + 8;                                // float32 biases after the bf16 block
constexpr int MLPD_BYTES = MLPD_NBF16 * 2 + MLPD_NBIAS * 4;              // device inference blob
constexpr int MLP_ACT_BYTES_PER_CELL = MLP_HS * 2;                       // shared activation row per cell

// blob index of weight (r, k) of a layer with K inputs (fragment order above)
__host__ __device__ constexpr int mlpd_frag_index(int r, int k, int K)
{
    return ((r * (K / 16) + k / 16) * 4 + (k % 8) / 2) * 4 + ((k % 16) / 8) * 2 + (k % 2);
}

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

// four 8x8 bf16 matrices from shared memory (row addresses from lanes 0..31)
__device__ __forceinline__ void ldmatrix_x4(uint32_t* r, const __nv_bfloat16* row_addr)
{
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(row_addr);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a));
}

__device__ __forceinline__ void mma_bf16(float* d, const uint32_t* a, const uint32_t* b)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// One dense layer for the 32 rows owned by this warp: act[r][0..NOUT) =
// f(act[r][0..K) . W^T + bias), in place (all reads of the warp's rows finish
// before its writes). The accumulators start from the bias; ReLU is applied
// after the bf16 rounding (rounding is monotonic and keeps 0). `row0` is the
// warp's first row.
template <int K, int NOUT, bool RELU, bool TO_FLOAT>
__device__ __forceinline__ void mlp_layer(__nv_bfloat16* act, const __nv_bfloat16* W, const float* bias, int row0,
                                          float* out_f)
{
    const int lane = threadIdx.x & 31, gid = lane >> 2, tig = lane & 3;
    constexpr int NT = NOUT / 8, KT = K / 16;
    float acc[2][NT][4];
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
        const float2 b = __ldg(reinterpret_cast<const float2*>(bias + 8 * nt + 2 * tig));
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
            acc[mt][nt][0] = b.x;
            acc[mt][nt][1] = b.y;
            acc[mt][nt][2] = b.x;
            acc[mt][nt][3] = b.y;
        }
    }
#pragma unroll
    for (int kt = 0; kt < KT; ++kt) {
        uint32_t a[2][4];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
            ldmatrix_x4(a[mt], act + (row0 + 16 * mt + (lane & 15)) * MLP_HS + 16 * kt + (lane >> 4) * 8);
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
            const uint2 bw = __ldg(reinterpret_cast<const uint2*>(W + (((8 * nt + gid) * KT + kt) * 4 + tig) * 4));
            const uint32_t b[2] = {bw.x, bw.y};
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) mma_bf16(acc[mt][nt], a[mt], b);
        }
    }
    __syncwarp();
    const __nv_bfloat162 zero2 = __floats2bfloat162_rn(0.0f, 0.0f);
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < NT; ++nt)
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                const int r = row0 + 16 * mt + gid + 8 * hh;
                const int col = 8 * nt + 2 * tig;
                if (TO_FLOAT) {
                    out_f[r * 8 + col] = acc[mt][nt][2 * hh];
                    out_f[r * 8 + col + 1] = acc[mt][nt][2 * hh + 1];
                } else {
                    __nv_bfloat162 v = __floats2bfloat162_rn(acc[mt][nt][2 * hh], acc[mt][nt][2 * hh + 1]);
                    if (RELU) v = __hmax2(v, zero2);
                    *reinterpret_cast<__nv_bfloat162*>(act + r * MLP_HS + col) = v;
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
    mlp_layer<MLP_K1, 64, true, false>(act, W + MLPD_W1, bias, row0, nullptr);
    mlp_layer<64, 64, true, false>(act, W + MLPD_W2, bias + 64, row0, nullptr);
    mlp_layer<64, 64, true, false>(act, W + MLPD_W3, bias + 128, row0, nullptr);
    mlp_layer<64, 8, false, true>(act, W + MLPD_W4, bias + 192, row0, out_f);
}

}  // namespace lb

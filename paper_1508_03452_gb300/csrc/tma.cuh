// tma.cuh -- the Blackwell data-movement primitives the tiled step kernel uses:
// mbarriers in shared memory, tensor-map (TMA) tile loads completed on an
// mbarrier, tensor-map tile stores from shared memory, and the proxy fences
// between them. Inline PTX (sm_90 and later; compiled for sm_103a).
//
// Every wait is bounded: a wait that has not seen its phase complete within
// kTmaWaitNs of global time returns false instead of spinning on, so a lost
// copy surfaces as an error status rather than a hung GPU.
#pragma once

#include <cuda.h>  // CUtensorMap (an opaque 128-byte descriptor)
#include <cuda_runtime.h>
#include <stdint.h>

namespace lb {

constexpr unsigned long long kTmaWaitNs = 500ull * 1000ull * 1000ull;  // 0.5 s

// Tile of the tiled step: kTileW x kTileH cells, one thread per cell; the
// input boxes reach kTileHaloY rows above and below and one 16-byte unit of
// columns on either side (tile_halo_x elements of `bytes` bytes).
#ifndef LB_TILE_H
#define LB_TILE_H 8  // tile rows (32 x 8 cells: 256 threads, two blocks per SM)
#endif
constexpr int kTileW = 32, kTileH = LB_TILE_H, kTileHaloY = 2;
constexpr int kTileThreads = kTileW * kTileH;
__host__ __device__ constexpr int tile_halo_x(int bytes) { return 16 / bytes; }

// Tensor maps of one run of the tiled step for one input buffer (the other
// buffer is the output, written by the cells' own vector stores and, for the
// primitives, by p_out). The population maps follow the group / pair storage
// order: a row of the fluid groups is the 4 nx values (4 per cell) of one
// group; boxes fg_in (4 (kTileW + 2 halo), kTileH + 4, 1 group), r_in (the
// rest pairs: 2 (kTileW + 2 halo), kTileH + 4), h_in (2 (kTileW + 8), kTileH + 4,
// 2 pairs), h24_in (kTileW + 8, kTileH + 4), p_in and p_out (4 kTileW, kTileH, 3: the
// primitives' three 4-vectors).
struct TileMaps {  // (aligned as CUtensorMap)
    CUtensorMap fg_in;   // (4 x, y, group 0..8) input fluid groups
    CUtensorMap r_in;    // (2 x, y) input rest pairs {f_0, g_0}
    CUtensorMap h_in;    // (2 x, y, pair 0..11) input h pairs
    CUtensorMap h24_in;  // (x, y) input h_24
    CUtensorMap p_in;    // (4 x, y, vector 0..2) input primitives
    CUtensorMap p_out;   // (4 x, y, vector) output primitives
};

// The tiles of a grid whose input boxes lie inside it: tiles (i, j),
// x0 = i kTileW, y0 = j kTileH, with x0 - halo_x >= 0, x0 + kTileW + halo_x <= nx,
// y0 - kTileHaloY >= 0, y0 + kTileH + kTileHaloY <= ny; a rectangle of nx x ny
// tiles from tile (x0, y0) (empty if either count is 0).
struct TileRange {
    int x0, y0, nx, ny;
};
__host__ __device__ inline TileRange interior_tiles(int nx, int ny, int halo_x)
{
    TileRange r;
    r.x0 = (halo_x + kTileW - 1) / kTileW;
    r.y0 = (kTileHaloY + kTileH - 1) / kTileH;
    const int xe = nx - kTileW - halo_x, ye = ny - kTileH - kTileHaloY;  // largest admissible x0, y0
    r.nx = xe < 0 ? 0 : xe / kTileW - r.x0 + 1;
    r.ny = ye < 0 ? 0 : ye / kTileH - r.y0 + 1;
    if (r.nx < 0) r.nx = 0;
    if (r.ny < 0) r.ny = 0;
    return r;
}

// What a run's tiled step needs besides its kernel arguments: its tensor
// maps, the device argument records of its input buffer's parity (indexed by
// the run number in the tiles) and its edge tiles, (run, x0, y0, z) of 32 x 4
// cells, which a per-cell launch updates.
struct TileLaunch {
    const TileMaps* maps;
    const unsigned char* args;
    const int4* edge_tiles;
    int nedge;
    int sms;  // SMs of the device (the tile kernel's grid is one wave of resident blocks)
};

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// makes the initialised barriers visible to the asynchronous (TMA) proxy
__device__ __forceinline__ void mbar_init_fence()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// waits for the phase of parity `parity` of *bar; false after kTmaWaitNs
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > kTmaWaitNs) return false;
    return true;
}

// 3-D / 4-D tile loads into shared memory, completing on *bar (byte count)
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int c0, int c1, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
        : "memory");
}

// 3-D tile store from shared memory (bulk-group completion)
__device__ __forceinline__ void tma_store_3d(const CUtensorMap* map, const void* src, int c0, int c1, int c2)
{
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%2, %3, %4}], [%1];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(smem_u32(src)), "r"(c0), "r"(c1), "r"(c2)
                 : "memory");
}

__device__ __forceinline__ void tma_store_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }

// the committed stores have finished reading shared memory
__device__ __forceinline__ void tma_store_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }

// orders this thread's generic-proxy shared-memory writes before later
// asynchronous-proxy (TMA) accesses to them
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void prefetch_tensormap(const CUtensorMap* map)
{
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

}  // namespace lb

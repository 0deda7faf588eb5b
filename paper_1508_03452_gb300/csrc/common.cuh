// common.cuh -- storage configurations, kernel argument blocks and lattice
// indexing shared by the kernels of the RRMHD lattice Boltzmann library.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstring>

#include "lattice.cuh"

namespace lb {

// Storage / arithmetic configurations. `pop` stores the fluid populations f,
// g as deviations from the reference rest equilibrium; `hpop` the Maxwell
// populations; `prim` the 12 primitive fields; `real` is the arithmetic type.
struct CfgF64 {
    using real = double;
    using pop = double;
    using hpop = double;
    using prim = double;
    static constexpr bool kHalf = false;
    static constexpr bool kVecSlots = true;  // shared-memory slot order of the step kernel
};
struct CfgF32 {
    using real = float;
    using pop = float;
    using hpop = float;
    using prim = float;
    static constexpr bool kHalf = false;
    static constexpr bool kVecSlots = true;  // shared-memory slot order of the step kernel
};
struct CfgF16 {  // float16 relative deviations for f and g
    using real = float;
    using pop = __half;
    using hpop = float;
    using prim = float;
    static constexpr bool kHalf = true;
    static constexpr bool kVecSlots = false;  // shared-memory slot order of the step kernel
};

// primitive fields, stored as three 4-vectors per cell: {n, eps, u_x, u_y},
// {u_z, E_x, E_y, E_z}, {B_x, B_y, B_z, rho_c} (vector P / 4 of the cell,
// component P % 4; three planes of `stride` 4-vectors)
enum { P_N = 0, P_EPS = 1, P_U = 2, P_E = 5, P_B = 8, P_RHO = 11, NPRIM = 12 };
constexpr int kPrimVecs = NPRIM / 4;
__host__ __device__ constexpr int64_t prim_elem(int P, int64_t c, int64_t stride)
{
    return 4 * ((P >> 2) * stride + c) + (P & 3);
}

// Storage order of the populations of one buffer (every plane holds `stride`
// cells). Fluid: the opposite D3Q19 directions i = 2G-1 and 2G (G = 1..9)
// stream over the same cells, and so do f and g of one direction, so group G
// keeps {f_{2G-1}, g_{2G-1}, f_{2G}, g_{2G}} of a cell together (4-vector G-1
// of the cell: one vector load per stencil point serves four populations); the
// rest pair {f_0, g_0} follows the nine group planes as 2-vectors. Maxwell: the
// D3Q13 populations 2m and 2m+1 (m = 0..11) hop the same way and form 2-vector
// m; the rest population h_24 follows as a plane of its own.
constexpr int kFGroups = 9;
__host__ __device__ constexpr int64_t fg_elem(int i, int which, int64_t c, int64_t stride)
{
    return i == 0 ? 4 * kFGroups * stride + 2 * c + which
                  : 4 * (((i - 1) >> 1) * stride + c) + 2 * ((i - 1) & 1) + which;
}
// element of Maxwell population k (0..24) of cell c
__host__ __device__ constexpr int64_t h_elem(int k, int64_t c, int64_t stride)
{
    return k < 24 ? 2 * ((k >> 1) * stride + c) + (k & 1) : 24 * stride + c;
}

// per-run recovery counters: [0] failures [1] iteration sum [2] iteration max,
// then kHistBins bins: cells that converged in 1, 2, ..., kHistBins - 1
// iterations, and in kHistBins or more
constexpr int kHistBins = 17;
constexpr int kNumStats = 3 + kHistBins;
// the counters are kept in kStatSlots copies (slot = block index mod
// kStatSlots) so that the warps' atomics do not all meet on one address; the
// host sums the copies (maximum for [2])
constexpr int kStatSlots = 128;

constexpr int kStepThreads = 128;  // threads (cells) per block of the step kernels

constexpr int FLAG_NO_EM_COLLISION = 1;
constexpr int FLAG_UNSHIFTED_POWER = 2;
constexpr int FLAG_ONE_PASS_RECOVERY = 4;
constexpr int FLAG_GAUSS_CHARGE = 8;  // Ohm's convection current with eps0 div E of the previous step
constexpr int FLAG_TMA_TILES = 16;  // 2-D periodic float32/float16 runs step by the TMA tile kernel
enum { SEED_PREV = 0, SEED_MLP = 1, SEED_COLD = 2 };

// Population scale for float16 relative deviations: stored value =
// deviation * inv[i]; deviation = stored * scale[i].
struct HalfScale {
    float f[19], finv[19], g[19], ginv[19];
};

template <class Cfg>
struct StepArgs {
    using pop = typename Cfg::pop;
    using hpop = typename Cfg::hpop;
    using prim = typename Cfg::prim;
    using real = typename Cfg::real;
    const pop* __restrict__ fgin;  // f and g in the group order of fg_elem
    const hpop* __restrict__ hin;  // h in the pair order of h_elem
    const prim* __restrict__ pin;
    pop* __restrict__ fgout;
    hpop* __restrict__ hout;
    prim* __restrict__ pout;
    int nx, ny, nz;
    int64_t stride;  // elements between consecutive planes
    int periodic[3];
    int open_mask;  // bit a: axis a has an open (or driven) face
    int flags;
    Phys<real> k;
    HalfScale hs;
    unsigned long long* stats;  // kStatSlots x kNumStats counters (see kHistBins)
    const unsigned char* mlp;   // device inference blob of the learned seed (SEED_MLP)
    float* dump;                // optional: per cell 20 features + 4 targets of the learned seed
    int seed;                   // SEED_PREV | SEED_MLP | SEED_COLD
    // photospheric body force (open-variant code): the pattern F of each (x, y)
    // column (2 float64, amplitude F0), applied in z < force_layers while the
    // input state's max |u|^2 (*umax_in) is below vmax2 (vmax2 <= 0: always);
    // force_cdt = c dt / (10 q) and force_dt = dt put it into the populations
    const double* fdrive;
    int force_layers;
    double vmax2;
    const double* umax_in;  // max |u|^2 of the input state (forced runs with a cut-off)
    double* umax_out;       // running max |u|^2 of the output state (float64 bits, atomicMax)
    real force_cdt, force_dt;
    // relaxed initialisation (open-variant code): the initial n, p, u (3), B (3)
    // planes (8 N float64) the fluid and B are held at, E_{k-1}, E_{k-2} (6 N
    // float64) and the running max |E - E_{k-2}|^2, max |E|^2 (2 float64 bits)
    const double* relax_in;
    double* relax_e;
    double* relax_red;
    // status word of the handle: kernels OR in STATUS_* bits (device int)
    int* status;
};
// status bits a step kernel can raise
constexpr int STATUS_TMA_TIMEOUT = 1;      // a tile's copy did not arrive within the wait limit
constexpr int STATUS_BARRIER_TIMEOUT = 2;  // a persistent launch's grid barrier gave up waiting
// open_mask bit for runs that need the open-variant code without an open face
constexpr int OPEN_EXTRA = 8;

// population load / store in the configured format
template <class Cfg>
__device__ __forceinline__ typename Cfg::real ld_pop(const typename Cfg::pop* p, float scale)
{
    if constexpr (Cfg::kHalf)
        return __half2float(__ldg(reinterpret_cast<const __half*>(p))) * scale;
    else
        return __ldg(p);
}

template <class Cfg>
__device__ __forceinline__ void st_pop(typename Cfg::pop* p, typename Cfg::real v, float inv_scale)
{
    if constexpr (Cfg::kHalf)
        *p = __float2half_rn(v * inv_scale);
    else
        *p = v;
}

// vector loads / stores of a fluid group (4 values at p, p 4-element aligned)
// and of a 2-vector (the rest pair, an h pair), in stored units
template <class R>
struct V4 {
    R x, y, z, w;
};
template <class R>
struct V2 {
    R x, y;
};

__device__ __forceinline__ float2 half2_bits_to_float2(unsigned u)
{
    __half2 h;
    static_assert(sizeof(h) == sizeof(u), "half2 size");
    memcpy(&h, &u, sizeof(u));
    return __half22float2(h);
}
__device__ __forceinline__ unsigned float2_to_half2_bits(float a, float b)
{
    const __half2 h = __floats2half2_rn(a, b);
    unsigned u;
    memcpy(&u, &h, sizeof(u));
    return u;
}

template <class Cfg>
__device__ __forceinline__ V4<typename Cfg::real> ld_quad(const typename Cfg::pop* p)
{
    if constexpr (Cfg::kHalf) {
        const uint2 u = __ldg(reinterpret_cast<const uint2*>(p));
        const float2 a = half2_bits_to_float2(u.x), b = half2_bits_to_float2(u.y);
        return {a.x, a.y, b.x, b.y};
    } else if constexpr (sizeof(typename Cfg::pop) == 8) {
        const double2 a = __ldg(reinterpret_cast<const double2*>(p));
        const double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
        return {a.x, a.y, b.x, b.y};
    } else {
        const float4 a = __ldg(reinterpret_cast<const float4*>(p));
        return {a.x, a.y, a.z, a.w};
    }
}

// inv: the float16 scales of the four values (unused for float32 / float64)
template <class Cfg>
__device__ __forceinline__ void st_quad(typename Cfg::pop* p, const V4<typename Cfg::real>& v, const V4<float>& inv)
{
    if constexpr (Cfg::kHalf) {
        *reinterpret_cast<uint2*>(p) =
            make_uint2(float2_to_half2_bits(v.x * inv.x, v.y * inv.y), float2_to_half2_bits(v.z * inv.z, v.w * inv.w));
    } else if constexpr (sizeof(typename Cfg::pop) == 8) {
        reinterpret_cast<double2*>(p)[0] = make_double2(v.x, v.y);
        reinterpret_cast<double2*>(p)[1] = make_double2(v.z, v.w);
    } else {
        *reinterpret_cast<float4*>(p) = make_float4(v.x, v.y, v.z, v.w);
    }
}

template <class Cfg>
__device__ __forceinline__ V2<typename Cfg::real> ld_fgpair(const typename Cfg::pop* p)
{
    if constexpr (Cfg::kHalf) {
        const float2 a = half2_bits_to_float2(__ldg(reinterpret_cast<const unsigned*>(p)));
        return {a.x, a.y};
    } else if constexpr (sizeof(typename Cfg::pop) == 8) {
        const double2 a = __ldg(reinterpret_cast<const double2*>(p));
        return {a.x, a.y};
    } else {
        const float2 a = __ldg(reinterpret_cast<const float2*>(p));
        return {a.x, a.y};
    }
}

template <class Cfg>
__device__ __forceinline__ void st_fgpair(typename Cfg::pop* p, typename Cfg::real f, typename Cfg::real g,
                                          float inv_f, float inv_g)
{
    if constexpr (Cfg::kHalf)
        *reinterpret_cast<unsigned*>(p) = float2_to_half2_bits(f * inv_f, g * inv_g);
    else if constexpr (sizeof(typename Cfg::pop) == 8)
        *reinterpret_cast<double2*>(p) = make_double2(f, g);
    else
        *reinterpret_cast<float2*>(p) = make_float2(f, g);
}

// the same from shared memory (a tile's staged copy)
template <class Cfg>
__device__ __forceinline__ V4<typename Cfg::real> ld_quad_sh(const typename Cfg::pop* p)
{
    if constexpr (Cfg::kHalf) {
        const uint2 u = *reinterpret_cast<const uint2*>(p);
        const float2 a = half2_bits_to_float2(u.x), b = half2_bits_to_float2(u.y);
        return {a.x, a.y, b.x, b.y};
    } else {
        static_assert(sizeof(typename Cfg::pop) == 4, "shared-memory tiles hold float32 or float16");
        const float4 a = *reinterpret_cast<const float4*>(p);
        return {a.x, a.y, a.z, a.w};
    }
}
template <class Cfg>
__device__ __forceinline__ V2<typename Cfg::real> ld_pair_sh(const typename Cfg::pop* p)
{
    if constexpr (Cfg::kHalf) {
        const float2 a = half2_bits_to_float2(*reinterpret_cast<const unsigned*>(p));
        return {a.x, a.y};
    } else {
        const float2 a = *reinterpret_cast<const float2*>(p);
        return {a.x, a.y};
    }
}

// the three primitive 4-vectors of a cell (p at its first element of plane 0)
// as 12 values in the order of the P_ indices; the planes are 4 stride apart
template <class Cfg>
__device__ __forceinline__ void ld_prims(const typename Cfg::prim* p, int64_t stride, typename Cfg::real (&v)[NPRIM])
{
    using R = typename Cfg::real;
#pragma unroll
    for (int q = 0; q < kPrimVecs; ++q) {
        const typename Cfg::prim* pq = p + 4 * q * stride;
        if constexpr (sizeof(typename Cfg::prim) == 8) {
            const double2 a = __ldg(reinterpret_cast<const double2*>(pq));
            const double2 b = __ldg(reinterpret_cast<const double2*>(pq) + 1);
            v[4 * q] = (R)a.x, v[4 * q + 1] = (R)a.y, v[4 * q + 2] = (R)b.x, v[4 * q + 3] = (R)b.y;
        } else {
            const float4 a = __ldg(reinterpret_cast<const float4*>(pq));
            v[4 * q] = (R)a.x, v[4 * q + 1] = (R)a.y, v[4 * q + 2] = (R)a.z, v[4 * q + 3] = (R)a.w;
        }
    }
}

template <class Cfg>
__device__ __forceinline__ void st_prims(typename Cfg::prim* p, int64_t stride, const typename Cfg::real (&v)[NPRIM])
{
#pragma unroll
    for (int q = 0; q < kPrimVecs; ++q) {
        typename Cfg::prim* pq = p + 4 * q * stride;
        if constexpr (sizeof(typename Cfg::prim) == 8) {
            reinterpret_cast<double2*>(pq)[0] = make_double2(v[4 * q], v[4 * q + 1]);
            reinterpret_cast<double2*>(pq)[1] = make_double2(v[4 * q + 2], v[4 * q + 3]);
        } else {
            *reinterpret_cast<float4*>(pq) =
                make_float4((float)v[4 * q], (float)v[4 * q + 1], (float)v[4 * q + 2], (float)v[4 * q + 3]);
        }
    }
}

// a Maxwell pair (2m, 2m+1) at p
template <class Cfg>
__device__ __forceinline__ V2<typename Cfg::real> ld_hpair(const typename Cfg::hpop* p)
{
    using R = typename Cfg::real;
    if constexpr (sizeof(typename Cfg::hpop) == 8) {
        const double2 a = __ldg(reinterpret_cast<const double2*>(p));
        return {(R)a.x, (R)a.y};
    } else {
        const float2 a = __ldg(reinterpret_cast<const float2*>(p));
        return {(R)a.x, (R)a.y};
    }
}

template <class Cfg>
__device__ __forceinline__ void st_hpair(typename Cfg::hpop* p, typename Cfg::real a, typename Cfg::real b)
{
    if constexpr (sizeof(typename Cfg::hpop) == 8)
        *reinterpret_cast<double2*>(p) = make_double2(a, b);
    else
        *reinterpret_cast<float2*>(p) = make_float2((float)a, (float)b);
}

// wrapped (periodic) or clamped (open / driven) coordinate
__host__ __device__ __forceinline__ int wrap_coord(int s, int n, int periodic)
{
    if (periodic) {
        while (s < 0) s += n;
        while (s >= n) s -= n;
    } else {
        s = s < 0 ? 0 : (s >= n ? n - 1 : s);
    }
    return s;
}

// neighbour offsets -2..+2 along each axis (y premultiplied by nx, z by nx ny)
struct Nb {
    int x[5];
    int64_t y[5], z[5];
    __device__ __forceinline__ int64_t at(int dx, int dy, int dz) const { return x[dx + 2] + y[dy + 2] + z[dz + 2]; }
};

__device__ __forceinline__ Nb make_nb(int x, int y, int z, int nx, int ny, int nz, const int* per)
{
    Nb nb;
#pragma unroll
    for (int d = -2; d <= 2; ++d) {
        nb.x[d + 2] = wrap_coord(x + d, nx, per[0]);
        nb.y[d + 2] = (int64_t)wrap_coord(y + d, ny, per[1]) * nx;
        nb.z[d + 2] = (int64_t)wrap_coord(z + d, nz, per[2]) * nx * (int64_t)ny;
    }
    return nb;
}

}  // namespace lb

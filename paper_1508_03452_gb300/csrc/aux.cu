// aux.cu -- initial state, open boundaries, normal-B fix, photospheric driving,
// output conversion and float64 diagnostics of the RRMHD lattice Boltzmann
// library (arXiv:1508.03452, Secs. III-IV).
#include <math_constants.h>

#include <climits>

#include "aux.cuh"

namespace lb {

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
template <class Cfg>
__device__ __forceinline__ void load_prim(const typename Cfg::prim* P, int64_t stride, int64_t c,
                                          Prim<typename Cfg::real>& s)
{
    using R = typename Cfg::real;
    s.n = (R)P[prim_elem(P_N, c, stride)];
    s.eps = (R)P[prim_elem(P_EPS, c, stride)];
    for (int a = 0; a < 3; ++a) {
        s.u[a] = (R)P[prim_elem(P_U + a, c, stride)];
        s.E[a] = (R)P[prim_elem(P_E + a, c, stride)];
        s.B[a] = (R)P[prim_elem(P_B + a, c, stride)];
    }
    s.rho = (R)P[prim_elem(P_RHO, c, stride)];
}

template <class Cfg, class R>
__device__ __forceinline__ void store_prim(typename Cfg::prim* P, int64_t stride, int64_t c, const Prim<R>& s)
{
    using T = typename Cfg::prim;
    P[prim_elem(P_N, c, stride)] = (T)s.n;
    P[prim_elem(P_EPS, c, stride)] = (T)s.eps;
    for (int a = 0; a < 3; ++a) {
        P[prim_elem(P_U + a, c, stride)] = (T)s.u[a];
        P[prim_elem(P_E + a, c, stride)] = (T)s.E[a];
        P[prim_elem(P_B + a, c, stride)] = (T)s.B[a];
    }
    P[prim_elem(P_RHO, c, stride)] = (T)s.rho;
}

template <int I, class Cfg, class R>
struct EqStore {
    static __device__ __forceinline__ void run(const PopView<Cfg>& V, int64_t c, const EqCell<R>& q)
    {
        st_pop<Cfg>(V.fg + fg_elem(I, 0, c, V.stride), (typename Cfg::real)feq_dev<I>(q), V.hs.finv[I]);
        st_pop<Cfg>(V.fg + fg_elem(I, 1, c, V.stride), (typename Cfg::real)geq_dev<I>(q), V.hs.ginv[I]);
        EqStore<I + 1, Cfg, R>::run(V, c, q);
    }
};
template <class Cfg, class R>
struct EqStore<19, Cfg, R> {
    static __device__ __forceinline__ void run(const PopView<Cfg>&, int64_t, const EqCell<R>&) {}
};

template <int K, class Cfg, class R>
struct HeqStore {
    static __device__ __forceinline__ void run(const PopView<Cfg>& V, int64_t c, const R* E, const R* B, const R* J,
                                               const Phys<R>& k)
    {
        V.h[h_elem(K, c, V.stride)] = (typename Cfg::hpop)heq13<K>(E, B, J, k);
        HeqStore<K + 1, Cfg, R>::run(V, c, E, B, J, k);
    }
};
template <class Cfg, class R>
struct HeqStore<24, Cfg, R> {
    static __device__ __forceinline__ void run(const PopView<Cfg>&, int64_t, const R*, const R*, const R*,
                                               const Phys<R>&) {}
};

// every population of cell c at its equilibrium for primitives s (the
// post-collision value of an equilibrium state is the equilibrium itself)
template <class Cfg, class R>
__device__ __forceinline__ void set_equilibrium(const PopView<Cfg>& V, int64_t c, const Prim<R>& s, const Phys<R>& k)
{
    EqCell<R> q;
    eq_cell(s, k, q);
    R J[3];
    ohm_current(s.E, s.u, s.B, s.rho, k, J);
    EqStore<0, Cfg, R>::run(V, c, q);
    const R dE[3] = {s.E[0] - k.Er[0], s.E[1] - k.Er[1], s.E[2] - k.Er[2]};
    const R dB[3] = {s.B[0] - k.Br[0], s.B[1] - k.Br[1], s.B[2] - k.Br[2]};
    HeqStore<0, Cfg, R>::run(V, c, dE, dB, J, k);
    V.h[h_elem(24, c, V.stride)] = (typename Cfg::hpop)s.rho;
}

// ---------------------------------------------------------------------------
// initial state (Sec. IV set-ups): eps from Eq. EOS, E = -u x B when not
// given (Eq. Ohm_ideal), rho_c = eps0 div E by central differences (Eq.
// Gauss_E), J from Eq. Ohm, populations at equilibrium. float64 arithmetic.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void input_E(const InitInputs& in, int64_t c, int64_t N, double* E)
{
    if (in.E) {
        E[0] = in.E[c]; E[1] = in.E[N + c]; E[2] = in.E[2 * N + c];
    } else {
        const double u[3] = {in.u[c], in.u[N + c], in.u[2 * N + c]};
        const double B[3] = {in.B[c], in.B[N + c], in.B[2 * N + c]};
        E[0] = -(u[1] * B[2] - u[2] * B[1]);
        E[1] = -(u[2] * B[0] - u[0] * B[2]);
        E[2] = -(u[0] * B[1] - u[1] * B[0]);
    }
}

template <class Cfg>
__global__ void init_kernel(PopView<Cfg> V, InitInputs in, Phys<double> k, int* bad)
{
    const int64_t N = (int64_t)V.nx * V.ny * V.nz;
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= N) return;
    const int x = (int)(c % V.nx), y = (int)((c / V.nx) % V.ny), z = (int)(c / ((int64_t)V.nx * V.ny));
    Prim<double> s;
    s.n = in.n[c];
    s.eps = s.n * k.c2 + in.p[c] / k.gm1;
    for (int a = 0; a < 3; ++a) {
        s.u[a] = in.u[a * N + c];
        s.B[a] = in.B[a * N + c];
    }
    input_E(in, c, N, s.E);
    if (!(s.u[0] * s.u[0] + s.u[1] * s.u[1] + s.u[2] * s.u[2] < k.c2) || !(s.n > 0)) atomicExch(bad, 1);
    const int q[3] = {x, y, z}, n[3] = {V.nx, V.ny, V.nz};
    double div = 0.0;
    for (int a = 0; a < 3; ++a) {
        if (n[a] == 1) continue;
        int qp[3] = {q[0], q[1], q[2]}, qm[3] = {q[0], q[1], q[2]};
        qp[a] = wrap_coord(q[a] + 1, n[a], V.periodic[a]);
        qm[a] = wrap_coord(q[a] - 1, n[a], V.periodic[a]);
        double Ep[3], Em[3];
        input_E(in, qp[0] + (int64_t)V.nx * (qp[1] + (int64_t)V.ny * qp[2]), N, Ep);
        input_E(in, qm[0] + (int64_t)V.nx * (qm[1] + (int64_t)V.ny * qm[2]), N, Em);
        div += (Ep[a] - Em[a]) / (2.0 * k.dx);
    }
    s.rho = k.eps0 * div;
    store_prim<Cfg>(V.prim, V.stride, c, s);
    set_equilibrium<Cfg, double>(V, c, s, k);
}

// float64 means for the reference state: n, p, E (3), B (3), E_a E_b (6: xx yy
// zz xy xz yz), B_a B_b (6), B x E (3). Pass 1: per-block partial sums
// (grid-stride); pass 2: one block adds the partials in block order, so the
// result does not depend on scheduling.
__global__ void means_partial_kernel(InitInputs in, int64_t N, double* partial)
{
    constexpr int M = NMEANS;
    __shared__ double sh[M][kMeansThreads / 32];
    double acc[M];
    for (int j = 0; j < M; ++j) acc[j] = 0.0;
    const int ia[6] = {0, 1, 2, 0, 0, 1}, ib[6] = {0, 1, 2, 1, 2, 2};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        double E[3], B[3];
        input_E(in, i, N, E);
        for (int a = 0; a < 3; ++a) B[a] = in.B[a * N + i];
        acc[0] += in.n[i];
        acc[1] += in.p[i];
        for (int a = 0; a < 3; ++a) {
            acc[2 + a] += E[a];
            acc[5 + a] += B[a];
        }
        for (int m = 0; m < 6; ++m) {
            acc[8 + m] += E[ia[m]] * E[ib[m]];
            acc[14 + m] += B[ia[m]] * B[ib[m]];
        }
        acc[20] += B[1] * E[2] - B[2] * E[1];
        acc[21] += B[2] * E[0] - B[0] * E[2];
        acc[22] += B[0] * E[1] - B[1] * E[0];
    }
    for (int j = 0; j < M; ++j)
        for (int o = 16; o > 0; o >>= 1) acc[j] += __shfl_down_sync(0xffffffffu, acc[j], o);
    if (threadIdx.x % 32 == 0)
        for (int j = 0; j < M; ++j) sh[j][threadIdx.x / 32] = acc[j];
    __syncthreads();
    if (threadIdx.x < M) {
        double a = 0.0;
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) a += sh[threadIdx.x][w];
        partial[(int64_t)blockIdx.x * M + threadIdx.x] = a;
    }
}

__global__ void means_final_kernel(const double* partial, int nblocks, int64_t N, double* out)
{
    if (threadIdx.x < NMEANS) {
        double a = 0.0;
        for (int b = 0; b < nblocks; ++b) a += partial[(int64_t)b * NMEANS + threadIdx.x];
        out[threadIdx.x] = a / (double)N;
    }
}

// ---------------------------------------------------------------------------
// open boundaries: copy of the first interior cell (faces in order -x .. +z,
// which is the same as clamping every open-axis coordinate into [1, n-2])
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// normal-B fix on one open face (axis a, side hi): B_n of the boundary cell is
// set so that the central-difference div B of the first interior cell
// vanishes; the change is carried by the h populations whose b is parallel to
// the normal (h_c += dB b_n / 8), and the f populations see the changed
// equilibrium through the collision (f_c += K_i [f_i^eq(new) - f_i^eq(old)]).
// ---------------------------------------------------------------------------
// f_c += K_i [f_i^eq(new) - f_i^eq(old)] for the 19 populations; `fv` holds
// their values, loaded before any store (the planes are distinct, which the
// compiler cannot prove)
template <int I, class Cfg, class R>
struct FixF {
    static __device__ __forceinline__ void run(const PopView<Cfg>& V, int64_t c, const EqCell<R>& qo,
                                               const EqCell<R>& qn, const R* fv)
    {
        const R d = k_aw<I>(qo) * (feq_dev<I>(qn) - feq_dev<I>(qo));
        st_pop<Cfg>(V.fg + fg_elem(I, 0, c, V.stride), fv[I] + d, V.hs.finv[I]);
        FixF<I + 1, Cfg, R>::run(V, c, qo, qn, fv);
    }
};
template <class Cfg, class R>
struct FixF<19, Cfg, R> {
    static __device__ __forceinline__ void run(const PopView<Cfg>&, int64_t, const EqCell<R>&, const EqCell<R>&,
                                               const R*)
    {
    }
};

// nfaces = 1: the face `hi` of axis a; nfaces = 2: both faces of axis a in one
// launch (independent when the axis has at least 4 cells: a face writes its
// boundary layer and reads the two layers inside it)
template <class Cfg>
__global__ void bfix_kernel(PopView<Cfg> V, Phys<typename Cfg::real> k, int a, int hi_first, int nfaces)
{
    using R = typename Cfg::real;
    const int n[3] = {V.nx, V.ny, V.nz};
    const int a1 = (a + 1) % 3, a2 = (a + 2) % 3;
    const int64_t face = (int64_t)n[a1] * n[a2];
    const int64_t mm = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (mm >= nfaces * face) return;
    const int hi = nfaces == 2 ? (int)(mm / face) : hi_first;
    const int64_t m = mm % face;
    int q[3];
    q[a1] = (int)(m % n[a1]);
    q[a2] = (int)(m / n[a1]);
    const int sgn = hi ? -1 : 1;
    const int b = hi ? n[a] - 1 : 0;
    auto idx = [&](const int* r) { return r[0] + (int64_t)V.nx * (r[1] + (int64_t)V.ny * r[2]); };
    int r1[3] = {q[0], q[1], q[2]};
    r1[a] = b + sgn;
    R tang = R(0);
    const int at[2] = {a1, a2};
    for (int t = 0; t < 2; ++t) {
        const int ax = at[t];
        if (n[ax] == 1) continue;
        int rp[3] = {r1[0], r1[1], r1[2]}, rm[3] = {r1[0], r1[1], r1[2]};
        rp[ax] = wrap_coord(r1[ax] + 1, n[ax], V.periodic[ax]);
        rm[ax] = wrap_coord(r1[ax] - 1, n[ax], V.periodic[ax]);
        tang += ((R)V.prim[prim_elem(P_B + ax, idx(rp), V.stride)] - (R)V.prim[prim_elem(P_B + ax, idx(rm), V.stride)]) /
                (R(2) * k.dx);
    }
    int r2[3] = {q[0], q[1], q[2]};
    r2[a] = b + 2 * sgn;
    int rb[3] = {q[0], q[1], q[2]};
    rb[a] = b;
    const int64_t cb = idx(rb);
    const R Bfar = (R)V.prim[prim_elem(P_B + a, idx(r2), V.stride)];
    const R Bn_new = Bfar + R(sgn) * R(2) * k.dx * tang;
    Prim<R> so;
    load_prim<Cfg>(V.prim, V.stride, cb, so);
    R fv[19], hv[8];
#pragma unroll
    for (int i = 0; i < 19; ++i) fv[i] = ld_pop<Cfg>(V.fg + fg_elem(i, 0, cb, V.stride), V.hs.f[i]);
    int hp = 0;  // the plane whose normal is axis a
#pragma unroll
    for (int p = 0; p < 3; ++p)
        if (plane_normal(p) == a) hp = p;
#pragma unroll
    for (int j = 0; j < 8; ++j) hv[j] = (R)V.h[h_elem(8 * hp + j, cb, V.stride)];
    const R dB = Bn_new - so.B[a];
    Prim<R> sn = so;
    sn.B[a] = Bn_new;
    V.prim[prim_elem(P_B + a, cb, V.stride)] = (typename Cfg::prim)Bn_new;
    // h: populations of the plane whose normal is axis a, b = -/+ o_p n_hat
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const R bn = R(((j % 2) == 0 ? -1 : 1) * plane_orient(hp));
        V.h[h_elem(8 * hp + j, cb, V.stride)] = (typename Cfg::hpop)(hv[j] + dB * bn / R(8));
    }
    EqCell<R> qo, qn;
    eq_cell(so, k, qo);
    eq_cell(sn, k, qn);
    FixF<0, Cfg, R>::run(V, cb, qo, qn, fv);
}

// ---------------------------------------------------------------------------
// photospheric driving: the lowest `layers` z-layers are reset to the
// equilibrium of their own n, eps, B, rho_c with the two-vortex drive velocity
// (max |u| = u0) and E = -u x B
// ---------------------------------------------------------------------------
// the two-vortex drive velocity of column (x, y), (u_x, u_y) with max |u| = u0:
// tabulated once per run (it does not change in time)
__global__ void drive_profile_kernel(int nx, int ny, double u0, double* uv)
{
    const int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (m >= (int64_t)nx * ny) return;
    const int x = (int)(m % nx), y = (int)(m / nx);
    const double X = -3.0 + (x + 0.5) * 6.0 / nx;
    const double Y = -3.0 + (y + 0.5) * 6.0 / ny;
    const double xs = X < 0.0 ? X : X - 3.0;
    const double pi = 3.14159265358979323846;
    uv[2 * m] = u0 * sin(pi * xs / 3.0) * cos(pi * Y / 6.0);
    uv[2 * m + 1] = u0 * cos(pi * xs / 3.0) * sin(pi * Y / 6.0);
}

template <class Cfg>
__global__ void drive_kernel(PopView<Cfg> V, Phys<typename Cfg::real> k, int layers, const double* __restrict__ uv)
{
    using R = typename Cfg::real;
    const int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t plane = (int64_t)V.nx * V.ny;
    if (m >= plane * layers) return;
    const int64_t c = m, col = m % plane;
    Prim<R> s;
    load_prim<Cfg>(V.prim, V.stride, c, s);
    s.u[0] = (R)uv[2 * col];
    s.u[1] = (R)uv[2 * col + 1];
    s.u[2] = R(0);
    s.E[0] = -(s.u[1] * s.B[2] - s.u[2] * s.B[1]);
    s.E[1] = -(s.u[2] * s.B[0] - s.u[0] * s.B[2]);
    s.E[2] = -(s.u[0] * s.B[1] - s.u[1] * s.B[0]);
    store_prim<Cfg>(V.prim, V.stride, c, s);
    set_equilibrium<Cfg, R>(V, c, s, k);
}

// ---------------------------------------------------------------------------
// outputs
// ---------------------------------------------------------------------------
// component P of every cell's primitives into out (N values)
template <class Cfg>
__global__ void prim_component_kernel(PopView<Cfg> V, int P, typename Cfg::prim* out)
{
    const int64_t N = (int64_t)V.nx * V.ny * V.nz;
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c < N) out[c] = V.prim[prim_elem(P, c, V.stride)];
}


template <class Cfg>
__global__ void moments_kernel(PopView<Cfg> V, Phys<double> k, double* out)
{
    const int64_t N = (int64_t)V.nx * V.ny * V.nz;
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= N) return;
    Prim<double> s;
    {
        typename Cfg::real pv[NPRIM];
        ld_prims<Cfg>(V.prim + prim_elem(0, c, V.stride), V.stride, pv);
        s.n = (double)pv[P_N];
        s.eps = (double)pv[P_EPS];
        for (int a = 0; a < 3; ++a) {
            s.u[a] = (double)pv[P_U + a];
            s.E[a] = (double)pv[P_E + a];
            s.B[a] = (double)pv[P_B + a];
        }
        s.rho = (double)pv[P_RHO];
    }
    double J[3];
    ohm_current(s.E, s.u, s.B, s.rho, k, J);
    out[0 * N + c] = s.n;
    out[1 * N + c] = k.gm1 * (s.eps - s.n * k.c2);
    out[2 * N + c] = s.eps;
    for (int a = 0; a < 3; ++a) {
        out[(3 + a) * N + c] = s.u[a];
        out[(6 + a) * N + c] = s.E[a];
        out[(9 + a) * N + c] = s.B[a];
        out[(13 + a) * N + c] = J[a];
    }
    out[12 * N + c] = s.rho;
}

// absolute post-collision populations (reference rest equilibrium added back)
template <class Cfg>
__global__ void populations_kernel(PopView<Cfg> V, RefPops ref, double* f, double* g, double* h)
{
    const int64_t N = (int64_t)V.nx * V.ny * V.nz;
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= N) return;
    for (int i = 0; i < 19; ++i) {
        if (f) f[i * N + c] = ref.f[i] + (double)ld_pop<Cfg>(V.fg + fg_elem(i, 0, c, V.stride), V.hs.f[i]);
        if (g) g[i * N + c] = ref.g[i] + (double)ld_pop<Cfg>(V.fg + fg_elem(i, 1, c, V.stride), V.hs.g[i]);
    }
    if (h)
        for (int i = 0; i < 25; ++i) h[i * N + c] = ref.h[i] + (double)V.h[h_elem(i, c, V.stride)];
}

// per-block float64 partial diagnostics: sum N^0, T^{0 nu} (4), rho_c, max |div B|,
// sum (div B)^2, non-finite count. A cell's sums over its populations and the
// sums over the 32 cells of a warp are taken in the storage's arithmetic type
// over the deviations (small numbers, rounded relative to themselves); the
// warp totals get the reference rest state of their cells and are summed
// over warps and blocks in float64. (float64 arithmetic per cell made this
// memory-bound pass bound by GB300's float64 rate, 15x slower.)
template <class Cfg>
__global__ void diag_kernel(PopView<Cfg> V, Phys<double> k, RefState r, double* partial)
{
    using R = typename Cfg::real;
    const int64_t N = (int64_t)V.nx * V.ny * V.nz;
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    R w[NPART] = {R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0)};  // deviations, |div B|, (div B)^2, bad
    if (c < N) {
        bool bad = false;
        R N0 = R(0), T0[4] = {R(0), R(0), R(0), R(0)}, rho = R(0);
        auto add = [&](int i, R fi, R gi) {
            bad = bad || !isfinite(fi) || !isfinite(gi);
            N0 += gi;
            T0[0] += fi;
#pragma unroll
            for (int a = 0; a < 3; ++a)
                if (c19(i, a)) T0[a + 1] += R(c19(i, a)) * fi;
        };
        {
            const V2<R> v = ld_fgpair<Cfg>(V.fg + fg_elem(0, 0, c, V.stride));
            add(0, Cfg::kHalf ? v.x * V.hs.f[0] : v.x, Cfg::kHalf ? v.y * V.hs.g[0] : v.y);
        }
#pragma unroll
        for (int i = 1; i < 19; i += 2) {
            const V4<R> v = ld_quad<Cfg>(V.fg + fg_elem(i, 0, c, V.stride));
            add(i, Cfg::kHalf ? v.x * V.hs.f[i] : v.x, Cfg::kHalf ? v.y * V.hs.g[i] : v.y);
            add(i + 1, Cfg::kHalf ? v.z * V.hs.f[i + 1] : v.z, Cfg::kHalf ? v.w * V.hs.g[i + 1] : v.w);
        }
#pragma unroll
        for (int m = 0; m < 12; ++m) {
            const V2<R> v = ld_hpair<Cfg>(V.h + h_elem(2 * m, c, V.stride));
            bad = bad || !isfinite(v.x) || !isfinite(v.y);
            rho += v.x;
            rho += v.y;
        }
        {
            const R hi = (R)V.h[h_elem(24, c, V.stride)];
            bad = bad || !isfinite(hi);
            rho += hi;
        }
#pragma unroll
        {
            R pv[NPRIM];
            ld_prims<Cfg>(V.prim + prim_elem(0, c, V.stride), V.stride, pv);
            for (int i = 0; i < NPRIM; ++i) bad = bad || !isfinite(pv[i]);
        }
        const int q[3] = {(int)(c % V.nx), (int)((c / V.nx) % V.ny), (int)(c / ((int64_t)V.nx * V.ny))};
        const int n[3] = {V.nx, V.ny, V.nz};
        R div = R(0);
        for (int a = 0; a < 3; ++a) {
            if (n[a] == 1) continue;
            int qp[3] = {q[0], q[1], q[2]}, qm[3] = {q[0], q[1], q[2]};
            qp[a] = wrap_coord(q[a] + 1, n[a], V.periodic[a]);
            qm[a] = wrap_coord(q[a] - 1, n[a], V.periodic[a]);
            const int64_t ip = qp[0] + (int64_t)V.nx * (qp[1] + (int64_t)V.ny * qp[2]);
            const int64_t im = qm[0] + (int64_t)V.nx * (qm[1] + (int64_t)V.ny * qm[2]);
            div += (R)V.prim[prim_elem(P_B + a, ip, V.stride)] - (R)V.prim[prim_elem(P_B + a, im, V.stride)];
        }
        div = div / (R(2) * (R)k.dx);
        w[0] = N0;
        for (int a = 0; a < 4; ++a) w[1 + a] = T0[a];
        w[5] = rho;
        w[6] = fabs(div);
        w[7] = div * div;
        w[8] = bad ? R(1) : R(0);
    }
    // the warp's cells in the arithmetic type (index 6 a max, the others sums)
#pragma unroll
    for (int j = 0; j < NPART; ++j)
        for (int o = 16; o > 0; o >>= 1) {
            const R other = __shfl_down_sync(0xffffffffu, w[j], o);
            w[j] = (j == 6) ? fmax(w[j], other) : w[j] + other;
        }
    __shared__ double sh[kDiagThreads / 32][NPART];
    const int wid = threadIdx.x / 32, lane = threadIdx.x % 32;
    if (lane == 0) {
        const int64_t first = c;  // the warp's first cell
        const double cells = (double)(first >= N ? 0 : (N - first < 32 ? N - first : 32));
        for (int j = 0; j < NPART; ++j) sh[wid][j] = (double)w[j];
        sh[wid][0] += cells * r.n_r;  // reference rest state of the warp's cells
        sh[wid][1] += cells * r.eps_r;
        for (int a = 0; a < 3; ++a) sh[wid][2 + a] *= kQ;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int j = 0; j < NPART; ++j) {
            double acc = sh[0][j];
            for (int ww = 1; ww < (int)(blockDim.x / 32); ++ww) acc = (j == 6) ? fmax(acc, sh[ww][j]) : acc + sh[ww][j];
            partial[(int64_t)blockIdx.x * NPART + j] = acc;
        }
    }
}

__global__ void diag_final_kernel(const double* partial, int64_t nblocks, int64_t ncells, double* out)
{
    double v[NPART] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int64_t b = threadIdx.x; b < nblocks; b += blockDim.x) {
        for (int j = 0; j < NPART; ++j) {
            const double x = partial[b * NPART + j];
            v[j] = (j == 6) ? fmax(v[j], x) : v[j] + x;
        }
    }
    block_reduce_partials(v, out);
    __syncthreads();
    if (threadIdx.x == 0) {
        // out layout of the C ABI: sums, max |div B|, rms div B, non-finite count, cells
        const double sumsq = out[7];
        out[7] = sqrt(sumsq / (double)ncells);
        out[9] = (double)ncells;
    }
}

// ---------------------------------------------------------------------------
// reconnection rate at the null point (Sec. IV, KH-driven reconnection):
// argmin of B_x^2 + B_y^2 over rows [y_lo, y_hi) of a 2-D run, ties to the
// lowest cell index (the reduction is exact, so its order does not matter)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void min_pair(double& v, long long& i, double v2, long long i2)
{
    if (v2 < v || (v2 == v && i2 < i)) {
        v = v2;
        i = i2;
    }
}

__device__ __forceinline__ void block_min_pair(double& v, long long& i)
{
    __shared__ double sv[32];
    __shared__ long long si[32];
    for (int o = 16; o > 0; o >>= 1)
        min_pair(v, i, __shfl_down_sync(0xffffffffu, v, o), __shfl_down_sync(0xffffffffu, i, o));
    const int w = threadIdx.x / 32, lane = threadIdx.x % 32;
    if (lane == 0) {
        sv[w] = v;
        si[w] = i;
    }
    __syncthreads();
    if (w == 0) {
        const int nw = (int)(blockDim.x / 32);
        v = lane < nw ? sv[lane] : CUDART_INF;
        i = lane < nw ? si[lane] : LLONG_MAX;
        for (int o = 16; o > 0; o >>= 1)
            min_pair(v, i, __shfl_down_sync(0xffffffffu, v, o), __shfl_down_sync(0xffffffffu, i, o));
    }
}

template <class Cfg>
__global__ void null_partial_kernel(PopView<Cfg> V, int y_lo, int y_hi, double* part_v, long long* part_i)
{
    const int64_t nb = (int64_t)V.nx * (y_hi - y_lo);
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double v = CUDART_INF;
    long long i = LLONG_MAX;
    if (t < nb) {
        const long long c = (long long)y_lo * V.nx + t;
        const double bx = (double)V.prim[prim_elem(P_B, c, V.stride)], by = (double)V.prim[prim_elem(P_B + 1, c, V.stride)];
        const double b2 = __dadd_rn(__dmul_rn(bx, bx), __dmul_rn(by, by));  // no FMA: rounds as written
        if (b2 == b2) {  // NaN never wins
            v = b2;
            i = c;
        }
    }
    block_min_pair(v, i);
    if (threadIdx.x == 0) {
        part_v[blockIdx.x] = v;
        part_i[blockIdx.x] = i;
    }
}

// out: R, x, y, |B| at the null (NaN when the band holds no finite field)
template <class Cfg>
__global__ void null_final_kernel(const double* part_v, const long long* part_i, int64_t nblocks, PopView<Cfg> V,
                                  const typename Cfg::prim* ez0, double B0, double* out)
{
    double v = CUDART_INF;
    long long i = LLONG_MAX;
    for (int64_t b = threadIdx.x; b < nblocks; b += blockDim.x) min_pair(v, i, part_v[b], part_i[b]);
    block_min_pair(v, i);
    if (threadIdx.x == 0) {
        const int64_t N = (int64_t)V.nx * V.ny;
        if (i >= 0 && i < N) {
            const double ez = (double)V.prim[prim_elem(P_E + 2, i, V.stride)];
            out[0] = (ez - (double)ez0[i]) / B0;
            out[1] = (double)(i % V.nx);
            out[2] = (double)(i / V.nx);
            out[3] = sqrt(v);
        } else {
            out[0] = out[1] = out[2] = out[3] = CUDART_NAN;
        }
    }
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
static inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

template <class Cfg>
cudaError_t launch_init(const PopView<Cfg>& V, const InitInputs& in, const Phys<double>& k, int* bad,
                        cudaStream_t s)
{
    const int64_t N = (int64_t)V.nx * V.ny * V.nz;
    init_kernel<Cfg><<<blocks_for(N, 128), 128, 0, s>>>(V, in, k, bad);
    return cudaGetLastError();
}

cudaError_t launch_means(const InitInputs& in, int64_t N, double* partial, double* out, cudaStream_t s)
{
    int nb = (int)((N + kMeansThreads - 1) / kMeansThreads);
    nb = nb < kMeansBlocks ? nb : kMeansBlocks;
    means_partial_kernel<<<nb, kMeansThreads, 0, s>>>(in, N, partial);
    means_final_kernel<<<1, 32, 0, s>>>(partial, nb, N, out);
    return cudaGetLastError();
}

cudaError_t launch_drive_profile(int nx, int ny, double u0, double* uv, cudaStream_t s)
{
    drive_profile_kernel<<<blocks_for((int64_t)nx * ny, 256), 256, 0, s>>>(nx, ny, u0, uv);
    return cudaGetLastError();
}

template <class Cfg>
cudaError_t launch_boundaries(const PopView<Cfg>& V, const Phys<typename Cfg::real>& k, const int* bc, int layers,
                              const double* drive_uv, cudaStream_t s)
{
    const int n[3] = {V.nx, V.ny, V.nz};
    // (the copy of the interior neighbour into the open faces is done by the
    // step kernel itself; here the normal-B fix and the driving follow it)
    for (int a = 0; a < 3; ++a) {
        const bool lo = bc[2 * a] != 0 && n[a] >= 3, hi = bc[2 * a + 1] != 0 && n[a] >= 3;
        const int64_t m = (int64_t)n[(a + 1) % 3] * n[(a + 2) % 3];
        if (lo && hi && n[a] >= 4) {
            bfix_kernel<Cfg><<<blocks_for(2 * m, 128), 128, 0, s>>>(V, k, a, 0, 2);
        } else {
            if (lo) bfix_kernel<Cfg><<<blocks_for(m, 128), 128, 0, s>>>(V, k, a, 0, 1);
            if (hi) bfix_kernel<Cfg><<<blocks_for(m, 128), 128, 0, s>>>(V, k, a, 1, 1);
        }
    }
    if (bc[4] == 2 && layers > 0 && drive_uv) {
        const int nl = layers < V.nz ? layers : V.nz;
        drive_kernel<Cfg><<<blocks_for((int64_t)V.nx * V.ny * nl, 128), 128, 0, s>>>(V, k, nl, drive_uv);
    }
    return cudaGetLastError();
}

template <class Cfg>
cudaError_t launch_moments(const PopView<Cfg>& V, const Phys<double>& k, double* out, cudaStream_t s)
{
    const int64_t N = (int64_t)V.nx * V.ny * V.nz;
    moments_kernel<Cfg><<<blocks_for(N, 128), 128, 0, s>>>(V, k, out);
    return cudaGetLastError();
}

template <class Cfg>
cudaError_t launch_prim_component(const PopView<Cfg>& V, int P, typename Cfg::prim* out, cudaStream_t s)
{
    const int64_t N = (int64_t)V.nx * V.ny * V.nz;
    prim_component_kernel<Cfg><<<blocks_for(N, 256), 256, 0, s>>>(V, P, out);
    return cudaGetLastError();
}

template <class Cfg>
cudaError_t launch_populations(const PopView<Cfg>& V, const RefPops& ref, double* f, double* g, double* h,
                               cudaStream_t s)
{
    const int64_t N = (int64_t)V.nx * V.ny * V.nz;
    populations_kernel<Cfg><<<blocks_for(N, 128), 128, 0, s>>>(V, ref, f, g, h);
    return cudaGetLastError();
}

template <class Cfg>
cudaError_t launch_diag(const PopView<Cfg>& V, const Phys<double>& k, const RefState& r, double* partial,
                        int64_t max_blocks, double* out, cudaStream_t s)
{
    const int64_t N = (int64_t)V.nx * V.ny * V.nz;
    const int64_t nb = blocks_for(N, kDiagThreads);
    if (nb > max_blocks) return cudaErrorInvalidValue;
    diag_kernel<Cfg><<<(unsigned)nb, kDiagThreads, 0, s>>>(V, k, r, partial);
    diag_final_kernel<<<1, kDiagThreads, 0, s>>>(partial, nb, N, out);
    return cudaGetLastError();
}

template <class Cfg>
cudaError_t launch_null(const PopView<Cfg>& V, int y_lo, int y_hi, const typename Cfg::prim* ez0, double B0,
                        double* scratch, int64_t scratch_doubles, double* out, cudaStream_t s)
{
    const int64_t nb = blocks_for((int64_t)V.nx * (y_hi - y_lo), kDiagThreads);
    if (2 * nb > scratch_doubles) return cudaErrorInvalidValue;
    double* pv = scratch;
    long long* pi = reinterpret_cast<long long*>(scratch + nb);
    null_partial_kernel<Cfg><<<(unsigned)nb, kDiagThreads, 0, s>>>(V, y_lo, y_hi, pv, pi);
    null_final_kernel<Cfg><<<1, kDiagThreads, 0, s>>>(pv, pi, nb, V, ez0, B0, out);
    return cudaGetLastError();
}

// max |u|^2 of a state into out[0] (float64 bits, atomicMax; out[0] zeroed
// before), out[1] (the running maximum of the next step) zeroed
template <class Cfg>
__global__ void umax_state_kernel(PopView<Cfg> V, double* out)
{
    const int64_t N = (int64_t)V.nx * V.ny * V.nz;
    double m = 0.0;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < N; c += (int64_t)gridDim.x * blockDim.x) {
        double u2 = 0.0;
        for (int a = 0; a < 3; ++a) {
            const double u = (double)V.prim[prim_elem(P_U + a, c, V.stride)];
            u2 += u * u;
        }
        m = fmax(m, u2);
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x % 32 == 0) atomicMax(reinterpret_cast<unsigned long long*>(out), (unsigned long long)__double_as_longlong(m));
    if (blockIdx.x == 0 && threadIdx.x == 0) out[1] = 0.0;
}

// after a step: the running maximum becomes the input state's, and restarts
__global__ void umax_roll_kernel(double* u)
{
    u[0] = u[1];
    u[1] = 0.0;
}

// E of a state into both history planes E_{k-1}, E_{k-2} (3 N float64 each)
template <class Cfg>
__global__ void relax_history_kernel(PopView<Cfg> V, double* e)
{
    const int64_t N = (int64_t)V.nx * V.ny * V.nz;
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= N) return;
    for (int a = 0; a < 3; ++a) {
        const double E = (double)V.prim[prim_elem(P_E + a, c, V.stride)];
        e[a * N + c] = E;
        e[(3 + a) * N + c] = E;
    }
}

template <class Cfg>
cudaError_t launch_umax_state(const PopView<Cfg>& V, double* out, cudaStream_t s)
{
    const int64_t N = (int64_t)V.nx * V.ny * V.nz;
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double), s);
    if (e != cudaSuccess) return e;
    const int64_t nb = blocks_for(N, 256);
    umax_state_kernel<Cfg><<<(unsigned)(nb < 1216 ? nb : 1216), 256, 0, s>>>(V, out);
    return cudaGetLastError();
}

cudaError_t launch_umax_roll(double* u, cudaStream_t s)
{
    umax_roll_kernel<<<1, 1, 0, s>>>(u);
    return cudaGetLastError();
}

template <class Cfg>
cudaError_t launch_relax_history(const PopView<Cfg>& V, double* e, cudaStream_t s)
{
    const int64_t N = (int64_t)V.nx * V.ny * V.nz;
    relax_history_kernel<Cfg><<<blocks_for(N, 256), 256, 0, s>>>(V, e);
    return cudaGetLastError();
}

#define LB_INSTANTIATE(CFG)                                                                                        \
    template cudaError_t launch_init<CFG>(const PopView<CFG>&, const InitInputs&, const Phys<double>&, int*,      \
                                          cudaStream_t);                                                           \
    template cudaError_t launch_boundaries<CFG>(const PopView<CFG>&, const Phys<CFG::real>&, const int*, int,      \
                                                const double*, cudaStream_t);                                      \
    template cudaError_t launch_moments<CFG>(const PopView<CFG>&, const Phys<double>&, double*, cudaStream_t);     \
    template cudaError_t launch_prim_component<CFG>(const PopView<CFG>&, int, CFG::prim*, cudaStream_t);           \
    template cudaError_t launch_populations<CFG>(const PopView<CFG>&, const RefPops&, double*, double*, double*,  \
                                                 cudaStream_t);                                                    \
    template cudaError_t launch_diag<CFG>(const PopView<CFG>&, const Phys<double>&, const RefState&, double*,      \
                                          int64_t, double*, cudaStream_t);                                         \
    template cudaError_t launch_null<CFG>(const PopView<CFG>&, int, int, const CFG::prim*, double, double*,       \
                                          int64_t, double*, cudaStream_t);                                         \
    template cudaError_t launch_umax_state<CFG>(const PopView<CFG>&, double*, cudaStream_t);                      \
    template cudaError_t launch_relax_history<CFG>(const PopView<CFG>&, double*, cudaStream_t);

LB_INSTANTIATE(CfgF64)
LB_INSTANTIATE(CfgF32)
LB_INSTANTIATE(CfgF16)

}  // namespace lb

// step_impl.cuh -- the fused time step of the RRMHD lattice Boltzmann method
// (arXiv:1508.03452, Sec. III), one thread per cell.
//
// The state holds post-collision populations, so one kernel does, per cell:
//   1. streaming (pull): f, g by the flux-limited (minmod) finite-volume
//      update of Eq. eq:rlb plus the bulk-viscosity term for f; h by the exact
//      D3Q13 hop of Eq. LB_Maxwell;
//   2. moments T^{mu nu}, N^mu (reference rest state added back), E', B,
//      rho_c (Eqs. Cal_E, Cal_B, Cal_rhoc);
//   3. Landau eigen-solve with the previous E, B (coupling subsection),
//      n = N^0 / U^0, the Ohm-coupled E solve and J (Eqs. Ohm, Ex_force), the
//      EOS (Eq. EOS);
//   4. collision at the new time level: Anderson-Witting for f towards Eq.
//      Dis_fun_EM, BGK for g towards Eq. Hupp, tau_h = 1/2 for h
//      (h -> 2 h^eq - h) towards Eq. Maxwell-eq; store populations and
//      primitives.
#pragma once
#include "common.cuh"

namespace lb {

// F_out - F_in of the limited upwind face values along one axis, for values
// ordered along the flow: um2 (two cells upwind), um1, u0 (this cell), up1.
// Face value = upwind + (1 - C)/2 * minmod(downwind - upwind, upwind - upwind2).
template <class R>
__device__ __forceinline__ R minmod(R a, R b)
{
    return (a > R(0) && b > R(0)) ? fmin(a, b) : ((a < R(0) && b < R(0)) ? fmax(a, b) : R(0));
}

template <class R>
__device__ __forceinline__ R flux_diff(R um2, R um1, R u0, R up1, R kappa)
{
    const R Fout = u0 + kappa * minmod(up1 - u0, u0 - um1);
    const R Fin = um1 + kappa * minmod(u0 - um1, um1 - um2);
    return Fout - Fin;
}

// One streamed fluid population (pre-collision value at t + dt).
template <int I, bool IS3D, bool VISC, class Cfg>
__device__ __forceinline__ typename Cfg::real stream_pop(const typename Cfg::pop* __restrict__ plane, const Nb& nb,
                                                         const Phys<typename Cfg::real>& k, float scale)
{
    using R = typename Cfg::real;
    constexpr int s[3] = {c19(I, 0), c19(I, 1), c19(I, 2)};
    const R v0 = ld_pop<Cfg>(plane + nb.at(0, 0, 0), scale);
    R flux = R(0), lap = R(0);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (a == 2 && !IS3D) continue;
        const int sa = s[a];
        auto at = [&](int d) {
            return ld_pop<Cfg>(plane + nb.at(a == 0 ? d : 0, a == 1 ? d : 0, a == 2 ? d : 0), scale);
        };
        if (sa != 0) {
            const R um2 = at(-2 * sa), um1 = at(-sa), up1 = at(sa);
            flux += flux_diff(um2, um1, v0, up1, k.kappa);
            if (VISC) lap += (um1 + up1) - R(2) * v0;
        } else if (VISC) {
            lap += (at(-1) + at(1)) - R(2) * v0;
        }
    }
    R out = v0 - k.C * flux;
    if (VISC && I != 0) out += k.kvisc * lap;
    return out;
}

template <int I, bool IS3D, class Cfg>
struct StreamAll {
    using R = typename Cfg::real;
    static __device__ __forceinline__ void run(const StepArgs<Cfg>& A, const Nb& nb, R* fd, R* gd, R (&Tm)[10],
                                               R (&Nm)[1])
    {
        fd[I] = stream_pop<I, IS3D, true, Cfg>(A.fin + (int64_t)I * A.stride, nb, A.k, A.hs.f[I]);
        gd[I] = stream_pop<I, IS3D, false, Cfg>(A.gin + (int64_t)I * A.stride, nb, A.k, A.hs.g[I]);
        constexpr int cx = c19(I, 0), cy = c19(I, 1), cz = c19(I, 2);
        const R f = fd[I];
        // T^{mu nu} of the deviations: p = (1, q chat)
        Tm[0] += f;
        if (cx) Tm[1] += R(cx) * f;
        if (cy) Tm[2] += R(cy) * f;
        if (cz) Tm[3] += R(cz) * f;
        if (cx) Tm[4] += f;  // xx (chat^2 = 1)
        if (cy) Tm[5] += f;  // yy
        if (cz) Tm[6] += f;  // zz
        if (cx * cy) Tm[7] += R(cx * cy) * f;
        if (cx * cz) Tm[8] += R(cx * cz) * f;
        if (cy * cz) Tm[9] += R(cy * cz) * f;
        Nm[0] += gd[I];
        StreamAll<I + 1, IS3D, Cfg>::run(A, nb, fd, gd, Tm, Nm);
    }
};
template <bool IS3D, class Cfg>
struct StreamAll<19, IS3D, Cfg> {
    using R = typename Cfg::real;
    static __device__ __forceinline__ void run(const StepArgs<Cfg>&, const Nb&, R*, R*, R (&)[10], R (&)[1]) {}
};

template <int I, class Cfg>
struct CollideFG {
    using R = typename Cfg::real;
    static __device__ __forceinline__ void run(const StepArgs<Cfg>& A, int64_t c, const R* fd, const R* gd,
                                               const EqCell<R>& q)
    {
        const R K = k_aw<I>(q);
        const R fo = fd[I] - K * (fd[I] - feq_dev<I>(q));
        const R go = gd[I] - A.k.inv_tau * (gd[I] - geq_dev<I>(q));
        st_pop<Cfg>(A.fout + (int64_t)I * A.stride + c, fo, A.hs.finv[I]);
        st_pop<Cfg>(A.gout + (int64_t)I * A.stride + c, go, A.hs.ginv[I]);
        CollideFG<I + 1, Cfg>::run(A, c, fd, gd, q);
    }
};
template <class Cfg>
struct CollideFG<19, Cfg> {
    using R = typename Cfg::real;
    static __device__ __forceinline__ void run(const StepArgs<Cfg>&, int64_t, const R*, const R*, const EqCell<R>&) {}
};

template <int K, class Cfg>
struct CollideH {
    using R = typename Cfg::real;
    static __device__ __forceinline__ void run(const StepArgs<Cfg>& A, int64_t c, const R* h, const R* E,
                                               const R* B, const R* J, bool em_coll)
    {
        const R v = em_coll ? R(2) * heq13<K>(E, B, J, A.k) - h[K] : h[K];
        A.hout[(int64_t)K * A.stride + c] = (typename Cfg::hpop)v;
        CollideH<K + 1, Cfg>::run(A, c, h, E, B, J, em_coll);
    }
};
template <class Cfg>
struct CollideH<24, Cfg> {
    using R = typename Cfg::real;
    static __device__ __forceinline__ void run(const StepArgs<Cfg>&, int64_t, const R*, const R*, const R*, const R*,
                                               bool) {}
};

template <class Cfg, bool IS3D>
__global__ void __launch_bounds__(128) step_kernel(const StepArgs<Cfg> A)
{
    using R = typename Cfg::real;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= A.nx || y >= A.ny) return;
    const Nb nb = make_nb(x, y, z, A.nx, A.ny, A.nz, A.periodic);
    const int64_t c = nb.at(0, 0, 0);
    const Phys<R>& k = A.k;

    // 1. streaming of f and g, with their moments
    R fd[19], gd[19];
    R Tm[10] = {R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0)};
    R Nm[1] = {R(0)};
    StreamAll<0, IS3D, Cfg>::run(A, nb, fd, gd, Tm, Nm);

    // 1b. exact streaming of h: h_k(x) = h_c,k(x - hop_k)
    R h[25];
#pragma unroll
    for (int kk = 0; kk < 24; ++kk)
        h[kk] = (R)A.hin[(int64_t)kk * A.stride + nb.at(-hop13(kk, 0), -hop13(kk, 1), -hop13(kk, 2))];
    h[24] = (R)A.hin[24 * A.stride + c];

    // previous primitives
    Prim<R> old;
    old.n = (R)A.pin[P_N * A.stride + c];
    old.eps = (R)A.pin[P_EPS * A.stride + c];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        old.u[a] = (R)A.pin[(P_U + a) * A.stride + c];
        old.E[a] = (R)A.pin[(P_E + a) * A.stride + c];
        old.B[a] = (R)A.pin[(P_B + a) * A.stride + c];
    }
    old.rho = (R)A.pin[P_RHO * A.stride + c];

    // 2. moments (reference rest state added back)
    const R qq = R(kQ), q2 = R(kQ2);
    R T[4][4];
    // reference moments: rest state (eps_r, p_r) plus the reference EM terms k.Tem
    T[0][0] = k.Tem[0] + Tm[0];  // T^00 - eps_r
    T[0][1] = T[1][0] = k.Tem[1] + qq * Tm[1];
    T[0][2] = T[2][0] = k.Tem[2] + qq * Tm[2];
    T[0][3] = T[3][0] = k.Tem[3] + qq * Tm[3];
    T[1][1] = k.p_r + k.Tem[4] + q2 * Tm[4];
    T[2][2] = k.p_r + k.Tem[5] + q2 * Tm[5];
    T[3][3] = k.p_r + k.Tem[6] + q2 * Tm[6];
    T[1][2] = T[2][1] = k.Tem[7] + q2 * Tm[7];
    T[1][3] = T[3][1] = k.Tem[8] + q2 * Tm[8];
    T[2][3] = T[3][2] = k.Tem[9] + q2 * Tm[9];
    const R dN0 = Nm[0];  // N^0 - n_r
    R dEp[3], dB[3], Ep[3], Bn[3], rho;
    em_moments(h, k, dEp, dB, rho);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        Ep[a] = k.Er[a] + dEp[a];
        Bn[a] = k.Br[a] + dB[a];
    }

    // 3. recovery
    R beta[3], lambda, s_old;
    const int it = landau(T, old, k, beta, lambda, s_old);
    Prim<R> nw;
    R J[3], n_dev, eps_dev;
    const bool ok = it > 0;
    if (ok) {
        const R b2 = beta[0] * beta[0] + beta[1] * beta[1] + beta[2] * beta[2];
        const R g2 = R(1) / (R(1) - b2);
        const R g = sqrt(g2);
        eps_dev = lambda - s_old;
        // n = N^0 / U^0: n - n_r = (dN0 - n_r (g - 1)) / g, g - 1 = g^2 b^2 / (g + 1)
        n_dev = (dN0 - k.n_r * (g2 * b2 / (g + R(1)))) / g;
        nw.eps = k.eps_r + eps_dev;
        nw.n = k.n_r + n_dev;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            nw.u[a] = k.c * beta[a];
            nw.B[a] = Bn[a];
        }
        nw.rho = rho;
        ohm_solve(Ep, nw.u, nw.B, rho, g2, k, nw.E, J);
    } else {
        nw = old;
        n_dev = old.n - k.n_r;
        eps_dev = old.eps - k.eps_r;
        ohm_current(old.E, old.u, old.B, old.rho, k, J);
    }

    // 4. collisions and stores
    R dE[3], dBn[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        dE[a] = nw.E[a] - k.Er[a];
        dBn[a] = ok ? dB[a] : nw.B[a] - k.Br[a];
    }
    EqCell<R> q;
    eq_cell(nw, n_dev, eps_dev, dE, dBn, k, q);
    CollideFG<0, Cfg>::run(A, c, fd, gd, q);
    const bool em_coll = (A.flags & FLAG_NO_EM_COLLISION) == 0;
    // h_c - h_ref = 2 h^eq(E - Er, B - Br, J) - (h - h_ref)  (Eq. Maxwell-eq is linear)
    CollideH<0, Cfg>::run(A, c, h, dE, dBn, J, em_coll);
    A.hout[24 * A.stride + c] = (typename Cfg::hpop)(em_coll ? R(2) * nw.rho - h[24] : h[24]);

    A.pout[P_N * A.stride + c] = (typename Cfg::prim)nw.n;
    A.pout[P_EPS * A.stride + c] = (typename Cfg::prim)nw.eps;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        A.pout[(P_U + a) * A.stride + c] = (typename Cfg::prim)nw.u[a];
        A.pout[(P_E + a) * A.stride + c] = (typename Cfg::prim)nw.E[a];
        A.pout[(P_B + a) * A.stride + c] = (typename Cfg::prim)nw.B[a];
    }
    A.pout[P_RHO * A.stride + c] = (typename Cfg::prim)nw.rho;

    // recovery counters, aggregated per warp
    const unsigned mask = __activemask();
    const unsigned fail = __reduce_add_sync(mask, ok ? 0u : 1u);
    const unsigned isum = __reduce_add_sync(mask, ok ? (unsigned)it : 0u);
    const unsigned imax = __reduce_max_sync(mask, ok ? (unsigned)it : 0u);
    if ((threadIdx.x + threadIdx.y * blockDim.x) % 32 == (unsigned)(__ffs(mask) - 1)) {
        if (fail) atomicAdd(&A.stats[0], (unsigned long long)fail);
        atomicAdd(&A.stats[1], (unsigned long long)isum);
        atomicMax(&A.stats[2], (unsigned long long)imax);
    }
}

template <class Cfg>
cudaError_t launch_step(const StepArgs<Cfg>& A, cudaStream_t stream)
{
    const int bx = A.nx >= 128 ? 128 : (A.nx >= 64 ? 64 : 32);
    const int by = 128 / bx;
    dim3 block(bx, by, 1);
    dim3 grid((A.nx + bx - 1) / bx, (A.ny + by - 1) / by, A.nz);
    if (A.nz > 1)
        step_kernel<Cfg, true><<<grid, block, 0, stream>>>(A);
    else
        step_kernel<Cfg, false><<<grid, block, 0, stream>>>(A);
    return cudaGetLastError();
}

}  // namespace lb

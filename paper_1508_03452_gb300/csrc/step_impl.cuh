// step_impl.cuh -- the fused time step of the RRMHD lattice Boltzmann method
// (arXiv:1508.03452, Sec. III), one thread per cell.
//
// The state holds post-collision populations, so one kernel does, per cell:
//   1. streaming (pull): f, g by the flux-limited (minmod) finite-volume
//      update of Eq. eq:rlb plus the bulk-viscosity term for f; h by the exact
//      D3Q13 hop of Eq. LB_Maxwell;
//   2. moments T^{mu nu}, N^mu (reference rest state added back), E', B,
//      rho_c (Eqs. Cal_E, Cal_B, Cal_rhoc);
//   3. recovery (coupling subsection): the Landau eigen-solve of T - eps0 F F
//      iterated with the Ohm-coupled E solve until the tensor's E reproduces
//      itself (starting from the previous step's E and the streamed B), then
//      n = N^0 / U^0, J (Eq. Ex_force) and the EOS (Eq. EOS); optionally the
//      body force of the flare set-up before it and the relaxed
//      initialisation's reset after it (open-face variant);
//   4. collision at the new time level: Anderson-Witting for f towards Eq.
//      Dis_fun_EM, BGK for g towards Eq. Hupp, tau_h = 1/2 for h
//      (h -> 2 h^eq - h) towards Eq. Maxwell-eq; store populations and
//      primitives.
#pragma once
#include "common.cuh"
#include "mlp.cuh"
#include "tma.cuh"

namespace lb {

// F_out - F_in of the limited upwind face values along one axis, for values
// ordered along the flow: um2 (two cells upwind), um1, u0 (this cell), up1.
// Face value = upwind + (1 - C)/2 * minmod(downwind - upwind, upwind - upwind2).
template <class R>
__device__ __forceinline__ R minmod(R a, R b)
{
    // the argument of smaller magnitude when both have the same sign, else 0:
    // the median of (a, b, 0), as four min / max operations
    return fmax(fmin(a, b), fmin(fmax(a, b), R(0)));
}

template <class R>
__device__ __forceinline__ R flux_diff(R um2, R um1, R u0, R up1, R kappa)
{
    // Fout - Fin = (u0 - um1) + kappa [minmod(up1 - u0, u0 - um1) - minmod(u0 - um1, um1 - um2)]
    const R d0 = u0 - um1;
    return d0 + kappa * (minmod(up1 - u0, d0) - minmod(d0, um1 - um2));
}

// Relative element offsets of the neighbours d = -2..+2 of one cell along each
// axis (index 2 is the cell itself), with the periodic wrap or the open-face
// clamp already applied; y offsets include the factor nx, z offsets nx ny.
struct Off {
    int x[5], y[5], z[5];
};

// neighbour coordinate s = x + d, |d| <= 2, wrapped (periodic) or clamped:
// one branch-free correction when the axis has at least 2 cells
__device__ __forceinline__ int near_coord(int s, int n, int periodic)
{
    if (n < 2) return wrap_coord(s, n, periodic);
    if (periodic) return s < 0 ? s + n : (s >= n ? s - n : s);
    return s < 0 ? 0 : (s >= n ? n - 1 : s);
}

template <bool IS3D>
__device__ __forceinline__ Off make_off(int x, int y, int z, int nx, int ny, int nz, const int* per)
{
    Off o;
#pragma unroll
    for (int d = -2; d <= 2; ++d) {
        o.x[d + 2] = near_coord(x + d, nx, per[0]) - x;
        o.y[d + 2] = (near_coord(y + d, ny, per[1]) - y) * nx;
        o.z[d + 2] = IS3D ? (near_coord(z + d, nz, per[2]) - z) * nx * ny : 0;  // unused in 2-D runs
    }
    return o;
}

// Moments of the streamed f_I, g_I (deviations): T^{mu nu} with p = (1, q chat)
// and N^mu.
template <int I, class R>
__device__ __forceinline__ void acc_fg(R f, R g, R (&Tm)[10], R& Nm, R (&Na)[3])
{
    constexpr int cx = c19(I, 0), cy = c19(I, 1), cz = c19(I, 2);
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
    Nm += g;
    if (cx) Na[0] += R(cx) * g;
    if (cy) Na[1] += R(cy) * g;
    if (cz) Na[2] += R(cz) * g;
}

// Moments of the opposite pair (I, J = -I) of one group from the sums and
// differences of its f and g: the even moments take f_I + f_J, the odd ones
// (momentum, particle flux) f_I - f_J, so these sums run over values of the
// momentum's size, and a group costs 9 (axis) or 13 (diagonal) additions
// instead of 10 or 18. Used in 2-D runs; in 3-D the longer stencil's registers
// are allocated better with the per-population sums (measured: +2.8 % float32
// and +4.4 % float16 in 2-D, -1.9 % in 3-D).
template <int I, class R>
__device__ __forceinline__ void acc_fg_pair(R fI, R gI, R fJ, R gJ, R (&Tm)[10], R& Nm, R (&Na)[3])
{
    constexpr int cx = c19(I, 0), cy = c19(I, 1), cz = c19(I, 2);
    const R sf = fI + fJ, df = fI - fJ, sg = gI + gJ, dg = gI - gJ;
    Tm[0] += sf;
    if (cx) Tm[1] += R(cx) * df;
    if (cy) Tm[2] += R(cy) * df;
    if (cz) Tm[3] += R(cz) * df;
    if (cx) Tm[4] += sf;  // xx (chat^2 = 1)
    if (cy) Tm[5] += sf;  // yy
    if (cz) Tm[6] += sf;  // zz
    if (cx * cy) Tm[7] += R(cx * cy) * sf;  // c_a c_b is even in the direction
    if (cx * cz) Tm[8] += R(cx * cz) * sf;
    if (cy * cz) Tm[9] += R(cy * cz) * sf;
    Nm += sg;
    if (cx) Na[0] += R(cx) * dg;
    if (cy) Na[1] += R(cy) * dg;
    if (cz) Na[2] += R(cz) * dg;
}

// The four streamed populations of fluid group G (pre-collision values at
// t + dt of f_I, g_I, f_J, g_J for the opposite directions I = 2G-1, J = 2G);
// ld(a, d) gives the group's 4-vector of the cell d cells away along axis a
// (d = 0: this cell). Along an axis where I moves by s = +-1 the values at
// -2..+2 serve both directions (I's upwind side is J's downwind side); along
// an axis where neither moves only the +-1 values enter (the bulk viscosity
// of f). The update is linear and the limiter positively homogeneous
// (minmod(s a, s b) = s minmod(a, b), s > 0), so float16 values are streamed
// in their stored units and scaled once.
template <int G, bool IS3D, class Cfg, class Ld>
__device__ __forceinline__ V4<typename Cfg::real> stream_group(const Ld& ld, const Phys<typename Cfg::real>& k,
                                                               const HalfScale& hs)
{
    using R = typename Cfg::real;
    constexpr int I = 2 * G - 1, J = 2 * G;
    constexpr int s[3] = {c19(I, 0), c19(I, 1), c19(I, 2)};
    const V4<R> v0 = ld(0, 0);
    R fl[4] = {R(0), R(0), R(0), R(0)}, lap[2] = {R(0), R(0)};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (a == 2 && !IS3D) continue;
        if (s[a] != 0) {
            const V4<R> m2 = ld(a, -2), m1 = ld(a, -1), p1 = ld(a, 1), p2 = ld(a, 2);
            const V4<R>& i2 = s[a] > 0 ? m2 : p2;  // I's second upwind cell (-2s)
            const V4<R>& i1 = s[a] > 0 ? m1 : p1;  // I's upwind cell (-s) = J's downwind cell
            const V4<R>& ip = s[a] > 0 ? p1 : m1;  // I's downwind cell (+s) = J's upwind cell
            const V4<R>& j2 = s[a] > 0 ? p2 : m2;  // J's second upwind cell (+2s)
            fl[0] += flux_diff(i2.x, i1.x, v0.x, ip.x, k.kappa);
            fl[1] += flux_diff(i2.y, i1.y, v0.y, ip.y, k.kappa);
            fl[2] += flux_diff(j2.z, ip.z, v0.z, i1.z, k.kappa);
            fl[3] += flux_diff(j2.w, ip.w, v0.w, i1.w, k.kappa);
            lap[0] += (i1.x + ip.x) - R(2) * v0.x;
            lap[1] += (ip.z + i1.z) - R(2) * v0.z;
        } else {
            const V4<R> m1 = ld(a, -1), p1 = ld(a, 1);
            lap[0] += (m1.x + p1.x) - R(2) * v0.x;
            lap[1] += (m1.z + p1.z) - R(2) * v0.z;
        }
    }
    V4<R> out;
    out.x = v0.x - k.C * fl[0];
    out.x += k.kvisc * lap[0];
    out.y = v0.y - k.C * fl[1];
    out.z = v0.z - k.C * fl[2];
    out.z += k.kvisc * lap[1];
    out.w = v0.w - k.C * fl[3];
    if constexpr (Cfg::kHalf) {
        out.x *= hs.f[I];
        out.y *= hs.g[I];
        out.z *= hs.f[J];
        out.w *= hs.g[J];
    }
    return out;
}

// the streamed rest pair (f_0, g_0): it does not move and takes no bulk viscosity
template <class Cfg>
__device__ __forceinline__ V2<typename Cfg::real> rest_pair(V2<typename Cfg::real> v, const HalfScale& hs)
{
    if constexpr (Cfg::kHalf) {
        v.x *= hs.f[0];
        v.y *= hs.g[0];
    }
    return v;
}

// Shared-memory slots of one thread's streamed (pre-collision) populations.
// Vector order (VEC; t: the thread's index in its block of nth threads): fluid
// group G (1..9) as a 4-vector at element 4 ((G - 1) nth + t), the rest pair
// {f_0, g_0} at 36 nth + 2 t, Maxwell pair m (0..11) at 38 nth + 2 (m nth + t),
// h_24 at 62 nth + t, so that a group or pair is one vector access. Row order
// (!VEC): one row of nth values per population, f_i in row i, g_i in 19 + i,
// h_k in 38 + k (float16 storage runs faster with it: fewer registers live
// around the vector accesses).
template <class R, bool VEC>
struct Slots {
    R* b;
    int nth, t;
    __device__ __forceinline__ R* f(int i) const
    {
        if constexpr (VEC)
            return i == 0 ? b + 36 * nth + 2 * t : b + 4 * (((i - 1) >> 1) * nth + t) + 2 * ((i - 1) & 1);
        else
            return b + i * nth + t;
    }
    __device__ __forceinline__ R* g(int i) const
    {
        if constexpr (VEC)
            return f(i) + 1;
        else
            return b + (19 + i) * nth + t;
    }
    __device__ __forceinline__ R* h(int k) const
    {
        if constexpr (VEC)
            return k < 24 ? b + 38 * nth + 2 * ((k >> 1) * nth + t) + (k & 1) : b + 62 * nth + t;
        else
            return b + (38 + k) * nth + t;
    }
};

// the slots of a storage configuration
template <class Cfg>
using CfgSlots = Slots<typename Cfg::real, Cfg::kVecSlots>;

template <class R>
__device__ __forceinline__ void st_v4(R* p, const V4<R>& v)
{
    if constexpr (sizeof(R) == 8) {
        reinterpret_cast<double2*>(p)[0] = make_double2(v.x, v.y);
        reinterpret_cast<double2*>(p)[1] = make_double2(v.z, v.w);
    } else {
        *reinterpret_cast<float4*>(p) = make_float4(v.x, v.y, v.z, v.w);
    }
}
template <class R>
__device__ __forceinline__ V4<R> ld_v4(const R* p)
{
    if constexpr (sizeof(R) == 8) {
        const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
        return {a.x, a.y, b.x, b.y};
    } else {
        const float4 a = *reinterpret_cast<const float4*>(p);
        return {a.x, a.y, a.z, a.w};
    }
}
template <class R>
__device__ __forceinline__ void st_v2(R* p, R x, R y)
{
    if constexpr (sizeof(R) == 8)
        *reinterpret_cast<double2*>(p) = make_double2(x, y);
    else
        *reinterpret_cast<float2*>(p) = make_float2(x, y);
}
template <class R>
__device__ __forceinline__ V2<R> ld_v2(const R* p)
{
    if constexpr (sizeof(R) == 8) {
        const double2 a = *reinterpret_cast<const double2*>(p);
        return {a.x, a.y};
    } else {
        const float2 a = *reinterpret_cast<const float2*>(p);
        return {a.x, a.y};
    }
}

// group G (f_I, g_I, f_J, g_J), the rest pair and Maxwell pair m in the slots
template <class R, bool VEC>
__device__ __forceinline__ void put_group(const Slots<R, VEC>& S, int G, const V4<R>& v)
{
    if constexpr (VEC) {
        st_v4(S.f(2 * G - 1), v);
    } else {
        *S.f(2 * G - 1) = v.x;
        *S.g(2 * G - 1) = v.y;
        *S.f(2 * G) = v.z;
        *S.g(2 * G) = v.w;
    }
}
template <class R, bool VEC>
__device__ __forceinline__ V4<R> get_group(const Slots<R, VEC>& S, int G)
{
    if constexpr (VEC)
        return ld_v4(S.f(2 * G - 1));
    else
        return {*S.f(2 * G - 1), *S.g(2 * G - 1), *S.f(2 * G), *S.g(2 * G)};
}
template <class R, bool VEC>
__device__ __forceinline__ void put_pair(R* a, R* b, R x, R y)
{
    if constexpr (VEC) {
        st_v2(a, x, y);
    } else {
        *a = x;
        *b = y;
    }
}
template <class R, bool VEC>
__device__ __forceinline__ V2<R> get_pair(const R* a, const R* b)
{
    if constexpr (VEC)
        return ld_v2(a);
    else
        return {*a, *b};
}

// slots and moments of the streamed populations of group G (G = 0: the rest pair in v.x, v.y)
template <int G, class Cfg, bool PAIRS>
__device__ __forceinline__ void store_group(const V4<typename Cfg::real>& v, const CfgSlots<Cfg>& S,
                                            typename Cfg::real (&Tm)[10], typename Cfg::real& Nm,
                                            typename Cfg::real (&Na)[3])
{
    if constexpr (G == 0) {
        put_pair<typename Cfg::real, Cfg::kVecSlots>(S.f(0), S.g(0), v.x, v.y);
        acc_fg<0>(v.x, v.y, Tm, Nm, Na);
    } else {
        constexpr int I = 2 * G - 1, J = 2 * G;
        put_group(S, G, v);
        if constexpr (PAIRS) {
            acc_fg_pair<I>(v.x, v.y, v.z, v.w, Tm, Nm, Na);
        } else {
            acc_fg<I>(v.x, v.y, Tm, Nm, Na);
            acc_fg<J>(v.z, v.w, Tm, Nm, Na);
        }
    }
}

// Streams f and g group by group (G onwards; G = 0 is the rest pair) into the
// shared-memory slots and accumulates their moments in the order of the
// populations.
template <int G, bool IS3D, class Cfg>
struct StreamAll {
    using R = typename Cfg::real;
    static __device__ __forceinline__ void run(const StepArgs<Cfg>& A, const Off& o, int64_t c, const CfgSlots<Cfg>& S,
                                               R (&Tm)[10], R& Nm, R (&Na)[3])
    {
        if constexpr (G == 0) {
            const V2<R> v = rest_pair<Cfg>(ld_fgpair<Cfg>(A.fgin + fg_elem(0, 0, c, A.stride)), A.hs);
            store_group<0, Cfg, !IS3D>(V4<R>{v.x, v.y, R(0), R(0)}, S, Tm, Nm, Na);
        } else {
            const typename Cfg::pop* p = A.fgin + fg_elem(2 * G - 1, 0, c, A.stride);
            auto ld = [&](int a, int d) {
                const int* oa = a == 0 ? o.x : (a == 1 ? o.y : o.z);
                return ld_quad<Cfg>(d == 0 ? p : p + 4 * oa[d + 2]);
            };
            store_group<G, Cfg, !IS3D>(stream_group<G, IS3D, Cfg>(ld, A.k, A.hs), S, Tm, Nm, Na);
        }
        StreamAll<G + 1, IS3D, Cfg>::run(A, o, c, S, Tm, Nm, Na);
    }
};
template <bool IS3D, class Cfg>
struct StreamAll<kFGroups + 1, IS3D, Cfg> {
    using R = typename Cfg::real;
    static __device__ __forceinline__ void run(const StepArgs<Cfg>&, const Off&, int64_t, const CfgSlots<Cfg>&,
                                               R (&)[10],
                                               R&, R (&)[3]) {}
};

// Exact D3Q13 pull h_k(x) = h_c,k(x - hop_k) into its slot, accumulating
// E' - Er (before the sqrt(2) c / 2 factor), the plane-normal B - Br sums and
// rho_c; the pair k = 2m, 2m + 1 hops the same way and arrives in one load.
template <int K, class R>
__device__ __forceinline__ void acc_h(R hv, R (&dEp)[3], R (&bn)[3], R& rho)
{
    constexpr int p = K / 8, i = (K % 8) / 2, j = K % 2, ie = (i + 3) % 4;
    rho += hv;
    constexpr int se = j == 0 ? 1 : -1;  // e_{i1} = -e_{i0}
    dEp[plane_a1(p)] += R(se * hop_s1(ie)) * hv;
    dEp[plane_a2(p)] += R(se * hop_s2(ie)) * hv;
    bn[plane_normal(p)] += R(-se * plane_orient(p)) * hv;  // b_{i0} = -o_p, b_{i1} = +o_p
}

template <int M, bool IS3D, class Cfg>
struct PullH {
    using R = typename Cfg::real;
    static __device__ __forceinline__ void run(const StepArgs<Cfg>& A, const Off& o, int64_t c, const CfgSlots<Cfg>& S,
                                               R (&dEp)[3], R (&bn)[3], R& rho)
    {
        constexpr int K = 2 * M;
        int off = o.x[2 - hop13(K, 0)] + o.y[2 - hop13(K, 1)];
        if (IS3D) off += o.z[2 - hop13(K, 2)];
        const V2<R> hv = ld_hpair<Cfg>(A.hin + h_elem(K, c + off, A.stride));
        put_pair<R, Cfg::kVecSlots>(S.h(K), S.h(K + 1), hv.x, hv.y);
        acc_h<K>(hv.x, dEp, bn, rho);
        acc_h<K + 1>(hv.y, dEp, bn, rho);
        PullH<M + 1, IS3D, Cfg>::run(A, o, c, S, dEp, bn, rho);
    }
};
template <bool IS3D, class Cfg>
struct PullH<12, IS3D, Cfg> {
    using R = typename Cfg::real;
    static __device__ __forceinline__ void run(const StepArgs<Cfg>&, const Off&, int64_t, const CfgSlots<Cfg>&,
                                               R (&)[3],
                                               R (&)[3], R&) {}
};

// (f_i^eq, g_i^eq) deviations of population I as one float32 pair: the
// per-direction parts of Eq. Dis_fun_EM and Eq. Hupp share their structure
// (even + s_a odd_a + s_b odd_b + s_a s_b cross), so they are formed with pair
// instructions (the same terms as feq_dev / geq_dev, summed in pairs)
template <int I>
__device__ __forceinline__ float2 eq_pair(const EqCell<float>& q)
{
    constexpr int a = ax1(I), b = ax2(I);
    float2 v;
    if constexpr (a < 0) {
        v = make_float2(q.f_rest, q.g_base);
    } else if constexpr (b < 0) {
        constexpr float sa = (float)c19(I, a);
        v = __ffma2_rn(make_float2(sa, sa), make_float2(q.f_odd[a], q.g_lin[a]),
                       make_float2(q.f_even_ax[a], q.g_base + q.g_sq[a]));
    } else {
        constexpr int m = a + b - 1;
        constexpr float sa = (float)c19(I, a), sb = (float)c19(I, b), sab = sa * sb;
        v = __ffma2_rn(make_float2(sab, sab), make_float2(q.f_cross[m], q.g_x[m]),
                       make_float2(q.f_even_dg[m], q.g_base + q.g_sq[a] + q.g_sq[b]));
        v = __ffma2_rn(make_float2(sa, sa), make_float2(q.f_odd[a], q.g_lin[a]), v);
        v = __ffma2_rn(make_float2(sb, sb), make_float2(q.f_odd[b], q.g_lin[b]), v);
    }
    return __fmul2_rn(make_float2((float)w19(I), (float)wg19(I)), v);
}

// post-collision (f_I, g_I) of one cell from the streamed values (fd, gd)
template <int I, class Cfg>
__device__ __forceinline__ void collide_fg(const StepArgs<Cfg>& A, typename Cfg::real fd, typename Cfg::real gd,
                                           const EqCell<typename Cfg::real>& q, typename Cfg::real& fo,
                                           typename Cfg::real& go)
{
    using R = typename Cfg::real;
    const R K = k_aw<I>(q);
    if constexpr (sizeof(R) == 4) {
        // f and g of one direction relax in lock-step: the float32 pair
        // instructions do both (fd - K (fd - feq), gd - (dt/tau)(gd - geq))
        const float2 eq = eq_pair<I>(q);
        const float2 d = make_float2(fd, gd);
        const float2 t = __fadd2_rn(d, make_float2(-eq.x, -eq.y));
        const float2 o = __ffma2_rn(make_float2(-K, -A.k.inv_tau), t, d);
        fo = o.x;
        go = o.y;
    } else {
        fo = fd - K * (fd - feq_dev<I>(q));
        go = gd - A.k.inv_tau * (gd - geq_dev<I>(q));
    }
}

// Collision of f and g and the stores, group by group (G onwards) into cell c
// of the output buffer.
template <int G, class Cfg>
struct CollideFG {
    using R = typename Cfg::real;
    static __device__ __forceinline__ void run(const StepArgs<Cfg>& A, int64_t c, const CfgSlots<Cfg>& S,
                                               const EqCell<R>& q)
    {
        if constexpr (G == 0) {
            R fo, go;
            const V2<R> d = get_pair<R, Cfg::kVecSlots>(S.f(0), S.g(0));
            collide_fg<0, Cfg>(A, d.x, d.y, q, fo, go);
            st_fgpair<Cfg>(A.fgout + fg_elem(0, 0, c, A.stride), fo, go, A.hs.finv[0], A.hs.ginv[0]);
        } else {
            constexpr int I = 2 * G - 1, J = 2 * G;
            V4<R> v;
            const V4<R> d = get_group(S, G);
            collide_fg<I, Cfg>(A, d.x, d.y, q, v.x, v.y);
            collide_fg<J, Cfg>(A, d.z, d.w, q, v.z, v.w);
            const V4<float> inv = {A.hs.finv[I], A.hs.ginv[I], A.hs.finv[J], A.hs.ginv[J]};
            st_quad<Cfg>(A.fgout + fg_elem(I, 0, c, A.stride), v, inv);
        }
        CollideFG<G + 1, Cfg>::run(A, c, S, q);
    }
};
template <class Cfg>
struct CollideFG<kFGroups + 1, Cfg> {
    using R = typename Cfg::real;
    static __device__ __forceinline__ void run(const StepArgs<Cfg>&, int64_t, const CfgSlots<Cfg>&, const EqCell<R>&) {}
};

// Collision of the Maxwell pair (2M, 2M + 1) into cell c of the output buffer.
template <int M, class Cfg>
struct CollideH {
    using R = typename Cfg::real;
    static __device__ __forceinline__ void run(const StepArgs<Cfg>& A, int64_t c, const CfgSlots<Cfg>& S, const R* E,
                                               const R* B, const R* J, bool em_coll)
    {
        constexpr int K = 2 * M;
        const V2<R> hs = get_pair<R, Cfg::kVecSlots>(S.h(K), S.h(K + 1));
        const R h0 = hs.x, h1 = hs.y;
        const R v0 = em_coll ? R(2) * heq13<K>(E, B, J, A.k) - h0 : h0;
        const R v1 = em_coll ? R(2) * heq13<K + 1>(E, B, J, A.k) - h1 : h1;
        st_hpair<Cfg>(A.hout + h_elem(K, c, A.stride), v0, v1);
        CollideH<M + 1, Cfg>::run(A, c, S, E, B, J, em_coll);
    }
};
template <class Cfg>
struct CollideH<12, Cfg> {
    using R = typename Cfg::real;
    static __device__ __forceinline__ void run(const StepArgs<Cfg>&, int64_t, const CfgSlots<Cfg>&, const R*, const R*,
                                               const R*, bool) {}
};

constexpr int kStepSlots = 63;  // 19 f + 19 g + 25 h pre-collision values per cell in shared memory
#ifndef LB_STEP_MIN_BLOCKS
// resident 128-thread blocks per SM targeted for 2-D runs in float32 storage:
// 5 (at most 102 registers) is 2.4 % faster than 4 with the vector loads,
// stores and slots, which hold fewer values live
#define LB_STEP_MIN_BLOCKS 5
#endif
#ifndef LB_STEP_MIN_BLOCKS_3D
// 3-D runs in float32 storage: 4 (128 registers); at 5 the longer stencil
// spills and the 256^3 flux rope runs 14 % slower
#define LB_STEP_MIN_BLOCKS_3D 4
#endif
#ifndef LB_STEP_BX
#define LB_STEP_BX 128  // block width along x (the block is LB_STEP_BX x 128 / LB_STEP_BX)
#endif
#ifndef LB_STEP_MIN_BLOCKS_F16
#define LB_STEP_MIN_BLOCKS_F16 4  // float16-deviation storage: 128 registers (no spills) beat 96 by 12 %
#endif
#ifndef LB_STEP_MIN_BLOCKS_MLP
#define LB_STEP_MIN_BLOCKS_MLP 3  // the learned-seed variant: 3 blocks (168 registers) beat 4 by 18 %
#endif
// float64: 2 blocks
template <class Cfg, int SEED, bool IS3D = false>
struct StepMinBlocks {
    static constexpr int value = sizeof(typename Cfg::real) == 8 ? 2
                                 : SEED == SEED_MLP             ? LB_STEP_MIN_BLOCKS_MLP
                                 : Cfg::kHalf                   ? LB_STEP_MIN_BLOCKS_F16
                                 : IS3D                         ? LB_STEP_MIN_BLOCKS_3D
                                                                : LB_STEP_MIN_BLOCKS;
};

// Photospheric body force (reading R25) on the streamed f of one cell: the
// rest population takes F.u dt, a moving one c dt (F . chat_i) / (10 q)
// (p_i = (1, q chat_i), sum_i chat_i^a chat_i^b = 10 delta_ab), so the added
// moments are T^00 += F.u dt and T^0a += c dt F^a, nothing else.
template <int I, class Cfg>
struct AddForce {
    using R = typename Cfg::real;
    static __device__ __forceinline__ void run(const CfgSlots<Cfg>& S, const R (&F)[3], R s, R w)
    {
        constexpr int cx = c19(I, 0), cy = c19(I, 1), cz = c19(I, 2);
        if constexpr (cx == 0 && cy == 0 && cz == 0)
            *S.f(I) += w;
        else
            *S.f(I) += s * (R(cx) * F[0] + R(cy) * F[1] + R(cz) * F[2]);
        AddForce<I + 1, Cfg>::run(S, F, s, w);
    }
};
template <class Cfg>
struct AddForce<19, Cfg> {
    using R = typename Cfg::real;
    static __device__ __forceinline__ void run(const CfgSlots<Cfg>&, const R (&)[3], R, R) {}
};

// Relaxed initialisation (reading R27): f and g of the cell at the
// equilibrium of its (reset) primitives, so that the collision returns it.
template <int I, class Cfg>
struct SetEqFG {
    using R = typename Cfg::real;
    static __device__ __forceinline__ void run(const CfgSlots<Cfg>& S, const EqCell<R>& q)
    {
        *S.f(I) = feq_dev<I>(q);
        *S.g(I) = geq_dev<I>(q);
        SetEqFG<I + 1, Cfg>::run(S, q);
    }
};
template <class Cfg>
struct SetEqFG<19, Cfg> {
    using R = typename Cfg::real;
    static __device__ __forceinline__ void run(const CfgSlots<Cfg>&, const EqCell<R>&) {}
};

// Relaxed initialisation: move the B carried by the streamed h by dB through
// the populations whose b carries it, h_k += (dB . b_k) / 8 (sum b b^T = 8 I,
// sum e b^T = 0, sum b = 0: E' and rho_c do not move).
template <int K, class Cfg>
struct ShiftHB {
    using R = typename Cfg::real;
    static __device__ __forceinline__ void run(const CfgSlots<Cfg>& S, const R (&dB)[3])
    {
        constexpr int p = K / 8, j = K % 2, se = j == 0 ? 1 : -1;
        *S.h(K) += R(-se * plane_orient(p)) * R(0.125) * dB[plane_normal(p)];
        ShiftHB<K + 1, Cfg>::run(S, dB);
    }
};
template <class Cfg>
struct ShiftHB<24, Cfg> {
    using R = typename Cfg::real;
    static __device__ __forceinline__ void run(const CfgSlots<Cfg>&, const R (&)[3]) {}
};

// warp-wide maximum of a non-negative float64, folded into *dst (atomicMax on
// the bit pattern, which orders non-negative doubles)
__device__ __forceinline__ void warp_max_into(double v, double* dst)
{
    const unsigned mask = __activemask();
    unsigned long long b = (unsigned long long)__double_as_longlong(v);
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long t = __shfl_xor_sync(mask, b, o);
        b = t > b ? t : b;
    }
    if ((threadIdx.x + blockDim.x * threadIdx.y) % 32 == (unsigned)(__ffs(mask) - 1))
        atomicMax(reinterpret_cast<unsigned long long*>(dst), b);
}

// ---------------------------------------------------------------------------
// TMA tile path (2-D runs with periodic faces, float32 / float16 storage).
// A block updates a tile of kTileW x kTileH cells (one thread per cell, thread
// tid = tx + kTileW ty). Its inputs arrive by tensor-map copies into shared
// memory: the f, g planes of two directions at a time, then the h planes four
// at a time, each as a box of the tile plus a halo of 2 rows and one 16-byte
// unit of columns on either side (the minmod stencil reaches 2 cells along
// each axis, the Maxwell hop 1 cell diagonally), through a ring of
// kRingStages buffers refilled as the block consumes them; the primitives of
// the tile come in one box. The stencil then reads shared memory at
// compile-time offsets. The post-collision populations and primitives are
// collected in shared memory and written back by three tensor-map stores.
// Tiles whose halo would leave the grid (within 2 rows or one unit of columns
// of an edge) take the per-cell path with its periodic wrap.
// ---------------------------------------------------------------------------
#ifndef LB_RING_STAGES
#define LB_RING_STAGES 4
#endif
constexpr int kRingStages = LB_RING_STAGES;  // copies in flight per block
constexpr int kFgStages = 1 + kFGroups;          // the rest pairs, then fluid groups 1..9
constexpr int kHStages = 7;                       // h pairs (0, 1), (2, 3), ..., (10, 11), then h_24
constexpr int kTileStages = kFgStages + kHStages;  // 17

template <class Cfg>
struct TileGeo {
    using pop = typename Cfg::pop;
    static constexpr int PX = tile_halo_x((int)sizeof(pop));  // f, g column halo (every box starts 16-byte aligned)
    static constexpr int PXH = tile_halo_x(4);                // h column halo (float)
    static constexpr int BWF = kTileW + 2 * PX;       // f, g box width in cells
    static constexpr int BWH = kTileW + 2 * PXH;      // h box width in cells
    static constexpr int BH = kTileH + 2 * kTileHaloY;  // box height
    static constexpr int FG_CELLS = BWF * BH;         // cells of an f, g box
    static constexpr int H_PLANE = BWH * BH;          // cells of an h box
    static constexpr unsigned FG_STAGE_BYTES = 4u * FG_CELLS * sizeof(pop);  // one group
    static constexpr unsigned R_STAGE_BYTES = 2u * FG_CELLS * sizeof(pop);   // the rest pairs
    static constexpr unsigned H_STAGE_BYTES = 4u * H_PLANE * sizeof(float);  // two h pairs
    static constexpr unsigned H24_STAGE_BYTES = 1u * H_PLANE * sizeof(float);
    static constexpr unsigned STAGE_BYTES =
        ((FG_STAGE_BYTES > H_STAGE_BYTES ? FG_STAGE_BYTES : H_STAGE_BYTES) + 127u) / 128u * 128u;
    static constexpr unsigned PRIM_BYTES = (unsigned)NPRIM * kTileThreads * sizeof(float);
};

// The block's view of its tile buffers (shared memory) and maps.
template <class Cfg>
struct TileCtx {
    unsigned char* ring;  // kRingStages x STAGE_BYTES
    float* pbuf;          // [3][kTileThreads][4]: input primitive 4-vectors, then the output ones
    uint64_t* bar;        // kRingStages ring barriers, then the primitives' barrier
    int* abort;           // set when a wait ran out: the whole block then stops
    const TileMaps* M;
    int x0, y0;           // this tile
    int nx0, ny0;         // the block's next tile (has_next), whose first stages follow in the ring
    bool has_next;
    int gbase;            // ring index of this tile's stage 0 (stages are numbered over the block's tiles)
    uint32_t ppar;        // phase parity of this tile's primitive copy
};

// issue the copy of stage j of the tile at (x0, y0), ring index g (one thread);
// the x coordinates count elements of the maps' rows (4 or 2 per cell for the
// groups and pairs)
template <class Cfg>
__device__ __forceinline__ void tile_issue(const TileCtx<Cfg>& t, int g, int x0, int y0, int j)
{
    using G = TileGeo<Cfg>;
    const int s = g % kRingStages;
    unsigned char* dst = t.ring + (size_t)s * G::STAGE_BYTES;
    if (j == 0) {
        mbar_arrive_expect_tx(&t.bar[s], G::R_STAGE_BYTES);
        tma_load_2d(dst, &t.M->r_in, 2 * (x0 - G::PX), y0 - kTileHaloY, &t.bar[s]);
    } else if (j < kFgStages) {
        mbar_arrive_expect_tx(&t.bar[s], G::FG_STAGE_BYTES);
        tma_load_3d(dst, &t.M->fg_in, 4 * (x0 - G::PX), y0 - kTileHaloY, j - 1, &t.bar[s]);
    } else if (j < kTileStages - 1) {
        mbar_arrive_expect_tx(&t.bar[s], G::H_STAGE_BYTES);
        tma_load_3d(dst, &t.M->h_in, 2 * (x0 - G::PXH), y0 - kTileHaloY, 2 * (j - kFgStages), &t.bar[s]);
    } else {
        mbar_arrive_expect_tx(&t.bar[s], G::H24_STAGE_BYTES);
        tma_load_2d(dst, &t.M->h24_in, x0 - G::PXH, y0 - kTileHaloY, &t.bar[s]);
    }
}

// Stage J of the ring: wait for its copy, stream its populations (the same
// operations in the same order as the per-cell path), release the buffer and
// refill it with stage J + kRingStages. Returns false (for every thread of the
// block) if a copy did not arrive in time.
template <int J, class Cfg>
struct TileStages {
    using R = typename Cfg::real;
    static __device__ __forceinline__ bool run(const TileCtx<Cfg>& t, const StepArgs<Cfg>& A, int tid,
                                               const CfgSlots<Cfg>& S, R (&Tm)[10], R& Nm, R (&Na)[3], R (&dEp)[3],
                                               R (&bn)[3], R& rho)
    {
        using G = TileGeo<Cfg>;
        using pop = typename Cfg::pop;
        const int g = t.gbase + J;
        const int s = g % kRingStages;
        const unsigned char* buf = t.ring + (size_t)s * G::STAGE_BYTES;
        const int tx = tid % kTileW, ty = tid / kTileW;
        bool arrived = mbar_wait_bounded(&t.bar[s], (uint32_t)((g / kRingStages) & 1));
        if constexpr (J == kTileStages - 1) arrived = arrived && mbar_wait_bounded(&t.bar[kRingStages], t.ppar);
        if (!arrived) *reinterpret_cast<volatile int*>(t.abort) = 1;
        if (arrived) {
            if constexpr (J < kFgStages) {
                const pop* b = reinterpret_cast<const pop*>(buf);
                const int cell = (ty + kTileHaloY) * G::BWF + tx + G::PX;
                if constexpr (J == 0) {
                    const V2<R> v = rest_pair<Cfg>(ld_pair_sh<Cfg>(b + 2 * cell), A.hs);
                    store_group<0, Cfg, true>(V4<R>{v.x, v.y, R(0), R(0)}, S, Tm, Nm, Na);
                } else {
                    auto ld = [&](int a, int d) { return ld_quad_sh<Cfg>(b + 4 * (cell + d * (a == 0 ? 1 : G::BWF))); };
                    store_group<J, Cfg, true>(stream_group<J, false, Cfg>(ld, A.k, A.hs), S, Tm, Nm, Na);
                }
            } else {
                const float* b = reinterpret_cast<const float*>(buf);
                const int cell = (ty + kTileHaloY) * G::BWH + tx + G::PXH;
                if constexpr (J < kTileStages - 1) {
                    constexpr int M0 = 2 * (J - kFgStages);  // pairs M0, M0 + 1
#pragma unroll
                    for (int d = 0; d < 2; ++d) {
                        // the pair 2m, 2m + 1 (m = M0 + d) hops the same way
                        constexpr int K0 = 2 * M0;
                        const int K = K0 + 2 * d;
                        const int src = d * G::H_PLANE + cell - hop13(K, 1) * G::BWH - hop13(K, 0);
                        const float2 hv = *reinterpret_cast<const float2*>(b + 2 * src);
                        put_pair<R, Cfg::kVecSlots>(S.h(K), S.h(K + 1), (R)hv.x, (R)hv.y);
                        if (d == 0) {
                            acc_h<K0>((R)hv.x, dEp, bn, rho);
                            acc_h<K0 + 1>((R)hv.y, dEp, bn, rho);
                        } else {
                            acc_h<K0 + 2>((R)hv.x, dEp, bn, rho);
                            acc_h<K0 + 3>((R)hv.y, dEp, bn, rho);
                        }
                    }
                } else {
                    const R hv = (R)b[cell];
                    *S.h(24) = hv;
                    rho += hv;
                }
            }
        }
        __syncthreads();  // every thread is done with buffer s (and has seen any abort)
        if (*reinterpret_cast<volatile int*>(t.abort)) {
            // let the copies already issued land before the block gives up its
            // shared memory (each wait again bounded)
            if (tid == 0) {
                const int last = t.has_next ? g + kRingStages - 1 : min(g + kRingStages - 1, t.gbase + kTileStages - 1);
                for (int i = g; i <= last; ++i) mbar_wait_bounded(&t.bar[i % kRingStages], (uint32_t)((i / kRingStages) & 1));
                mbar_wait_bounded(&t.bar[kRingStages], t.ppar);
            }
            return false;
        }
        if (tid == 0) {
            // refill slot s: a later stage of this tile, or one of the next tile's first stages
            constexpr int jn = J + kRingStages;
            if (jn < kTileStages)
                tile_issue<Cfg>(t, g + kRingStages, t.x0, t.y0, jn);
            else if (t.has_next)
                tile_issue<Cfg>(t, g + kRingStages, t.nx0, t.ny0, jn - kTileStages);
        }
        return TileStages<J + 1, Cfg>::run(t, A, tid, S, Tm, Nm, Na, dEp, bn, rho);
    }
};
template <class Cfg>
struct TileStages<kTileStages, Cfg> {
    using R = typename Cfg::real;
    static __device__ __forceinline__ bool run(const TileCtx<Cfg>&, const StepArgs<Cfg>&, int, const CfgSlots<Cfg>&,
                                               R (&)[10], R&, R (&)[3], R (&)[3], R (&)[3], R&)
    {
        return true;
    }
};

// One cell update (x, y, z) of one run; `tid` is the thread's index in its
// block of kStepThreads threads (its rows of the shared-memory buffers). Threads of
// cells outside the grid return at once, except in the learned-seed variant,
// whose warp-wide MMA needs all 32 lanes: there they work on a clamped cell
// and store nothing.
// TILE: a cell of an interior tile of the TMA tile path (2-D, periodic,
// every cell active): its inputs come from the block's ring and primitive
// buffers (tc), its outputs go to the block's shared-memory output tiles.
template <class Cfg, bool IS3D, int SEED, bool OPEN, bool TILE = false, int NTH = kStepThreads>
__device__ __forceinline__ void step_cell(const StepArgs<Cfg>& A, int x, int y, const int z, const int tid,
                                          unsigned char* smem_raw, const TileCtx<Cfg>* tc = nullptr)
{
    constexpr int nth = NTH;  // threads of the block: a compile-time stride of the shared-memory slots
    using R = typename Cfg::real;
    const CfgSlots<Cfg> S{reinterpret_cast<R*>(smem_raw), nth, tid};
    const bool active = x < A.nx && y < A.ny;
    if constexpr (SEED != SEED_MLP) {
        if (!active) return;  // no block-wide barrier follows
    } else {
        // the warp-wide tensor-core MMA of the learned seed needs every lane:
        // out-of-range lanes work on a clamped cell and store nothing
        x = x < A.nx ? x : A.nx - 1;
        y = y < A.ny ? y : A.ny - 1;
    }
    // Open faces (Sec. IV: the boundary cells copy their interior neighbour): a
    // cell on an open face takes the update of the cell clamped into
    // [1, n - 2] along every open axis, so the copy happens in this pass and
    // lands in the ordinary coalesced stores. `c` is the cell whose update is
    // computed (loads), `co` the cell written.
    // The open-face code is compiled into the variant for runs with an open or
    // driven face, and (as a run-time branch) into the learned-seed variant,
    // whose registers are allocated better with it (15 % in a same-box A/B).
    constexpr bool kOpenCode = OPEN || SEED == SEED_MLP;
    int xs = x, ys = y, zs = z;
    if (kOpenCode && A.open_mask) {
        if ((A.open_mask & 1) && A.nx >= 3) xs = min(max(x, 1), A.nx - 2);
        if ((A.open_mask & 2) && A.ny >= 3) ys = min(max(y, 1), A.ny - 2);
        if ((A.open_mask & 4) && A.nz >= 3) zs = min(max(z, 1), A.nz - 2);
    }
    const Off o = make_off<IS3D>(xs, ys, zs, A.nx, A.ny, A.nz, A.periodic);
    const int64_t c = xs + (int64_t)A.nx * (ys + (int64_t)A.ny * zs);
    // offset of the written cell from the computed one (0 away from open faces)
    const int dco = kOpenCode ? (x - xs) + A.nx * ((y - ys) + A.ny * (z - zs)) : 0;
    const Phys<R>& k = A.k;

    // 1. streaming of f and g (with their moments) and of h (with its moments)
    R Tm[10] = {R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0)};
    R Nm = R(0), Na[3] = {R(0), R(0), R(0)};
    R dEp[3] = {R(0), R(0), R(0)}, bn[3] = {R(0), R(0), R(0)}, rho = R(0);
    if constexpr (TILE) {
        if (!TileStages<0, Cfg>::run(*tc, A, tid, S, Tm, Nm, Na, dEp, bn, rho)) return;
    } else {
        StreamAll<0, IS3D, Cfg>::run(A, o, c, S, Tm, Nm, Na);
        PullH<0, IS3D, Cfg>::run(A, o, c, S, dEp, bn, rho);
        const R h24 = (R)A.hin[h_elem(24, c, A.stride)];
        *S.h(24) = h24;
        rho += h24;
    }
    // previous primitives (the tile path's box has arrived with the last stage)
    auto ldp = [&](int P) -> R {
        if constexpr (TILE)
            return (R)tc->pbuf[4 * ((P >> 2) * nth + tid) + (P & 3)];
        else
            return (R)A.pin[prim_elem(P, c, A.stride)];
    };

    // previous primitives used by the recovery
    Prim<R> old;
    {
        R pv[NPRIM];
        if constexpr (TILE) {
#pragma unroll
            for (int q = 0; q < kPrimVecs; ++q) {
                const float4 a = reinterpret_cast<const float4*>(tc->pbuf)[q * nth + tid];
                pv[4 * q] = (R)a.x, pv[4 * q + 1] = (R)a.y, pv[4 * q + 2] = (R)a.z, pv[4 * q + 3] = (R)a.w;
            }
        } else {
            ld_prims<Cfg>(A.pin + prim_elem(0, c, A.stride), A.stride, pv);
        }
        old.n = pv[P_N];
        old.eps = pv[P_EPS];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            old.u[a] = pv[P_U + a];
            old.E[a] = pv[P_E + a];
            old.B[a] = pv[P_B + a];
        }
    }
    old.rho = R(0);
    if constexpr (kOpenCode) {
        if (zs < A.force_layers && (A.vmax2 <= 0.0 || *A.umax_in < A.vmax2)) {
            const double* fd = A.fdrive + 2 * (xs + (int64_t)A.nx * ys);
            const R F[3] = {(R)fd[0], (R)fd[1], R(0)};
            const R w = (F[0] * old.u[0] + F[1] * old.u[1]) * A.force_dt;
            AddForce<0, Cfg>::run(S, F, A.force_cdt, w);
            Tm[0] += w;
#pragma unroll
            for (int a = 0; a < 3; ++a) Tm[a + 1] += R(10) * A.force_cdt * F[a];
        }
    }

    // 2. moments (reference state added back): rest state (eps_r, p_r) and the
    // reference EM terms k.Tem
    const R qq = R(kQ), q2 = R(kQ2);
    R T[4][4];
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
    const R dN0 = Nm;  // N^0 - n_r
    R Ep[3], Bn[3], dB[3];
    const R es = R(kSqrt2 / 2.0) * k.c;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        dEp[a] *= es;
        dB[a] = bn[a];
        Ep[a] = k.Er[a] + dEp[a];
        Bn[a] = k.Br[a] + dB[a];
    }

    // 3. recovery, seeded with the previous velocity, the learned guess or zero
    R seed[3];
    float feat[MLP_IN];
    // the training-data dump exists only in the cold-seed and learned-seed
    // variants (the seed does not change the converged result)
    constexpr bool kCanDump = SEED != SEED_PREV;
    const bool want_feat = SEED == SEED_MLP || (kCanDump && A.dump != nullptr);
    if (want_feat) {
        const R T0a[3] = {T[0][1], T[0][2], T[0][3]};
        const R Tab[6] = {T[1][1], T[2][2], T[3][3], T[1][2], T[1][3], T[2][3]};
        const R Nq[3] = {qq * Na[0], qq * Na[1], qq * Na[2]};
        mlp_features(k.eps_r + T[0][0], T0a, Tab, k.n_r + dN0, Nq, old.E, old.B, feat);
    }
    if constexpr (SEED == SEED_MLP) {
        __nv_bfloat16* act =
            reinterpret_cast<__nv_bfloat16*>(smem_raw + (size_t)kStepSlots * sizeof(R) * nth);
        float* out_f = reinterpret_cast<float*>(smem_raw + (size_t)kStepSlots * sizeof(R) * nth +
                                                (size_t)MLP_ACT_BYTES_PER_CELL * nth);
        __nv_bfloat16* row = act + tid * MLP_HS;
#pragma unroll
        for (int j = 0; j < 32; j += 2)
            *reinterpret_cast<__nv_bfloat162*>(row + j) =
                __floats2bfloat162_rn(j < MLP_IN ? feat[j] : 0.0f, j + 1 < MLP_IN ? feat[j + 1] : 0.0f);
        __syncwarp();
        mlp_forward_warp(act, A.mlp, out_f);
        R sb[3] = {(R)out_f[tid * 8], (R)out_f[tid * 8 + 1], (R)out_f[tid * 8 + 2]};
        const R sb2 = sb[0] * sb[0] + sb[1] * sb[1] + sb[2] * sb[2];
        const R lim = R(0.9);  // keep the guess well inside the light cone
        const R scale = sb2 > lim * lim ? lim / sqrt(sb2) : R(1);
        for (int a = 0; a < 3; ++a) seed[a] = sb[a] * scale;
    } else if constexpr (SEED == SEED_COLD) {
        seed[0] = seed[1] = seed[2] = R(0);
    } else {
        for (int a = 0; a < 3; ++a) seed[a] = old.u[a] * k.inv_c;
    }
    // Self-consistent recovery (reading R24 of the coupling subsection): the
    // previous step's E starts a relaxed fixed-point iteration in which the
    // tensor T - eps0 F F is formed with the E that Ohm's law gives for the
    // recovered velocity and the streamed B, until that E reproduces itself;
    // the collision below then conserves T^{mu nu}, and the EM momentum keeps
    // its inertia. FLAG_ONE_PASS_RECOVERY: one solve with the previous E, B.
    // the charge of Ohm's convection current: the moment rho_c = sum h (Eq.
    // Cal_rhoc), or with FLAG_GAUSS_CHARGE eps0 div E of the previous step's
    // E by central differences (Eq. Gauss_E), which carries no grid-scale
    // mode for a flow to amplify
    R rho_j = rho;
    if (!TILE && (A.flags & FLAG_GAUSS_CHARGE)) {
        R div = R(0);
        if (A.nx > 1)
            div += (R)A.pin[prim_elem(P_E, c + o.x[3], A.stride)] - (R)A.pin[prim_elem(P_E, c + o.x[1], A.stride)];
        if (A.ny > 1)
            div += (R)A.pin[prim_elem(P_E + 1, c + o.y[3], A.stride)] -
                   (R)A.pin[prim_elem(P_E + 1, c + o.y[1], A.stride)];
        if (IS3D && A.nz > 1)
            div += (R)A.pin[prim_elem(P_E + 2, c + o.z[3], A.stride)] -
                   (R)A.pin[prim_elem(P_E + 2, c + o.z[1], A.stride)];
        rho_j = k.eps0 * div / (R(2) * k.dx);
    }
    const bool one_pass = (A.flags & FLAG_ONE_PASS_RECOVERY) != 0;
    const bool shifted = (A.flags & FLAG_UNSHIFTED_POWER) == 0;
    R Ec[3], Bc[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        Ec[a] = old.E[a];
        Bc[a] = one_pass ? old.B[a] : Bn[a];
    }
    R p_shift = k.gm1 * (old.eps - old.n * k.c2);
    const R tol_o = k.tol * (sizeof(R) == 8 ? R(100) : R(10));
    const R Bn2 = Bn[0] * Bn[0] + Bn[1] * Bn[1] + Bn[2] * Bn[2];
    R beta[3] = {seed[0], seed[1], seed[2]}, lambda, s_old, b2 = R(0), g2 = R(1), g = R(1), ig = R(1);
    LandauB<R> LB;
    landau_b(T, Bc, k, LB);
    Prim<R> nw;
    R J[3], n_dev, eps_dev;
    int it = 0;
    bool ok = true;
    R d_prev = R(1e30);
#pragma unroll 1
    for (int outer = 0;; ++outer) {
        const R sd[3] = {beta[0], beta[1], beta[2]};
        // each solve starts from the latest velocity and may stop after one
        // iteration (the last solve's own test then confirms the eigenvector);
        // a single solve with the previous fields iterates at least twice
        const int i1 =
            outer < 64 ? landau(LB, Ec, p_shift, k, beta, lambda, s_old, sd, shifted, one_pass ? 2 : 1) : -1;
        if (i1 <= 0) {  // the eigen-solve failed, or the fields did not settle
            ok = false;
            break;
        }
        it += i1;
        b2 = beta[0] * beta[0] + beta[1] * beta[1] + beta[2] * beta[2];
        g = rsqrt_r(R(1) - b2);
        g2 = g * g;
        ig = (R(1) - b2) * g;
#pragma unroll
        for (int a = 0; a < 3; ++a) nw.u[a] = k.c * beta[a];
        ohm_solve(Ep, nw.u, Bn, rho_j, g, ig, k, nw.E);
        if (one_pass) break;
        R d = R(0), e2 = R(0), dB = R(0);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            d += (nw.E[a] - Ec[a]) * (nw.E[a] - Ec[a]);
            e2 += nw.E[a] * nw.E[a];
            dB += (nw.E[a] - Ec[a]) * Bn[a];
        }
        // E is judged against the motional field scale |E| + c |B| |beta|: a
        // mismatch below it moves the fluid part of T by less than the outer
        // tolerance times the EM momentum it could carry. |beta| is floored at
        // the resolution of E itself: float32 sums of the Maxwell populations
        // carry ~1e-7 c |B| of rounding, which no iteration removes (1e-6 in
        // float64). A residual that stops decreasing near the bound is at its
        // round-off floor (the inner solve leaves noise ~ tol).
        constexpr R beta_floor2 = sizeof(R) == 8 ? R(1e-12) : R(1e-4);
        const R bound = tol_o * tol_o * (e2 + k.c2 * Bn2 * (b2 + beta_floor2));
        if (d <= bound || (d >= d_prev && d <= R(1e6) * bound)) break;
        d_prev = d;
        // Relaxed update: the part of E across B feeds back through the EM
        // momentum eps0 E x B with gain -r, r = B^2 k/(1+k) / (w gamma^2) (the
        // EM-to-fluid inertia ratio), and takes 1/(1+r) of the step; the part
        // along B does not feed back and takes all of it. Only the rate of
        // convergence depends on these factors.
        const R ed = lambda - s_old;  // eps - eps_r
        const R W = (k.eps_r + k.p_r + ed + k.gm1 * ed) * g2;
        const R kk = k.half_dt_c2 * k.sigma * g;
        const R q = kk * rcp_approx((R(1) + kk) * W);  // r / B^2
        const R th = rcp_approx(R(1) + Bn2 * q);
        const R par = th * q * dB;                      // (1 - th) (dE.B) / B^2
#pragma unroll
        for (int a = 0; a < 3; ++a) Ec[a] += th * (nw.E[a] - Ec[a]) + par * Bn[a];
        const R nd = (dN0 - k.n_r * (g2 * b2 * rcp_approx(g + R(1)))) * ig;  // n - n_r
        p_shift = k.p_r + k.gm1 * (ed - nd * k.c2);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) J[a] = (Ep[a] - nw.E[a]) * k.inv_half_dt_c2;
    if (ok) {
        eps_dev = lambda - s_old;
        // n = N^0 / U^0: n - n_r = (dN0 - n_r (g - 1)) / g, g - 1 = g^2 b^2 / (g + 1)
        n_dev = (dN0 - k.n_r * (g2 * b2 / (g + R(1)))) / g;
        nw.eps = k.eps_r + eps_dev;
        nw.n = k.n_r + n_dev;
#pragma unroll
        for (int a = 0; a < 3; ++a) nw.B[a] = Bn[a];
        nw.rho = rho;
    } else {
        // keep the previous primitives (the failure is counted)
        nw = old;
        nw.rho = ldp(P_RHO);
        n_dev = nw.n - k.n_r;
        eps_dev = nw.eps - k.eps_r;
#pragma unroll
        for (int a = 0; a < 3; ++a) dB[a] = nw.B[a] - k.Br[a];
        ohm_current(nw.E, nw.u, nw.B, nw.rho, k, J);
    }

    if (!active) return;  // (only reached by clamped lanes of the learned-seed variant)
    if (kCanDump && A.dump != nullptr && ok) {
        float* d = A.dump + (c + dco) * (MLP_IN + MLP_OUT);
        for (int j = 0; j < MLP_IN; ++j) d[j] = feat[j];
        for (int a = 0; a < 3; ++a) d[MLP_IN + a] = (float)beta[a];
        d[MLP_IN + 3] = (float)((nw.eps) / (k.eps_r + T[0][0]) - R(1));
    }
    bool relax_eq = false;
    if constexpr (kOpenCode) {
        if (A.umax_out)
            warp_max_into((double)(nw.u[0] * nw.u[0] + nw.u[1] * nw.u[1] + nw.u[2] * nw.u[2]), A.umax_out);
        if (A.relax_in) {
            // relaxed initialisation (reading R27): track E of every written
            // cell, then hold the cell at the initial n, p, u, B before the
            // collision (the boundary pass follows)
            const int64_t NN = (int64_t)A.nx * A.ny * A.nz, cw = c + dco;
            double d2 = 0.0, e2 = 0.0;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const double E = (double)nw.E[a];
                const double em2 = A.relax_e[(3 + a) * NN + cw];
                d2 += (E - em2) * (E - em2);
                e2 += E * E;
                A.relax_e[(3 + a) * NN + cw] = A.relax_e[a * NN + cw];
                A.relax_e[a * NN + cw] = E;
            }
            warp_max_into(d2, A.relax_red);
            warp_max_into(e2, A.relax_red + 1);
            {  // (an open-face cell is held at the fields of its interior source, whose update it is)
                const double* in = A.relax_in;
                const double n0 = in[c], p0 = in[NN + c];
                nw.n = (R)n0;
                nw.eps = (R)(n0 * (double)k.c2 + p0 / (double)k.gm1);
                n_dev = (R)(n0 - (double)k.n_r);
                eps_dev = (R)((n0 - (double)k.n_r) * (double)k.c2 + (p0 - (double)k.p_r) / (double)k.gm1);
                R dBs[3];
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    nw.u[a] = (R)in[(2 + a) * NN + c];
                    const double B0 = in[(5 + a) * NN + c];
                    dBs[a] = (R)(B0 - (double)nw.B[a]);
                    nw.B[a] = (R)B0;
                    dB[a] = (R)(B0 - (double)k.Br[a]);
                }
                ShiftHB<0, Cfg>::run(S, dBs);
                ohm_current(nw.E, nw.u, nw.B, nw.rho, k, J);
                relax_eq = true;
            }
        }
    }

    // 4. collisions at the new time level and stores
    R dE[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) dE[a] = nw.E[a] - k.Er[a];
    EqCell<R> q;
    eq_cell(nw, n_dev, eps_dev, dE, dB, k, q);
    if (kOpenCode && relax_eq) SetEqFG<0, Cfg>::run(S, q);
    CollideFG<0, Cfg>::run(A, c + dco, S, q);
    const bool em_coll = (A.flags & FLAG_NO_EM_COLLISION) == 0;
    // h_c - h_ref = 2 h^eq(E - Er, B - Br, J) - (h - h_ref)  (Eq. Maxwell-eq is linear)
    const int64_t co = c + dco;
    CollideH<0, Cfg>::run(A, co, S, dE, dB, J, em_coll);
    const R h24o = em_coll ? R(2) * nw.rho - *S.h(24) : *S.h(24);
    A.hout[h_elem(24, co, A.stride)] = (typename Cfg::hpop)h24o;
    {
        R pv[NPRIM];
        pv[P_N] = nw.n;
        pv[P_EPS] = nw.eps;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            pv[P_U + a] = nw.u[a];
            pv[P_E + a] = nw.E[a];
            pv[P_B + a] = nw.B[a];
        }
        pv[P_RHO] = nw.rho;
        if constexpr (TILE) {
#pragma unroll
            for (int q = 0; q < kPrimVecs; ++q)
                reinterpret_cast<float4*>(tc->pbuf)[q * nth + tid] =
                    make_float4((float)pv[4 * q], (float)pv[4 * q + 1], (float)pv[4 * q + 2], (float)pv[4 * q + 3]);
        } else {
            st_prims<Cfg>(A.pout + prim_elem(0, co, A.stride), A.stride, pv);
        }
    }

    // recovery counters, aggregated per warp
    const unsigned mask = __activemask();
    const unsigned fail = __reduce_add_sync(mask, ok ? 0u : 1u);
    const unsigned isum = __reduce_add_sync(mask, ok ? (unsigned)it : 0u);
    const unsigned imax = __reduce_max_sync(mask, ok ? (unsigned)it : 0u);
    const bool leader = (tid & 31) == __ffs(mask) - 1;
    const unsigned slot = (blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z)) % kStatSlots;
    unsigned long long* st = A.stats + (size_t)slot * kNumStats;
    if (leader) {
        if (fail) atomicAdd(&st[0], (unsigned long long)fail);
        atomicAdd(&st[1], (unsigned long long)isum);
        atomicMax(&st[2], (unsigned long long)imax);
    }
    // iteration histogram over the warp's own range of counts (usually 1-2 bins)
    const unsigned ib = ok ? (unsigned)(it < kHistBins ? it : kHistBins) : 0u;
    const unsigned bmin = __reduce_min_sync(mask, ok ? ib : 0xffffffffu);
    const unsigned bmax = __reduce_max_sync(mask, ib);
    for (unsigned b = bmin; b <= bmax; ++b) {
        const unsigned cnt = __popc(__ballot_sync(mask, ib == b));
        if (leader && cnt) atomicAdd(&st[2 + b], (unsigned long long)cnt);
    }
}

// one run: a 2-D grid of blocks over (x, y) and z
template <class Cfg, bool IS3D, int SEED, bool OPEN>
__global__ void __launch_bounds__(kStepThreads, StepMinBlocks<Cfg, SEED, IS3D>::value)
    step_kernel(const StepArgs<Cfg> A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    step_cell<Cfg, IS3D, SEED, OPEN>(A, blockIdx.x * blockDim.x + threadIdx.x,
                                     blockIdx.y * blockDim.y + threadIdx.y, blockIdx.z,
                                     threadIdx.x + threadIdx.y * blockDim.x, smem_raw);
}

template <class Cfg, int NTH = kStepThreads>
__host__ __device__ constexpr size_t step_cell_smem(int seed)
{
    return seed == SEED_MLP ? (size_t)kStepSlots * sizeof(typename Cfg::real) * NTH +
                                  (size_t)(MLP_ACT_BYTES_PER_CELL + 8 * sizeof(float)) * NTH
                            : (size_t)kStepSlots * sizeof(typename Cfg::real) * NTH;
}

// the tile path applies to storage formats whose h and primitives are float
template <class Cfg>
constexpr bool kTileCapable = sizeof(typename Cfg::hpop) == 4 && sizeof(typename Cfg::prim) == 4 &&
                              sizeof(typename Cfg::real) == 4;

__host__ __device__ constexpr size_t align128(size_t b) { return (b + 127) / 128 * 128; }

// shared memory of the tile kernel: the per-cell slots (and learned-seed
// buffers), the ring, the primitive tile, barriers
template <class Cfg>
__host__ __device__ constexpr size_t tile_smem_bytes(int seed)
{
    return align128(step_cell_smem<Cfg, kTileThreads>(seed)) + (size_t)kRingStages * TileGeo<Cfg>::STAGE_BYTES +
           TileGeo<Cfg>::PRIM_BYTES + 128;
}

// resident tile blocks per SM targeted: as many threads per SM as the per-cell kernel
template <class Cfg, int SEED>
struct TileMinBlocks {
    static constexpr int v = StepMinBlocks<Cfg, SEED>::value * kStepThreads / kTileThreads;
    static constexpr int value = v > 0 ? v : 1;
};

// The interior tiles of one run of a 2-D periodic grid (tiles of kTileW x
// kTileH cells whose input boxes lie inside the grid), block (bx, by) on tile
// (bx + tx0, by + ty0), by TMA copies through shared memory; the edge tiles
// are a separate per-cell launch.
template <class Cfg, int SEED>
__global__ void __launch_bounds__(kTileThreads, TileMinBlocks<Cfg, SEED>::value)
    step_tile_kernel(const __grid_constant__ StepArgs<Cfg> A, const __grid_constant__ TileMaps M,
                     const __grid_constant__ TileRange tr)
{
    using G = TileGeo<Cfg>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int tid = threadIdx.x;
    const int ntiles = tr.nx * tr.ny;
    size_t off = align128(step_cell_smem<Cfg, kTileThreads>(SEED));
    TileCtx<Cfg> t;
    t.ring = smem_raw + off;
    off += (size_t)kRingStages * G::STAGE_BYTES;
    t.pbuf = reinterpret_cast<float*>(smem_raw + off);
    off += G::PRIM_BYTES;
    t.bar = reinterpret_cast<uint64_t*>(smem_raw + off);
    t.abort = reinterpret_cast<int*>(t.bar + kRingStages + 1);
    t.M = &M;
    if (tid == 0) {
        for (int i = 0; i <= kRingStages; ++i) mbar_init(&t.bar[i], 1u);
        *t.abort = 0;
        mbar_init_fence();
    }
    __syncthreads();
    auto coords = [&](int i, int& x0, int& y0) {
        x0 = (tr.x0 + i % tr.nx) * kTileW;
        y0 = (tr.y0 + i / tr.nx) * kTileH;
    };
    int k = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++k) {
        coords(tile, t.x0, t.y0);
        t.has_next = tile + (int)gridDim.x < ntiles;
        if (t.has_next) coords(tile + gridDim.x, t.nx0, t.ny0);
        t.gbase = kTileStages * k;
        t.ppar = (uint32_t)(k & 1);
        if (tid == 0) {
            // the previous tile's primitive copy-out has read the primitive
            // tile; this tile's first stages are already in flight (issued as
            // the previous tile's last stages were consumed)
            if (k > 0) tma_store_wait_read();
            mbar_arrive_expect_tx(&t.bar[kRingStages], G::PRIM_BYTES);
            tma_load_3d(t.pbuf, &M.p_in, 4 * t.x0, t.y0, 0, &t.bar[kRingStages]);
            if (k == 0)
                for (int j = 0; j < kRingStages; ++j) tile_issue<Cfg>(t, j, t.x0, t.y0, j);
        }
        __syncthreads();
        step_cell<Cfg, false, SEED, false, true, kTileThreads>(A, t.x0 + tid % kTileW, t.y0 + tid / kTileW, 0, tid,
                                                              smem_raw, &t);
        if (*reinterpret_cast<volatile int*>(t.abort)) {  // every thread returned from the same stage
            if (tid == 0) atomicOr(A.status, STATUS_TMA_TIMEOUT);
            return;
        }
        fence_proxy_async_smem();  // the primitive tile written by every thread, before the copy reads it
        __syncthreads();
        if (tid == 0) {
            tma_store_3d(&M.p_out, t.pbuf, 4 * t.x0, t.y0, 0);
            tma_store_commit();
        }
    }
    if (tid == 0) tma_store_wait_read();  // the block's shared memory stays until the stores have read it
}

// the batched kernel keeps the arguments of its current run in shared memory,
// after the per-cell buffers; in device memory they are stored with this
// (16-byte) stride
template <class Cfg>
__host__ __device__ constexpr size_t batch_args_bytes()
{
    return (sizeof(StepArgs<Cfg>) + 15) / 16 * 16;
}

// Many runs in one launch: a list of tiles (run, x0, y0, z) of bx x
// (kStepThreads / bx) cells each, walked by the blocks with stride gridDim.x
// (persistent when the grid is one wave of resident blocks). A block copies
// the arguments of a tile's run from device memory into shared memory when
// the run changes from its previous tile.
template <class Cfg, bool IS3D, int SEED, bool OPEN>
__global__ void __launch_bounds__(kStepThreads, StepMinBlocks<Cfg, SEED, IS3D>::value)
    step_batch_kernel(const unsigned char* __restrict__ args, const int4* __restrict__ tiles, int ntiles, int bx)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    StepArgs<Cfg>* sA = reinterpret_cast<StepArgs<Cfg>*>(smem_raw + step_cell_smem<Cfg>(SEED));
    const int tid = threadIdx.x;
    const int tx = tid % bx, ty = tid / bx;
    int run = -1;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int4 td = __ldg(tiles + t);  // block-uniform
        if (td.x != run) {
            __syncthreads();  // the previous tile's readers are done
            const int4* src = reinterpret_cast<const int4*>(args + (size_t)td.x * batch_args_bytes<Cfg>());
            int4* dst = reinterpret_cast<int4*>(sA);
            for (int i = tid; i < (int)(batch_args_bytes<Cfg>() / 16); i += kStepThreads) dst[i] = __ldg(src + i);
            __syncthreads();
            run = td.x;
        }
        __syncwarp();  // every lane starts a tile together (the learned seed's MMA)
        step_cell<Cfg, IS3D, SEED, OPEN>(*sA, td.y + tx, td.z + ty, td.w, tid, smem_raw);
    }
}

// ---------------------------------------------------------------------------
// Persistent multi-step launch: one cooperative grid (every block resident)
// walks the tile list of all runs for `nsteps` steps, with a grid-wide
// barrier between steps (step t + 1 of a cell reads its neighbours' step t).
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int* p)
{
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Every block arrives on *counter and waits until it reaches `target`; the
// wait gives up after wait_ns of global time (status bit, false for every
// thread of the block). All blocks of the grid must be resident (cooperative
// launch) for the barrier to complete.
__device__ __forceinline__ bool grid_barrier(unsigned int* counter, unsigned int target, int* status,
                                             unsigned long long wait_ns)
{
    __syncthreads();
    int ok = 1;
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(counter, 1u);
        const unsigned long long t0 = global_ns();
        while (ld_acquire_u32(counter) < target) {
            if (global_ns() - t0 > wait_ns) {
                atomicOr(status, STATUS_BARRIER_TIMEOUT);
                ok = 0;
                break;
            }
            __nanosleep(100);
        }
        __threadfence();
    }
    return __syncthreads_and(ok) != 0;
}

template <class Cfg, bool IS3D, int SEED, bool OPEN>
__global__ void __launch_bounds__(kStepThreads, StepMinBlocks<Cfg, SEED, IS3D>::value)
    step_persistent_kernel(const unsigned char* __restrict__ args, size_t parity_bytes, int in0,
                           const int4* __restrict__ tiles, int ntiles, int bx, int nsteps, unsigned int* counter,
                           int* status, unsigned long long wait_ns)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    StepArgs<Cfg>* sA = reinterpret_cast<StepArgs<Cfg>*>(smem_raw + step_cell_smem<Cfg>(SEED));
    const int tid = threadIdx.x;
    const int tx = tid % bx, ty = tid / bx;
    for (int t = 0; t < nsteps; ++t) {
        // argument records of the runs for this step's input buffer
        const unsigned char* a = args + (size_t)((in0 + t) & 1) * parity_bytes;
        int run = -1;
        for (int i = blockIdx.x; i < ntiles; i += gridDim.x) {
            const int4 td = __ldg(tiles + i);
            if (td.x != run) {
                __syncthreads();
                const int4* src = reinterpret_cast<const int4*>(a + (size_t)td.x * batch_args_bytes<Cfg>());
                int4* dst = reinterpret_cast<int4*>(sA);
                for (int j = tid; j < (int)(batch_args_bytes<Cfg>() / 16); j += kStepThreads) dst[j] = __ldg(src + j);
                __syncthreads();
                run = td.x;
            }
            __syncwarp();
            step_cell<Cfg, IS3D, SEED, OPEN>(*sA, td.y + tx, td.z + ty, td.w, tid, smem_raw);
        }
        if (t + 1 < nsteps && !grid_barrier(counter, (unsigned int)(t + 1) * gridDim.x, status, wait_ns)) return;
        __syncthreads();  // the block's args copy is rewritten by the next step's first tile
    }
}

template <class Cfg>
size_t step_smem_bytes(int seed)
{
    return step_cell_smem<Cfg>(seed);
}

template <class Cfg>
size_t batch_smem_bytes(int seed)
{
    return step_cell_smem<Cfg>(seed) + batch_args_bytes<Cfg>();
}

// Calls f.template run<IS3D, SEED, OPEN>() for the kernel variant of a run:
// 2-D / 3-D, recovery seed, periodic only / with an open or driven face.
template <class F>
cudaError_t dispatch_variant(bool is3d, int seed, bool open, F&& f)
{
#define LB_VARIANT(D, S, O) \
    if (is3d == D && seed == S && open == O) return f.template run<D, S, O>();
    LB_VARIANT(false, SEED_PREV, false)
    LB_VARIANT(false, SEED_PREV, true)
    LB_VARIANT(false, SEED_COLD, false)
    LB_VARIANT(false, SEED_COLD, true)
    LB_VARIANT(false, SEED_MLP, false)
    LB_VARIANT(false, SEED_MLP, true)
    LB_VARIANT(true, SEED_PREV, false)
    LB_VARIANT(true, SEED_PREV, true)
    LB_VARIANT(true, SEED_COLD, false)
    LB_VARIANT(true, SEED_COLD, true)
    LB_VARIANT(true, SEED_MLP, false)
    LB_VARIANT(true, SEED_MLP, true)
#undef LB_VARIANT
    return cudaErrorInvalidValue;
}

template <class Cfg>
struct SetSmemAttr {
    template <bool D, int S, bool O>
    cudaError_t run()
    {
        const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
        cudaError_t e = cudaFuncSetAttribute(step_kernel<Cfg, D, S, O>, a, (int)step_smem_bytes<Cfg>(S));
        if (e == cudaSuccess) e = cudaFuncSetAttribute(step_batch_kernel<Cfg, D, S, O>, a, (int)batch_smem_bytes<Cfg>(S));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(step_persistent_kernel<Cfg, D, S, O>, a, (int)batch_smem_bytes<Cfg>(S));
        return e;
    }
};

template <class Cfg>
cudaError_t configure_step_kernels()
{
    static bool configured = false;  // one attribute call per instantiation
    if (configured) return cudaSuccess;
    for (int d = 0; d < 2; ++d)
        for (int seed = 0; seed < 3; ++seed)
            for (int o = 0; o < 2; ++o) {
                const cudaError_t e = dispatch_variant(d == 1, seed, o == 1, SetSmemAttr<Cfg>{});
                if (e != cudaSuccess) return e;
            }
    if constexpr (kTileCapable<Cfg>) {
        const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
        cudaError_t e = cudaFuncSetAttribute(step_tile_kernel<Cfg, SEED_PREV>, a, (int)tile_smem_bytes<Cfg>(SEED_PREV));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(step_tile_kernel<Cfg, SEED_COLD>, a, (int)tile_smem_bytes<Cfg>(SEED_COLD));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(step_tile_kernel<Cfg, SEED_MLP>, a, (int)tile_smem_bytes<Cfg>(SEED_MLP));
        if (e != cudaSuccess) return e;
    }
    configured = true;
    return cudaSuccess;
}

// whether a run's step takes the TMA tile kernel (given its tensor maps)
template <class Cfg>
bool tile_path(const StepArgs<Cfg>& A, const TileMaps* maps)
{
    return kTileCapable<Cfg> && maps != nullptr && A.nz == 1 && A.open_mask == 0 && (A.flags & FLAG_TMA_TILES) != 0 &&
           (A.flags & FLAG_GAUSS_CHARGE) == 0;
}

template <class Cfg>
struct BatchOccupancy {
    int* nb;
    template <bool D, int S, bool O>
    cudaError_t run()
    {
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(nb, step_batch_kernel<Cfg, D, S, O>, kStepThreads,
                                                             batch_smem_bytes<Cfg>(S));
    }
};

// resident blocks per SM of the batched kernel (for a one-wave persistent grid)
template <class Cfg>
int batch_blocks_per_sm(bool is3d, int seed, bool open)
{
    if (configure_step_kernels<Cfg>() != cudaSuccess) return 0;
    int nb = 0;
    return dispatch_variant(is3d, seed, open, BatchOccupancy<Cfg>{&nb}) == cudaSuccess ? nb : 0;
}

template <class Cfg>
struct LaunchBatch {
    const unsigned char* args;
    const int4* tiles;
    int ntiles, bx, grid;
    cudaStream_t stream;
    template <bool D, int S, bool O>
    cudaError_t run()
    {
        step_batch_kernel<Cfg, D, S, O><<<grid, kStepThreads, batch_smem_bytes<Cfg>(S), stream>>>(args, tiles, ntiles, bx);
        return cudaGetLastError();
    }
};

template <class Cfg>
cudaError_t launch_step_batch(const unsigned char* d_args, const int4* d_tiles, int ntiles, int bx, int grid,
                              bool is3d, int seed, bool open, cudaStream_t stream)
{
    if (ntiles <= 0) return cudaSuccess;
    if (bx != 32 && bx != 64 && bx != 128) return cudaErrorInvalidValue;
    const cudaError_t e = configure_step_kernels<Cfg>();
    if (e != cudaSuccess) return e;
    const int g = grid > 0 && grid < ntiles ? grid : ntiles;
    return dispatch_variant(is3d, seed, open, LaunchBatch<Cfg>{d_args, d_tiles, ntiles, bx, g, stream});
}

template <class Cfg>
struct PersistentOccupancy {
    int* nb;
    template <bool D, int S, bool O>
    cudaError_t run()
    {
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(nb, step_persistent_kernel<Cfg, D, S, O>,
                                                             kStepThreads, batch_smem_bytes<Cfg>(S));
    }
};

template <class Cfg>
struct LaunchPersistent {
    const unsigned char* args;
    size_t parity_bytes;
    int in0;
    const int4* tiles;
    int ntiles, bx, nsteps, grid;
    unsigned int* counter;
    int* status;
    unsigned long long wait_ns;
    cudaStream_t stream;
    template <bool D, int S, bool O>
    cudaError_t run()
    {
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3(grid);
        cfg.blockDim = dim3(kStepThreads);
        cfg.dynamicSmemBytes = batch_smem_bytes<Cfg>(S);
        cfg.stream = stream;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeCooperative;
        at[0].val.cooperative = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        return cudaLaunchKernelEx(&cfg, step_persistent_kernel<Cfg, D, S, O>, args, parity_bytes, in0, tiles, ntiles,
                                  bx, nsteps, counter, status, wait_ns);
    }
};

// resident blocks per SM of the persistent kernel (its grid is this times the SM count)
template <class Cfg>
int persistent_blocks_per_sm(bool is3d, int seed, bool open)
{
    if (configure_step_kernels<Cfg>() != cudaSuccess) return 0;
    int nb = 0;
    const cudaError_t e = dispatch_variant(is3d, seed, open, PersistentOccupancy<Cfg>{&nb});
    return e == cudaSuccess ? nb : 0;
}

// nsteps steps of every run of one kernel variant in one cooperative launch;
// *counter must be 0 on entry (the caller clears it on the stream)
template <class Cfg>
cudaError_t launch_step_persistent(const unsigned char* d_args, size_t parity_bytes, int in0, const int4* d_tiles,
                                   int ntiles, int bx, int nsteps, int grid, bool is3d, int seed, bool open,
                                   unsigned int* counter, int* status, unsigned long long wait_ns,
                                   cudaStream_t stream)
{
    if (ntiles <= 0 || nsteps <= 0) return cudaSuccess;
    if (bx != 32 && bx != 64 && bx != 128) return cudaErrorInvalidValue;
    const cudaError_t e = configure_step_kernels<Cfg>();
    if (e != cudaSuccess) return e;
    return dispatch_variant(is3d, seed, open,
                            LaunchPersistent<Cfg>{d_args, parity_bytes, in0, d_tiles, ntiles, bx, nsteps, grid,
                                                  counter, status, wait_ns, stream});
}

template <class Cfg>
struct LaunchRun {
    const StepArgs<Cfg>* A;
    dim3 grid, block;
    cudaStream_t stream;
    template <bool D, int S, bool O>
    cudaError_t run()
    {
        step_kernel<Cfg, D, S, O><<<grid, block, step_smem_bytes<Cfg>(S), stream>>>(*A);
        return cudaGetLastError();
    }
};

template <class Cfg>
cudaError_t launch_step(const StepArgs<Cfg>& A, cudaStream_t stream, const TileLaunch* tl)
{
    if constexpr (kTileCapable<Cfg>) {
        if (tl && tile_path(A, tl->maps)) {
            const cudaError_t ce = configure_step_kernels<Cfg>();
            if (ce != cudaSuccess) return ce;
            const TileRange tr = interior_tiles(A.nx, A.ny, TileGeo<Cfg>::PX);
            if (tr.nx > 0 && tr.ny > 0) {
                // persistent: one wave of resident blocks walking the tiles
                const int per_sm = A.seed == SEED_MLP ? TileMinBlocks<Cfg, SEED_MLP>::value
                                   : A.seed == SEED_COLD ? TileMinBlocks<Cfg, SEED_COLD>::value
                                                         : TileMinBlocks<Cfg, SEED_PREV>::value;
                const int ntiles = tr.nx * tr.ny;
                const int grid = min(ntiles, per_sm * tl->sms);
                const size_t sm = tile_smem_bytes<Cfg>(A.seed);
                if (A.seed == SEED_MLP)
                    step_tile_kernel<Cfg, SEED_MLP><<<grid, kTileThreads, sm, stream>>>(A, *tl->maps, tr);
                else if (A.seed == SEED_COLD)
                    step_tile_kernel<Cfg, SEED_COLD><<<grid, kTileThreads, sm, stream>>>(A, *tl->maps, tr);
                else
                    step_tile_kernel<Cfg, SEED_PREV><<<grid, kTileThreads, sm, stream>>>(A, *tl->maps, tr);
                const cudaError_t e = cudaGetLastError();
                if (e != cudaSuccess) return e;
            }
            // the edge tiles, cell by cell, from the run's argument record in device memory
            return launch_step_batch<Cfg>(tl->args, tl->edge_tiles, tl->nedge, 32, 0, false, A.seed, false, stream);
        }
    }
    const int bx = A.nx >= LB_STEP_BX ? LB_STEP_BX : (A.nx >= 64 ? 64 : 32);
    const int by = kStepThreads / bx;
    const cudaError_t ce = configure_step_kernels<Cfg>();
    if (ce != cudaSuccess) return ce;
    const dim3 block(bx, by, 1);
    const dim3 grid((A.nx + bx - 1) / bx, (A.ny + by - 1) / by, A.nz);
    return dispatch_variant(A.nz > 1, A.seed, A.open_mask != 0, LaunchRun<Cfg>{&A, grid, block, stream});
}

}  // namespace lb

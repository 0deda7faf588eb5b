// lattice.cuh -- lattice constants and per-cell physics of the RRMHD lattice
// Boltzmann step (arXiv:1508.03452, Sec. III), written for the GPU path.
//
// Conventions (shared with the C ABI, restated here from the paper):
//  * D3Q19 (Eq. cellconfigs1), population order: rest; +x,-x,+y,-y,+z,-z;
//    +x+y,-x-y,+x-y,-x+y; +x+z,-x-z,+x-z,-x+z; +y+z,-y-z,+y-z,-y+z.
//  * The temperature parameter is nu = sqrt(27), so c_t = c_0, the momentum
//    vectors are p_i = (1, q chat_i) with q = c_a = sqrt(19/27), and the
//    weights are w_0 = -44/361, w_axis = 99/722, w_diag = 9/361 (nu cancels
//    from them) and, for Eq. Hupp, w'_0 = 1/10, w'_axis = 6/95, w'_diag = 33/760.
//  * D3Q13 (Maxwell subsection): moving population k = 8 p + 2 i + j, plane p
//    spanned by axes (a1, a2) = (x, y), (x, z), (y, z); v_i^p = sqrt(2) c hop_i
//    with hop_0..3 = (+,+), (-,+), (-,-), (+,-) in (a1, a2); e_{i0} = v_{(i+3)%4}/2,
//    e_{i1} = -e_{i0}; b_{i0} = -o_p, b_{i1} = +o_p with o_p = a1 x a2 (= +z, -y,
//    +x). Index 24 is the rest population h_0.
//  * Fluid populations are handled as deviations from the rest equilibrium of a
//    reference state (n_r, eps_r, p_r): d_i = f_i - f_i^eq(n_r, eps_r, 0, 0, 0),
//    so that small flows keep full relative precision in float32.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lb {

// ---------------------------------------------------------------------------
// tables
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int c19(int i, int a)
{
    constexpr int t[19][3] = {{0, 0, 0},  {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},  {0, 0, -1},
                              {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}, {1, 0, 1},  {-1, 0, -1}, {1, 0, -1},
                              {-1, 0, 1}, {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
    return t[i][a];
}

__host__ __device__ constexpr int c19_norm1(int i) { return (c19(i, 0) != 0) + (c19(i, 1) != 0) + (c19(i, 2) != 0); }

// weight of Eq. Dis_fun_EM (nu = sqrt 27)
__host__ __device__ constexpr double w19(int i)
{
    return c19_norm1(i) == 0 ? -44.0 / 361.0 : (c19_norm1(i) == 1 ? 99.0 / 722.0 : 9.0 / 361.0);
}

// weight of Eq. Hupp (nu = sqrt 27, c_a^2 = 19/27)
__host__ __device__ constexpr double wg19(int i)
{
    return c19_norm1(i) == 0 ? 1.0 / 10.0 : (c19_norm1(i) == 1 ? 6.0 / 95.0 : 33.0 / 760.0);
}

// D3Q13: plane axes, hop signs, normal orientation
__host__ __device__ constexpr int plane_a1(int p) { return p == 2 ? 1 : 0; }
__host__ __device__ constexpr int plane_a2(int p) { return p == 0 ? 1 : 2; }
__host__ __device__ constexpr int plane_normal(int p) { return p == 0 ? 2 : (p == 1 ? 1 : 0); }
__host__ __device__ constexpr int plane_orient(int p) { return p == 1 ? -1 : 1; }
__host__ __device__ constexpr int hop_s1(int i) { return (i == 0 || i == 3) ? 1 : -1; }
__host__ __device__ constexpr int hop_s2(int i) { return (i == 0 || i == 1) ? 1 : -1; }
// lattice hop of moving population k along axis a
__host__ __device__ constexpr int hop13(int k, int a)
{
    return a == plane_a1(k / 8) ? hop_s1((k % 8) / 2) : (a == plane_a2(k / 8) ? hop_s2((k % 8) / 2) : 0);
}

// numerical constants
constexpr double kQ = 0.838870492807861077470742756327;      // sqrt(19/27): c_a with nu = sqrt 27
constexpr double kQ2 = 19.0 / 27.0;
constexpr double kL1 = 3.35548197123144430988297102531;     // sqrt(19) (sqrt(27)/2 - 1) / c_0, c_0 = 3/8 (9 - 2 sqrt 3)
constexpr double kSqrt19_3 = 2.51661147842358323241222826898; // sqrt(19/3): Poynting term, nu c_a / sqrt 3
constexpr double kRest = 3.0 / 4.0 * 361.0 / 33.0;          // 3/4 * 361/33 (rest-population EOS term)
constexpr double kSqrt2 = 1.41421356237309504880168872421;

// ---------------------------------------------------------------------------
// per-run constants in compute precision
// ---------------------------------------------------------------------------
template <class R>
struct Phys {
    R c, c2, inv_c, eps0;      // eps0 = 1 / c^2 (mu0 = 1)
    R sigma, inv_tau;          // conductivity, dt / tau
    R half_dt_c2;              // (dt/2) mu0 c^2
    R inv_half_dt_c2;          // 1 / ((dt/2) mu0 c^2)
    R gm1;                     // Gamma - 1
    R C, kappa, kvisc;         // Courant number, (1 - C)/2, alpha c dt / dx
    R n_r, eps_r, p_r;         // reference rest state of the deviations
    R dx;                      // lattice spacing
    R Er[3], Br[3];            // reference fields of the h deviations (h_ref = h^eq(Er, Br, J = 0, rho = 0))
    R dXr[3][3], dYr[3];       // reference EM terms of the f deviations minus their values at (Er, Br)
    R Tem[10];                 // moments of the reference EM terms: T^00, T^0a (3), T^ab (xx, yy, zz, xy, xz, yz)
    R tol;                     // recovery tolerance (relative change of beta)
    int maxit;
};

template <class R>
struct Prim {
    R n, eps, u[3], E[3], B[3], rho;
};

template <class R>
__device__ __forceinline__ R sq(R a) { return a * a; }

__device__ __forceinline__ float rsqrt_r(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_r(double x) { return rsqrt(x); }

// 1/x where a few ulp do not matter (a relaxation factor, a spectral shift):
// the hardware reciprocal approximation in float32, the division in float64
__device__ __forceinline__ float rcp_approx(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double rcp_approx(double x) { return 1.0 / x; }

// ---------------------------------------------------------------------------
// equilibria in deviation form (restated from Eq. Dis_fun_EM with the
// readings of the delta_{i0} term, the sign of the nu^2/5 term, the
// c_a^y c_a^z typo and the c in the Poynting term; and Eq. Hupp)
//
//   f_i^eq = w_i [ 3 p + d_{i0} (3/4)(361/33)(3p - eps) + (3/4)(eps + p) Q_i + EM_i ]
//   Q_i  = L1 g^2 (c.b) + 19 g^2 sum_{a<b} c_a c_b b_a b_b + (4/15) g^2 (19 sum_a c_a^2 b_a^2 - 4 b^2)
//   EM_i = 2.3 tr X - sqrt(19/3) Y.c - 3.8 sum_a c_a^2 X_aa - 14.25 sum_{a<b} c_a c_b X_ab,
//          X_ab = eps0 (E_a E_b + c^2 B_a B_b), Y = eps0 c (B x E)
// The deviations subtract the reference rest state and a reference (Xr, Yr)
// of the EM terms; X - Xr and Y - Yr are formed from the field deviations
// dE = E - Er, dB = B - Br so that a uniform background field costs no
// float32 precision.
//   g_i^eq = w'_i n g (1 + 3 q c.b + 4.5 q^2 (c.b)^2 - 1.5 b^2)
// (b = u / c, g = Lorentz factor, c = chat_i)
// ---------------------------------------------------------------------------
// Per-cell terms of the equilibria. With chat_i having one (axis a, sign s) or
// two (axes a < b, signs s_a, s_b) non-zero components:
//   f^eq - W = w_i (even + s odd_a)                                    axis
//            = w_i (even_ab + s_a odd_a + s_b odd_b + s_a s_b cross_ab)   diagonal
//            = w_0 rest                                                rest
// with odd_a = (3/4)(eps + p) g^2 L1 b_a + EM_lin_a, and the even parts
// collecting 3 (p - p_r), the quadratic velocity terms and the EM terms; the
// same split for g^eq (base, lin_a, sq_a, x_ab) and for K_i = kf - sum s_a kq_a.
template <class R>
struct EqCell {
    R f_rest, f_even_ax[3], f_odd[3], f_even_dg[3], f_cross[3];
    R g_base, g_lin[3], g_sq[3], g_x[3];
    R kf, kq[3];
};

// n_dev = n - n_r, eps_dev = eps - eps_r, dE = E - Er and dB = B - Br are passed
// separately so that the float32 path never rounds the large reference values
// into the deviations.
template <class R>
__device__ __forceinline__ void eq_cell(const Prim<R>& s, R n_dev, R eps_dev, const R* dE, const R* dB,
                                        const Phys<R>& k, EqCell<R>& q)
{
    const R b[3] = {s.u[0] * k.inv_c, s.u[1] * k.inv_c, s.u[2] * k.inv_c};
    const R b2 = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
    const R g2 = R(1) / (R(1) - b2);
    const R g = sqrt(g2);
    const R p_dev = k.gm1 * (eps_dev - n_dev * k.c2);
    const R three_dp = R(3) * p_dev;
    const R rest_dev = R(kRest) * (R(3) * p_dev - eps_dev);
    const R wq = R(0.75) * (s.eps + k.p_r + p_dev);
    const R* E = s.E;
    const R* B = s.B;
    // X - Xr = eps0 [dE_a E_b + Er_a dE_b + c^2 (dB_a B_b + Br_a dB_b)] - dXr
    R X[3][3];
    for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 3; ++c)
            X[a][c] = k.eps0 * (dE[a] * E[c] + k.Er[a] * dE[c] + k.c2 * (dB[a] * B[c] + k.Br[a] * dB[c])) - k.dXr[a][c];
    // Y - Yr = eps0 c (dB x E + Br x dE) - dYr
    const R Yd[3] = {
        k.eps0 * k.c * (dB[1] * E[2] - dB[2] * E[1] + k.Br[1] * dE[2] - k.Br[2] * dE[1]) - k.dYr[0],
        k.eps0 * k.c * (dB[2] * E[0] - dB[0] * E[2] + k.Br[2] * dE[0] - k.Br[0] * dE[2]) - k.dYr[1],
        k.eps0 * k.c * (dB[0] * E[1] - dB[1] * E[0] + k.Br[0] * dE[1] - k.Br[1] * dE[0]) - k.dYr[2]};
    const R em_iso = R(2.3) * (X[0][0] + X[1][1] + X[2][2]);
    const R qd = g2 * R(16.0 / 15.0) * b2;  // Q of the rest population is -qd
    R qs[3];
    for (int a = 0; a < 3; ++a) {
        qs[a] = g2 * R(4.0 / 15.0) * (R(19) * b[a] * b[a] - R(4) * b2);
        q.f_even_ax[a] = three_dp + wq * qs[a] + em_iso - R(3.8) * X[a][a];
        q.f_odd[a] = wq * g2 * R(kL1) * b[a] - R(kSqrt19_3) * Yd[a];
    }
    q.f_rest = three_dp + rest_dev - wq * qd + em_iso;
    const int pa[3] = {0, 0, 1}, pb[3] = {1, 2, 2};
    for (int m = 0; m < 3; ++m) {
        const int a = pa[m], c = pb[m];
        q.f_even_dg[m] = three_dp + wq * (qs[a] + qs[c] + qd) + em_iso - R(3.8) * (X[a][a] + X[c][c]);
        q.f_cross[m] = wq * R(19) * g2 * b[a] * b[c] - R(14.25) * X[a][c];
    }
    const R ng = s.n * g;
    // n g - n_r = n_dev g + n_r (g - 1), g - 1 = g^2 b^2 / (g + 1)
    const R dng = n_dev * g + k.n_r * (g2 * b2 / (g + R(1)));
    q.g_base = dng - R(1.5) * ng * b2;
    for (int a = 0; a < 3; ++a) {
        q.g_lin[a] = R(3) * R(kQ) * ng * b[a];
        q.g_sq[a] = R(4.5) * R(kQ2) * ng * b[a] * b[a];
    }
    for (int m = 0; m < 3; ++m) q.g_x[m] = R(9) * R(kQ2) * ng * b[pa[m]] * b[pb[m]];
    q.kf = g * k.inv_tau;
    for (int a = 0; a < 3; ++a) q.kq[a] = q.kf * R(kQ) * b[a];
}

template <class R>
__device__ __forceinline__ void eq_cell(const Prim<R>& s, const Phys<R>& k, EqCell<R>& q)
{
    const R dE[3] = {s.E[0] - k.Er[0], s.E[1] - k.Er[1], s.E[2] - k.Er[2]};
    const R dB[3] = {s.B[0] - k.Br[0], s.B[1] - k.Br[1], s.B[2] - k.Br[2]};
    eq_cell(s, s.n - k.n_r, s.eps - k.eps_r, dE, dB, k, q);
}

// axes of population I: first and second non-zero component (-1 if none)
__host__ __device__ constexpr int ax1(int i) { return c19(i, 0) ? 0 : (c19(i, 1) ? 1 : (c19(i, 2) ? 2 : -1)); }
__host__ __device__ constexpr int ax2(int i)
{
    return ax1(i) < 0 ? -1 : (ax1(i) < 1 && c19(i, 1) ? 1 : (ax1(i) < 2 && c19(i, 2) ? 2 : -1));
}

// f_i^eq - f_i^eq(reference state), population I
template <int I, class R>
__device__ __forceinline__ R feq_dev(const EqCell<R>& q)
{
    constexpr int a = ax1(I), b = ax2(I);
    if constexpr (a < 0) {
        return R(w19(I)) * q.f_rest;
    } else if constexpr (b < 0) {
        constexpr int sa = c19(I, a);
        return R(w19(I)) * (q.f_even_ax[a] + R(sa) * q.f_odd[a]);
    } else {
        constexpr int sa = c19(I, a), sb = c19(I, b), m = a + b - 1;
        return R(w19(I)) * (q.f_even_dg[m] + R(sa) * q.f_odd[a] + R(sb) * q.f_odd[b] + R(sa * sb) * q.f_cross[m]);
    }
}

// g_i^eq - g_i^eq(reference state), population I
template <int I, class R>
__device__ __forceinline__ R geq_dev(const EqCell<R>& q)
{
    constexpr int a = ax1(I), b = ax2(I);
    if constexpr (a < 0) {
        return R(wg19(I)) * q.g_base;
    } else if constexpr (b < 0) {
        constexpr int sa = c19(I, a);
        return R(wg19(I)) * (q.g_base + q.g_sq[a] + R(sa) * q.g_lin[a]);
    } else {
        constexpr int sa = c19(I, a), sb = c19(I, b), m = a + b - 1;
        return R(wg19(I)) * (q.g_base + q.g_sq[a] + q.g_sq[b] + R(sa * sb) * q.g_x[m] + R(sa) * q.g_lin[a] +
                             R(sb) * q.g_lin[b]);
    }
}

// Anderson-Witting collision factor K_i = (dt/tau) g (1 - v_i.u / c^2), v_i = c q chat_i
template <int I, class R>
__device__ __forceinline__ R k_aw(const EqCell<R>& q)
{
    constexpr int a = ax1(I), b = ax2(I);
    if constexpr (a < 0) {
        return q.kf;
    } else if constexpr (b < 0) {
        return q.kf - R(c19(I, a)) * q.kq[a];
    } else {
        return q.kf - R(c19(I, a)) * q.kq[a] - R(c19(I, b)) * q.kq[b];
    }
}

// ---------------------------------------------------------------------------
// Maxwell equilibrium (Eq. Maxwell-eq), restated per (plane, i):
//   h_{i0}^eq = a + e - m,  h_{i1}^eq = a - e + m
//   a = (sqrt2 c / 16) hop_i . J,  e = (sqrt2 / (16 c)) hop_{(i+3)%4} . E,
//   m = (1/8) o_p B_normal
// ---------------------------------------------------------------------------
template <int K, class R>
__device__ __forceinline__ R heq13(const R* E, const R* B, const R* J, const Phys<R>& k)
{
    constexpr int p = K / 8, i = (K % 8) / 2, j = K % 2;
    constexpr int a1 = plane_a1(p), a2 = plane_a2(p);
    constexpr int ie = (i + 3) % 4;
    const R a = R(kSqrt2 / 16.0) * k.c * (R(hop_s1(i)) * J[a1] + R(hop_s2(i)) * J[a2]);
    const R e = R(kSqrt2 / 16.0) * k.inv_c * (R(hop_s1(ie)) * E[a1] + R(hop_s2(ie)) * E[a2]);
    const R m = R(0.125) * R(plane_orient(p)) * B[plane_normal(p)];
    return j == 0 ? a + e - m : a - e + m;
}

// EM moments of the 25 populations (Eqs. Cal_E, Cal_B, Cal_rhoc) for h stored as
// deviations from h_ref = h^eq(Er, Br, 0, 0): returns E' - Er, B - Br and rho_c
// (h_ref carries no charge)
template <class R>
__device__ __forceinline__ void em_moments(const R* h, const Phys<R>& k, R* Ep, R* B, R& rho)
{
    Ep[0] = Ep[1] = Ep[2] = R(0);
    B[0] = B[1] = B[2] = R(0);
    rho = h[24];
#pragma unroll
    for (int p = 0; p < 3; ++p) {
        R bn = R(0);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const R h0 = h[8 * p + 2 * i], h1 = h[8 * p + 2 * i + 1];
            const R d = h0 - h1;
            const int ie = (i + 3) % 4;
            Ep[plane_a1(p)] += d * R(hop_s1(ie));
            Ep[plane_a2(p)] += d * R(hop_s2(ie));
            bn += h1 - h0;
            rho += h0 + h1;
        }
        B[plane_normal(p)] = R(plane_orient(p)) * bn;
    }
    const R s = R(kSqrt2 / 2.0) * k.c;
    Ep[0] *= s; Ep[1] *= s; Ep[2] *= s;
}

// ---------------------------------------------------------------------------
// Ohm-coupled E solve (Eqs. Ohm and Ex_force, closed form)
//   [(1+k) I - (k/c^2) u u^T] E = E' - k u x B - (dt/2) c^2 rho u,  k = (dt/2) c^2 sigma g
//   E = a/(1+k) - k/(1+k) u x B + k/(1+k) (u.a) u / (c^2 (1 + k/g^2)),  a = E' - (dt/2) c^2 rho u
// The caller takes J from Eq. Ex_force, J = (E' - E) / ((dt/2) mu0 c^2),
// which equals Eq. Ohm at the solution and stays accurate at large sigma in
// float32.
// ---------------------------------------------------------------------------
// With ig = 1/g: 1 + k/g^2 = 1 + (dt/2) c^2 sigma ig, and one reciprocal of
// D = (1 + k)(1 + k/g^2) gives both 1/(1+k) and the u u^T coefficient.
template <class R>
__device__ __forceinline__ void ohm_solve(const R* Ep, const R* u, const R* B, R rho, R g, R ig, const Phys<R>& k,
                                          R* E)
{
    const R hs = k.half_dt_c2 * k.sigma;
    const R kk = hs * g;
    const R kg = R(1) + hs * ig;  // 1 + k/g^2
    const R inv = R(1) / ((R(1) + kk) * kg);
    const R inv1k = kg * inv;
    const R kfrac = kk * inv1k;
    R a[3];
    for (int c = 0; c < 3; ++c) a[c] = Ep[c] - k.half_dt_c2 * rho * u[c];
    const R ua = u[0] * a[0] + u[1] * a[1] + u[2] * a[2];
    const R s = kk * ua * inv * (k.inv_c * k.inv_c);
    const R uxB[3] = {u[1] * B[2] - u[2] * B[1], u[2] * B[0] - u[0] * B[2], u[0] * B[1] - u[1] * B[0]};
    for (int c = 0; c < 3; ++c) E[c] = a[c] * inv1k - kfrac * uxB[c] + s * u[c];
}

// J from Eq. Ohm for stored primitives (initial state, outputs, driven cells)
template <class R>
__device__ __forceinline__ void ohm_current(const R* E, const R* u, const R* B, R rho, const Phys<R>& k, R* J)
{
    const R g = R(1) / sqrt(R(1) - (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]) * k.inv_c * k.inv_c);
    const R uxB[3] = {u[1] * B[2] - u[2] * B[1], u[2] * B[0] - u[0] * B[2], u[0] * B[1] - u[1] * B[0]};
    const R Eu = E[0] * u[0] + E[1] * u[1] + E[2] * u[2];
    for (int c = 0; c < 3; ++c) J[c] = k.sigma * g * (E[c] + uxB[c] - Eu * u[c] * k.inv_c * k.inv_c) + rho * u[c];
}

// ---------------------------------------------------------------------------
// Landau eigen-solve (coupling subsection): largest eigenpair of
// A = [T - eps0 F F(E, B)] eta (T and B given by landau_b) by a power
// iteration, shifted by p_old - s
// (s = eps0 (c^2 B^2 - E^2) / 2; the shift pushes the spacelike eigenvalues
// to ~0) unless `shifted` is false (the paper's plain power method), started
// from the velocity `seed` (beta); convergence is accepted from iteration
// `min_it` on. T holds the moments with eps_r taken out of T^00 (the
// reference rest state's other entries included); the returned lambda is the
// eigenvalue minus eps_r, s_old the s of (E, B). Returns the iteration count,
// or -1 if it failed.
// ---------------------------------------------------------------------------
template <class R>
struct LandauB {
    R t00, t0[3], tab[3][3];  // T with the magnetic stresses eps0 c^2 (d_ab B^2 - B_a B_b) taken out
    R B[3], sB;               // B and eps0 c^2 B^2 / 2
};

// The part of the Landau matrix that does not depend on E (for fixed B).
// T[0][0] holds T^00 - eps_r: A[0][0] and lambda are deviations from eps_r.
template <class R>
__device__ __forceinline__ void landau_b(const R T[4][4], const R* B, const Phys<R>& k, LandauB<R>& L)
{
    const R B2 = B[0] * B[0] + B[1] * B[1] + B[2] * B[2];
    L.t00 = T[0][0];
    for (int a = 0; a < 3; ++a) {
        L.B[a] = B[a];
        L.t0[a] = T[0][a + 1];
        for (int b = 0; b < 3; ++b)
            L.tab[a][b] = T[a + 1][b + 1] - k.eps0 * k.c2 * ((a == b ? B2 : R(0)) - B[a] * B[b]);
    }
    L.sB = R(0.5) * k.eps0 * k.c2 * B2;
}

template <class R>
__device__ __forceinline__ int landau(const LandauB<R>& L, const R* E, R p_old, const Phys<R>& k, R beta[3],
                                      R& lambda, R& s_old, const R* seed, bool shifted, int min_it)
{
    const R* B = L.B;
    const R E2 = E[0] * E[0] + E[1] * E[1] + E[2] * E[2];
    const R ExB[3] = {E[1] * B[2] - E[2] * B[1], E[2] * B[0] - E[0] * B[2], E[0] * B[1] - E[1] * B[0]};
    // S = eps0 F^{mu rho} F_rho^nu: S00 = eps0 E^2, S0a = eps0 c (E x B)_a,
    // Sab = eps0 [-E_a E_b + c^2 (d_ab B^2 - B_a B_b)]; A = (T - S) eta
    R A[4][4];
    A[0][0] = L.t00 - k.eps0 * E2;
    for (int a = 0; a < 3; ++a) {
        const R m0a = L.t0[a] - k.eps0 * k.c * ExB[a];
        A[0][a + 1] = -m0a;
        A[a + 1][0] = m0a;
        for (int b = 0; b < 3; ++b) A[a + 1][b + 1] = -(L.tab[a][b] + k.eps0 * E[a] * E[b]);
    }
    s_old = L.sB - R(0.5) * k.eps0 * E2;
    const R shift = shifted ? p_old - s_old : R(0);
    const R a00_full = k.eps_r + shift;  // eps_r restored in the first row only
    R v1 = seed[0], v2 = seed[1], v3 = seed[2];
    int it = 0;
    bool done = false;
#pragma unroll 1
    for (it = 1; it <= k.maxit; ++it) {
        const R w0 = A[0][0] + A[0][1] * v1 + A[0][2] * v2 + A[0][3] * v3 + a00_full;
        const R w1 = A[1][0] + (A[1][1] + shift) * v1 + A[1][2] * v2 + A[1][3] * v3;
        const R w2 = A[2][0] + A[2][1] * v1 + (A[2][2] + shift) * v2 + A[2][3] * v3;
        const R w3 = A[3][0] + A[3][1] * v1 + A[3][2] * v2 + (A[3][3] + shift) * v3;
        const R iw = rcp_approx(w0);  // a scale error is undone by the next iteration
        const R n1 = w1 * iw, n2 = w2 * iw, n3 = w3 * iw;
        const R d2 = sq(n1 - v1) + sq(n2 - v2) + sq(n3 - v3);
        const R b2 = n1 * n1 + n2 * n2 + n3 * n3;
        v1 = n1; v2 = n2; v3 = n3;
        if (it >= min_it && (d2 <= k.tol * k.tol * b2 || d2 == R(0))) {
            done = true;
            break;
        }
    }
    if (!done) return -1;
    lambda = A[0][0] + A[0][1] * v1 + A[0][2] * v2 + A[0][3] * v3;
    beta[0] = v1; beta[1] = v2; beta[2] = v3;
    const R b2 = v1 * v1 + v2 * v2 + v3 * v3;
    if (!(b2 < R(1)) || !(lambda == lambda)) return -1;
    return it;
}

}  // namespace lb

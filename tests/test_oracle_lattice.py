"""Pins of the oracle's lattices and equilibria against what the paper fixes.

Each test compares the oracle with something independent of it: the printed
components of the stress-energy tensors, the printed moment definitions, the
geometry the paper states for the D3Q13 lattice, or Maxwell's equations.
"""
import itertools
import math

import numpy as np
import pytest

import oracle as O

NUS = [0.0, 5.0, 4.5]  # 0 -> the default sqrt(27)
CS = [1.0, 2.5]


def textbook_stress_energy(n, p, u, E, B, c, gamma_ad=4.0 / 3.0):
    """Eq. EM_Fluid (perfect fluid) + the printed components of T_EM, in
    components with x^0 = c t; written here from the printed formulas, not from
    the oracle."""
    eps = n * c * c + p / (gamma_ad - 1.0)
    gam = 1.0 / math.sqrt(1.0 - u @ u / (c * c))
    U = gam * np.array([c, *u])
    eta = np.diag([1.0, -1.0, -1.0, -1.0])
    Tf = (eps + p) * np.outer(U, U) / (c * c) - p * eta
    eps0 = 1.0 / (c * c)
    Tem = np.zeros((4, 4))
    Tem[0, 0] = 0.5 * eps0 * (E @ E + c * c * B @ B)
    Tem[0, 1:] = Tem[1:, 0] = np.cross(E, B) / c  # 1/(mu0 c) (E x B)
    Tem[1:, 1:] = eps0 * (-np.outer(E, E) - c * c * np.outer(B, B) + 0.5 * (E @ E + c * c * B @ B) * np.eye(3))
    return eps, Tf, Tem


def random_state(rng, c):
    n = rng.uniform(0.5, 2.0)
    p = rng.uniform(0.2, 3.0)
    u = rng.uniform(-0.4, 0.4, 3) * c
    E = rng.uniform(-0.3, 0.3, 3) * c
    B = rng.uniform(-0.3, 0.3, 3)
    return n, p, u, E, B


def test_weights_sum_to_one():
    """The D3Q19 weights satisfy sum w_i = 1 and the Eq. Hupp weights sum to 1,
    for any value of the temperature parameter nu."""
    for nu in NUS:
        L = O.lattice(O.make_params(nu=nu))
        assert abs(L["w"].sum() - 1.0) < 1e-14
        assert abs(L["wg"].sum() - 1.0) < 1e-14


def test_d3q19_directions():
    """Eq. cellconfigs1: one rest vector, 6 axis and 12 face-diagonal vectors,
    each set fully symmetric."""
    L = O.lattice(O.make_params())
    ch = L["chat"]
    assert len({tuple(v) for v in ch}) == 19
    norms = np.abs(ch).sum(axis=1)
    assert (norms == 0).sum() == 1 and (norms == 1).sum() == 6 and (norms == 2).sum() == 12
    assert np.all(ch.sum(axis=0) == 0)
    assert np.all(np.abs(ch).max(axis=1) <= 1)


@pytest.mark.parametrize("c", CS)
def test_d3q13_geometry(c):
    """Sec. III (Maxwell): |v| = 2c, e perpendicular to v in the same plane,
    b perpendicular to the plane; 13 distinct e and 7 distinct b vectors once the
    null vectors are added; with dx/dt = sqrt(2) c each v dt is one face-diagonal
    lattice hop."""
    P = O.make_params(c=c)
    L = O.lattice(P)
    v, e, b, hop = L["v"], L["e"], L["b"], L["hop"]
    assert np.allclose(np.linalg.norm(v, axis=1), 2 * c, rtol=0, atol=1e-14 * c)
    assert np.allclose(np.einsum("ka,ka->k", v, e), 0, atol=1e-14 * c * c)
    for k in range(24):
        normal = np.cross(v[k], e[k])
        assert np.linalg.norm(np.cross(b[k], normal)) < 1e-13 * c * c
    keys = lambda arr: {tuple(np.round(r / (c if c else 1), 12) + 0.0) for r in arr}
    assert len(keys(e) | {(0.0, 0.0, 0.0)}) == 13
    assert len({tuple(np.round(r, 12) + 0.0) for r in b} | {(0.0, 0.0, 0.0)}) == 7
    dt = O.dt(P)
    assert np.allclose(v * dt / P.dx, hop, atol=1e-12)
    assert np.all(np.abs(hop).sum(axis=1) == 2) and np.all(np.abs(hop).max(axis=1) == 1)


@pytest.mark.parametrize("c,nu", list(itertools.product(CS, NUS)))
def test_feq_reproduces_total_stress_energy(c, nu):
    """Eq. Dis_fun_EM: sum_i p_i^mu p_i^nu f_i^eq = T_fluid + T_EM exactly (the
    paper's stated purpose of the equilibrium); nu drops out."""
    rng = np.random.default_rng(1)
    P = O.make_params(c=c, nu=nu)
    for _ in range(6):
        n, p, u, E, B = random_state(rng, c)
        eps, Tf, Tem = textbook_stress_energy(n, p, u, E, B, c)
        f = O.feq(P, n, eps, u, E, B)
        T, _, _, _, _ = O.moments(P, f, np.zeros(19), np.zeros(25))
        assert np.abs(T - Tf - Tem).max() <= 1e-13 * np.abs(Tf).max()


def test_feq_as_printed_breaks_the_moments():
    """The printed delta_{i0} term and the printed sign of the nu^2/5 term give
    O(1) errors in the moments: the readings are forced by the printed T_EM."""
    rng = np.random.default_rng(2)
    P = O.make_params(flags=O.PRINTED_FEQ)
    n, p, u, E, B = random_state(rng, 1.0)
    eps, Tf, Tem = textbook_stress_energy(n, p, u, E, B, 1.0)
    T, _, _, _, _ = O.moments(P, O.feq(P, n, eps, u, E, B), np.zeros(19), np.zeros(25))
    assert np.abs(T - Tf - Tem).max() > 1e-2 * np.abs(Tf).max()


@pytest.mark.parametrize("c,nu", list(itertools.product(CS, NUS)))
def test_geq_reproduces_number_current(c, nu):
    """Eq. Hupp: sum_i p_i^mu g_i^eq = n U^mu / c (the density current N^mu =
    n U^mu of Eq. Density_cons, in units of c)."""
    rng = np.random.default_rng(3)
    P = O.make_params(c=c, nu=nu)
    for _ in range(6):
        n, _, u, _, _ = random_state(rng, c)
        g = O.geq(P, n, u)
        _, N, _, _, _ = O.moments(P, np.zeros(19), g, np.zeros(25))
        gam = 1.0 / math.sqrt(1.0 - u @ u / (c * c))
        assert np.allclose(N, n * gam * np.array([1.0, *(u / c)]), rtol=0, atol=1e-14 * n * gam)


@pytest.mark.parametrize("c", CS)
def test_heq_moments(c):
    """Eqs. Cal_E, Cal_B, Cal_rhoc applied to Eq. Maxwell-eq return E, B and
    rho_c."""
    rng = np.random.default_rng(4)
    P = O.make_params(c=c)
    for _ in range(5):
        E, B, J = rng.normal(size=3), rng.normal(size=3), rng.normal(size=3)
        rc = rng.normal()
        h = O.heq(P, E, B, J, rc)
        _, _, Ep, Bm, rcm = O.moments(P, np.zeros(19), np.zeros(19), h)
        assert np.allclose(Ep, E, atol=1e-14) and np.allclose(Bm, B, atol=1e-14)
        assert abs(rcm - rc) < 1e-14


@pytest.mark.parametrize("c", CS)
def test_maxwell_fluxes_give_ampere_and_faraday(c):
    """First-order fluxes of Eq. Maxwell-eq: sum h^eq v (x) e = c^2 eps_abc B_c and
    sum h^eq v (x) b = -eps_abc E_c, i.e. the streaming reproduces dE/dt = c^2
    curl B (Eq. Ampere) and dB/dt = -curl E (Eq. Faraday)."""
    P = O.make_params(c=c)
    L = O.lattice(P)
    eps3 = np.zeros((3, 3, 3))
    for a, b_, cc in itertools.permutations(range(3)):
        eps3[a, b_, cc] = np.linalg.det(np.eye(3)[[a, b_, cc]])
    rng = np.random.default_rng(5)
    E, B = rng.normal(size=3), rng.normal(size=3)
    h = O.heq(P, E, B, np.zeros(3), 0.0)[:24]
    assert np.allclose(np.einsum("k,ka,kb->ab", h, L["v"], L["e"]), c * c * np.einsum("abc,c->ab", eps3, B),
                       atol=1e-13 * c * c)
    assert np.allclose(np.einsum("k,ka,kb->ab", h, L["v"], L["b"]), -np.einsum("abc,c->ab", eps3, E), atol=1e-13)


@pytest.mark.parametrize("c", CS)
def test_em_contraction_matches_printed_tensor(c):
    """eps0 F^{mu rho} F^nu_rho + (eps0/4) F^2 eta (Eq. EM_EM, F from Eq.
    Maxwell_tensor) equals the printed T^00_EM, T^0i_EM, T^ij_EM, and
    F^{ab}F_{ab} = 2 (c^2 B^2 - E^2) as stated in the coupling subsection."""
    rng = np.random.default_rng(6)
    P = O.make_params(c=c)
    eta = np.diag([1.0, -1.0, -1.0, -1.0])
    for _ in range(4):
        E, B = rng.normal(size=3), rng.normal(size=3)
        S = O.em_ff(P, E, B)
        F = np.zeros(16)
        O.lib().orc_maxwell_tensor(c, O.oracle._dp(np.ascontiguousarray(E)), O.oracle._dp(np.ascontiguousarray(B)),
                                   O.oracle._dp(F))
        F = F.reshape(4, 4)
        F2 = np.einsum("ab,ac,bd,cd->", F, eta, eta, F)
        assert abs(F2 - 2 * (c * c * B @ B - E @ E)) < 1e-12 * (1 + c * c * B @ B + E @ E)
        _, _, Tem = textbook_stress_energy(1.0, 1.0, np.zeros(3), E, B, c)
        eps0 = 1.0 / (c * c)
        assert np.allclose(S + 0.25 * eps0 * F2 * eta, Tem, atol=1e-13 * (1 + np.abs(Tem).max()))

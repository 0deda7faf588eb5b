"""Pins of the oracle's Ohm solve and Landau eigen-solve (coupling subsection of
Sec. III) against closed forms, a direct linear solve and numpy's eigen-solver."""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_1508_03452_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def gamma_of(u, c):
    return 1.0 / math.sqrt(1.0 - u @ u / (c * c))


@pytest.mark.parametrize("c,sigma", [(1.0, 10.0), (1.0, 1e4), (2.5, 100.0)])
def test_ohm_solve_matches_direct_solve(c, sigma):
    """Eq. Ex_force with Eq. Ohm substituted is linear in E; the closed form must
    equal a direct 3x3 solve assembled here from the two printed equations, and
    satisfy E = E' - (dt/2) mu0 c^2 J(E)."""
    rng = np.random.default_rng(10)
    P = O.make_params(c=c, sigma=sigma)
    dt = O.dt(P)
    for _ in range(8):
        u = rng.uniform(-0.5, 0.5, 3) * c
        B, Ep = rng.normal(size=3), rng.normal(size=3) * c
        rc = rng.normal()
        gam = gamma_of(u, c)
        # J(E) = sigma gamma [E + u x B - (E.u) u / c^2] + rho_c u = A E + j0
        A = sigma * gam * (np.eye(3) - np.outer(u, u) / (c * c))
        j0 = sigma * gam * np.cross(u, B) + rc * u
        M = np.eye(3) + 0.5 * dt * c * c * A
        E_direct = np.linalg.solve(M, Ep - 0.5 * dt * c * c * j0)
        E = O.ohm_solve(P, Ep, u, B, rc)
        assert np.allclose(E, E_direct, rtol=1e-12, atol=1e-12 * np.abs(E_direct).max())
        J = O.ohm_current(P, E, u, B, rc)
        assert np.allclose(E, Ep - 0.5 * dt * c * c * J, rtol=0, atol=1e-10 * (1 + np.abs(Ep).max()))


def test_ohm_rest_frame():
    """In the fluid rest frame Eq. Ohm reduces to J = sigma E."""
    P = O.make_params(sigma=37.0)
    E = np.array([0.3, -0.2, 0.7])
    assert np.allclose(O.ohm_current(P, E, np.zeros(3), np.array([1.0, 2.0, 3.0]), 0.0), 37.0 * E, atol=1e-14)


def test_ohm_ideal_limit():
    """sigma -> infinity gives the ideal-MHD field E = -u x B (Eq. Ohm_ideal), with
    an O(1/sigma) remainder."""
    rng = np.random.default_rng(11)
    u, B, Ep = rng.uniform(-0.4, 0.4, 3), rng.normal(size=3), rng.normal(size=3)
    errs = []
    for sigma in (1e4, 1e6, 1e8):
        P = O.make_params(sigma=sigma)
        E = O.ohm_solve(P, Ep, u, B, 0.0)
        errs.append(np.abs(E + np.cross(u, B)).max())
    assert errs[1] < errs[0] / 50 and errs[2] < errs[1] / 50 and errs[2] < 1e-7


@pytest.mark.parametrize("c", [1.0, 2.5])
def test_landau_recovers_equilibrium_primitives(c):
    """The eigenvalue problem of the coupling subsection applied to the moments of
    an equilibrium (with the same E, B subtracted) returns eps, u and then
    n = N^0/U^0 of that equilibrium."""
    rng = np.random.default_rng(12)
    P = O.make_params(c=c)
    for _ in range(10):
        n, p = rng.uniform(0.5, 2.0), rng.uniform(0.2, 50.0)
        eps = n * c * c + p / (P.gamma_ad - 1.0)
        u = rng.uniform(-0.45, 0.45, 3) * c
        E, B = rng.uniform(-0.3, 0.3, 3) * c, rng.uniform(-0.3, 0.3, 3)
        f = O.feq(P, n, eps, u, E, B)
        g = O.geq(P, n, u)
        T, N, _, _, _ = O.moments(P, f, g, np.zeros(25))
        it, U, lam = O.landau(P, T, E, B, np.array([1.0, 0, 0, 0]))
        assert it > 0
        gam = gamma_of(u, c)
        assert np.allclose(U, gam * np.array([1.0, *(u / c)]), rtol=0, atol=1e-12 * gam)
        shift = 0.5 / (c * c) * (c * c * B @ B - E @ E)
        assert abs(lam - shift - eps) < 1e-12 * eps
        assert abs(N[0] / U[0] - n) < 1e-12 * n


def test_landau_matches_numpy_eig_off_equilibrium():
    """For a non-equilibrium tensor (equilibrium plus a random symmetric
    perturbation) the power method must land on numpy's largest eigenpair of
    [T - eps0 F F] eta."""
    rng = np.random.default_rng(13)
    P = O.make_params()
    eta = np.diag([1.0, -1.0, -1.0, -1.0])
    for _ in range(10):
        u = rng.uniform(-0.4, 0.4, 3)
        E, B = rng.uniform(-0.2, 0.2, 3), rng.uniform(-0.2, 0.2, 3)
        f = O.feq(P, 1.2, 4.0, u, E, B)
        T, _, _, _, _ = O.moments(P, f, np.zeros(19), np.zeros(25))
        D = rng.normal(scale=0.05, size=(4, 4))
        T = T + 0.5 * (D + D.T)
        it, U, lam = O.landau(P, T, E, B, np.array([1.0, 0, 0, 0]))
        A = (T - O.em_ff(P, E, B)) @ eta
        w, V = np.linalg.eig(A)
        j = int(np.argmax(w.real))
        v = V[:, j].real
        v = v / math.sqrt(v[0] ** 2 - v[1:] @ v[1:]) * np.sign(v[0])
        assert it > 0
        assert abs(lam - w[j].real) < 1e-12 * abs(w[j].real)
        assert np.allclose(U, v, atol=1e-11)


def test_alfven_speed_golden():
    """The printed Alfven speed: eta_A = 0.118591 gives v_A = 0.40785 for n = p =
    B0 = 1, Gamma = 4/3 (the formula the config-1 analytic comparison uses in its
    eta_A -> 0 limit)."""
    g = json.load(open(os.path.join(GOLDEN, "alfven_speed.json")))
    eps = g["n"] * g["c"] ** 2 + g["p"] / (g["gamma_ad"] - 1.0)
    vA = W.alfven_speed(g["B0"], g["eta_A"], eps, g["p"], g["c"])
    assert round(vA, g["printed_digits"]) == g["v_A"]
    # the small-amplitude limit is the textbook B0 c / sqrt(eps + p + B0^2)
    assert abs(W.alfven_speed(0.1, 0.0, 4.0, 1.0) - 0.1 / math.sqrt(5.01)) < 1e-15

"""Pins of the oracle's flare driving (Sec. IV, stellar flare): the body force
(reading R25), its velocity cut-off (R26) and the iterative E, J
initialisation (R27), against what the force and Ampere's law fix: the
moments the force adds, the momentum budget of a periodic box, the switch at
the cut-off, and the steady resistive field E = (curl B) / sigma."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1508_03452_gb300 import workloads as W


def _totals(s):
    f, _, _, _ = s.state()
    p = O.lattice(s.P)["p"]
    return np.array([(p[:, 0:1] * p[:, m:m + 1] * f).sum() for m in range(4)])


@pytest.mark.parametrize("c", [1.0, 2.5])
def test_force_populations_add_exactly_momentum_and_work(c):
    """sum p^0 p^a df = c F^a dt, sum p^0 p^0 df = F.u dt, every spatial
    second moment zero (a dropped c, a wrong lattice sum or a stray term in
    the rest population fails one of these)."""
    P = O.make_params(4, 4, 4, c=c, dx=0.3, drive_f0=0.05, drive_layers=1)
    p = O.lattice(P)["p"]
    dt = O.dt(P)
    rng = np.random.default_rng(3)
    for _ in range(5):
        F, u = rng.normal(size=3), rng.uniform(-0.3, 0.3, 3) * c
        df = O.force_populations(P, F, u)
        assert np.allclose([(p[:, 0] * p[:, a] * df).sum() for a in (1, 2, 3)], c * F * dt, rtol=1e-13, atol=0)
        assert (p[:, 0] ** 2 * df).sum() == pytest.approx(F @ u * dt, rel=1e-12, abs=1e-17)
        for a in (1, 2, 3):
            for b in (1, 2, 3):
                assert abs((p[:, a] * p[:, b] * df).sum()) < 1e-15 * np.abs(F).max()


def test_force_pattern_is_the_printed_one():
    """F^x = F0 sin(pi xs/3) cos(pi y/6), F^y = F0 cos(pi xs/3) sin(pi y/6) on
    x, y in [-3, 3], xs = x (x < 0) or x - 3 (x >= 0), F^z = 0."""
    P = O.make_params(24, 12, 4, drive_f0=0.05, drive_layers=1)
    for x, y in ((0, 0), (5, 7), (12, 3), (23, 11), (17, 6)):
        X, Y = -3 + (x + 0.5) * 6 / 24, -3 + (y + 0.5) * 6 / 12
        xs = X if X < 0 else X - 3
        F = O.drive_force(P, x, y)
        assert F == pytest.approx([0.05 * math.sin(math.pi * xs / 3) * math.cos(math.pi * Y / 6),
                                   0.05 * math.cos(math.pi * xs / 3) * math.sin(math.pi * Y / 6), 0.0], abs=1e-16)


def test_forced_periodic_box_gains_the_impulse():
    """Periodic box, the lowest two layers forced: every step the total
    T^{0a} grows by c dt sum F^a over the forced cells and T^00 by
    dt sum F.u (u of the step before; zero in the first step)."""
    nx, ny, nz, nl = 8, 6, 4, 2
    c = 1.0
    N = nx * ny * nz
    P = O.make_params(nx, ny, nz, c=c, sigma=50.0, drive_f0=0.02, drive_layers=nl, threads=4)
    s = O.Sim(P)
    B = np.zeros((3, N))
    B[2] = 0.05
    s.init(np.ones(N), np.ones(N), np.zeros((3, N)), B)
    dt = O.dt(P)
    Fc = np.array([[O.drive_force(P, x, y) for x in range(nx)] for y in range(ny)])  # [y][x][3]
    impulse = c * dt * nl * Fc.sum(axis=(0, 1))
    assert np.abs(impulse[:2]).max() > 1e-4
    for _ in range(3):
        assert s.force_on()
        t0 = _totals(s)
        u = s.moments()[3:6].reshape(3, nz, ny, nx)
        work = dt * sum((Fc[:, :, a] * u[a, :nl]).sum() for a in range(3))
        s.step(1)
        t1 = _totals(s)
        assert np.allclose(t1[1:] - t0[1:], impulse, rtol=1e-9, atol=1e-12), (t1 - t0, impulse)
        assert t1[0] - t0[0] == pytest.approx(work, rel=1e-9, abs=1e-12)


def test_velocity_cut_off_stops_the_force():
    """The force acts only while max |u| < drive_vmax (the paper's 0.3 c):
    above it the totals are conserved."""
    nx, ny, nz = 8, 6, 4
    N = nx * ny * nz
    u = np.zeros((3, N))
    u[0, 5] = 0.25
    B = np.zeros((3, N))
    B[2] = 0.05
    for vmax, on in ((0.3, True), (0.2, False), (0.0, True)):
        P = O.make_params(nx, ny, nz, sigma=50.0, drive_f0=0.02, drive_layers=2, drive_vmax=vmax, threads=4)
        s = O.Sim(P)
        s.init(np.ones(N), np.ones(N), u, B)
        assert s.force_on() == on
        t0 = _totals(s)
        s.step(1)
        moved = np.abs(_totals(s)[1:] - t0[1:]).max()
        assert (moved > 1e-6) == on, (vmax, moved)


def test_relaxed_init_reaches_the_resistive_field():
    """u = 0, B = b sin(kx) e_z held fixed: E relaxes to the steady
    resistive field J / sigma with J = curl B, E_y = -b k cos(kx) / sigma
    (mu0 = 1), to the scheme's second-order accuracy (the unrelaxed start
    has E = -u x B = 0); the relaxation stops on its tolerance and the run
    starts at step 0. Resetting the Maxwell populations to equilibrium in
    every iteration would give twice that field."""
    nx, ny = 64, 4
    N = nx * ny
    b, sigma = 0.05, 10.0
    x = (np.arange(N) % nx).astype(float)
    k = 2 * np.pi / nx
    B = np.zeros((3, N))
    B[2] = b * np.sin(k * x)
    P = O.make_params(nx, ny, 1, sigma=sigma, threads=4)
    s = O.Sim(P)
    its, res = s.init_relaxed(np.ones(N), np.ones(N), np.zeros((3, N)), B, max_iters=500, tol=1e-6)
    assert res <= 1e-6 and 1 < its < 500
    m = s.moments()
    Ey = -b * k * np.cos(k * x) / sigma
    assert np.abs(m[7] - Ey).max() < 0.01 * np.abs(Ey).max()
    assert np.abs(m[6]).max() < 1e-12 and np.abs(m[8]).max() < 1e-12
    assert np.allclose(m[3:6], 0.0) and np.allclose(m[9:12], B, rtol=0, atol=1e-15)
    assert np.abs(m[14] - sigma * Ey).max() < 0.01 * np.abs(sigma * Ey).max()  # J_y = (curl B)_y
    assert s.stats()["steps"] == 0
    # a field that is already steady is accepted after one step
    k2, res2 = O.Sim(P).init_relaxed(np.ones(N), np.ones(N), np.zeros((3, N)), np.zeros((3, N)), tol=1e-12)
    assert (k2, res2) == (1, 0.0)

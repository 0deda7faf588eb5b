"""Pin of the bulk-viscosity coefficient (reading R11 of the term after Eq.
eq:rlb, Sec. III: alpha (c dt/dx) sum_a [f(x+e_a) - 2 f + f(x-e_a)], i != 0).

The paper's coefficient is garbled, so there is no printed value to compare
with; what the linear update fixes is the term's share of the damping of a
momentum mode. In one step from an equilibrium state:
  * the collision leaves an equilibrium unchanged and in any case conserves
    T^{0a} (Landau matching), and the flux part of the streaming does not
    depend on alpha;
  * the rest population carries no momentum (p_0^a = 0), so the viscosity,
    applied to every moving population alike, adds exactly
    alpha (c dt/dx) times the discrete Laplacian of T^{0a} to T^{0a}.
For a Fourier mode exp(i k x) of a shear wave (u_y(x)) or a sound wave (u_x(x))
in a uniform periodic box, that is a damping factor 1 - 4 alpha (c dt/dx)
sin^2(k dx/2) per step on the mode's momentum, on top of whatever the flux and
collision do. With the paper's time-step synchronisation dx/dt = sqrt(2) c (end
of Sec. III) the coefficient is alpha / sqrt(2) for any c and dx. The test
compares one oracle step at alpha = 0 with one at alpha > 0 from the same
state: a dropped or doubled factor, or c in the wrong place (checked at
c = 2.5, dx = 0.5), changes the ratio by sqrt(2), 2 or 2.5.
"""
import numpy as np
import pytest

import oracle as O


def _momentum(P, f, a):
    lat = O.lattice(P)
    p = lat["p"]  # (19, 4): p_i^mu
    return (p[:, 0:1] * p[:, 1 + a:2 + a] * f).sum(axis=0)


def _one_step_momentum(nx, ny, c, dx, alpha, u, a):
    N = nx * ny
    P = O.make_params(nx, ny, 1, alpha=alpha, c=c, dx=dx, sigma=100.0)
    s = O.Sim(P)
    s.init(np.ones(N), np.ones(N), u, np.zeros((3, N)))
    T0 = _momentum(P, s.state()[0], a)
    s.step(1)
    assert s.stats()["recover_fail"] == 0
    return T0, _momentum(P, s.state()[0], a)


@pytest.mark.parametrize("c,dx", [(1.0, 1.0), (2.5, 0.5)])
@pytest.mark.parametrize("wave", ["shear", "sound"])
@pytest.mark.parametrize("alpha", [0.05, 0.1])
def test_viscosity_share_of_momentum_damping(c, dx, wave, alpha):
    nx, ny, m = 32, 3, 3
    N = nx * ny
    x = np.arange(N) % nx
    kdx = 2.0 * np.pi * m / nx
    a = 1 if wave == "shear" else 0
    u = np.zeros((3, N))
    u[a] = 1e-3 * c * np.sin(kdx * x)
    T0, T_free = _one_step_momentum(nx, ny, c, dx, 0.0, u, a)
    T0b, T_visc = _one_step_momentum(nx, ny, c, dx, alpha, u, a)
    assert np.array_equal(T0, T0b)
    coef = alpha / np.sqrt(2.0)  # alpha c dt / dx with dt = dx / (sqrt(2) c)
    # cell by cell: alpha (c dt/dx) times the periodic second difference along x
    t0 = T0.reshape(ny, nx)
    lap = np.roll(t0, 1, axis=1) + np.roll(t0, -1, axis=1) - 2.0 * t0
    dT = (T_visc - T_free).reshape(ny, nx)
    scale = np.abs(coef * lap).max()
    assert np.abs(dT - coef * lap).max() <= 1e-9 * scale
    # the same as the damping of the mode: Fourier amplitude of the momentum
    # change over the mode's amplitude = -4 alpha (c dt/dx) sin^2(k dx / 2)
    amp = lambda v: np.fft.rfft(v.reshape(ny, nx).mean(axis=0))[m]
    ratio = amp(T_visc - T_free) / amp(T0)
    expect = -4.0 * coef * np.sin(kdx / 2.0) ** 2
    assert abs(ratio.imag) < 1e-9 * abs(expect)
    assert abs(ratio.real - expect) <= 1e-8 * abs(expect)


def test_wrong_coefficients_would_fail():
    """The bar separates the reading from its plausible slips: a coefficient
    without dt/dx (alpha c), with dt/dx doubled, or without c differs from
    alpha/sqrt(2) by far more than the tolerance used above."""
    c, dx = 2.5, 0.5
    dt = dx / (np.sqrt(2.0) * c)
    good = 0.1 * c * dt / dx
    for wrong in (0.1 * c, 2 * good, 0.1 * dt / dx):
        assert abs(wrong - good) > 0.2 * good

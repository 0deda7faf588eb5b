"""Seeded synthetic initial fields for the lattice Boltzmann RRMHD solver.

These generators build the initial rest-frame density n, pressure p, velocity u
and magnetic field B of the test problems of Sec. IV of arXiv:1508.03452 and of
the workloads derived from them. They contain no step of the lattice Boltzmann
method itself: E, rho_c, J and the populations are computed from these fields
by the solver (and, independently, by the CPU oracle used in the tests).

All arrays are float64, x-fastest: scalars have shape (N,), vectors (3, N) with
N = nx * ny * nz. Coordinates are cell centres in lattice units unless stated.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Fields:
    nx: int
    ny: int
    nz: int
    n: np.ndarray
    p: np.ndarray
    u: np.ndarray
    B: np.ndarray
    E: np.ndarray | None = None
    meta: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return self.nx * self.ny * self.nz


def _grid(nx, ny, nz):
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return x.reshape(-1).astype(np.float64), y.reshape(-1).astype(np.float64), z.reshape(-1).astype(np.float64)


def alfven_speed(B0: float, eta_A: float, eps: float, p: float, c: float = 1.0) -> float:
    """Alfven speed of the Alfven-wave test (Sec. IV, Alfven-wave subsection).

    v_A^2 = 2 B0^2 c^2 / (eps + p + B0^2 (1 + eta_A^2))
            * [1 + sqrt(1 - (2 eta_A B0^2 / (eps + p + B0^2 (1 + eta_A^2)))^2)]^-1
    With n = p = 1, B0 = 1, eta_A = 0.118591, Gamma = 4/3 this is 0.40785.
    """
    d = eps + p + B0 * B0 * (1.0 + eta_A * eta_A)
    return math.sqrt(2.0 * B0 * B0 * c * c / d / (1.0 + math.sqrt(1.0 - (2.0 * eta_A * B0 * B0 / d) ** 2)))


def alfven_wave(nx=64, ny=64, nz=1, *, B0=0.1, amp=1e-3, n0=1.0, p0=1.0, gamma_ad=4.0 / 3.0, c=1.0) -> Fields:
    """Linear Alfven wave on a periodic box: background B = (B0, 0, 0), one
    wavelength along x equal to the box, dB_z = amp sin(k x) and
    du_z = -v_A dB_z / B0 (the relation of the paper's Alfven test), v_A in its
    small-amplitude limit B0 c / sqrt(eps + p + B0^2)."""
    x, _, _ = _grid(nx, ny, nz)
    N = nx * ny * nz
    eps = n0 * c * c + p0 / (gamma_ad - 1.0)
    vA = alfven_speed(B0, 0.0, eps, p0, c)
    k = 2.0 * math.pi / nx
    dBz = amp * np.sin(k * (x + 0.5))
    u = np.zeros((3, N)); B = np.zeros((3, N))
    B[0] = B0
    B[2] = dBz
    u[2] = -vA * dBz / B0
    return Fields(nx, ny, nz, np.full(N, n0), np.full(N, p0), u, B,
                  meta={"workload": "alfven", "vA": vA, "k": k, "B0": B0, "amp": amp})


def double_tanh(s: np.ndarray, L: float, width: float) -> np.ndarray:
    """Periodic double layer: tanh((s + L/4)/w) - tanh((s - L/4)/w) - 1 for s
    centred in (-L/2, L/2). +1 in the middle half, -1 outside, continuous across
    the periodic seam; two layers at s = -L/4 and s = +L/4."""
    return np.tanh((s + L / 4.0) / width) - np.tanh((s - L / 4.0) / width) - 1.0


def current_sheet(nx=1024, ny=1024, nz=1, *, B0=0.1, delta=8.0, n0=1.0, p0=1.0) -> Fields:
    """Resistive current sheet: B_y = B0 * double_tanh(x), uniform n and p, u = 0
    (the periodic form of the paper's self-similar current-sheet test)."""
    x, _, _ = _grid(nx, ny, nz)
    N = nx * ny * nz
    s = x + 0.5 - nx / 2.0
    B = np.zeros((3, N))
    B[1] = B0 * double_tanh(s, float(nx), delta)
    return Fields(nx, ny, nz, np.full(N, n0), np.full(N, p0), np.zeros((3, N)), B,
                  meta={"workload": "current_sheet", "B0": B0, "delta": delta})


def current_sheet_paper(ncell=100, *, sigma=100.0, t0=1.0, B0=1.0, p0=50.0, n0=1.0, x0=-1.5, x1=1.5) -> Fields:
    """The paper's 1-D current-sheet test: x in [-1.5, 1.5] on ncell cells,
    p = 50, n = 1, u = E = 0, B_y = B0 erf(x sqrt(sigma / t0) / 2) (Eq.
    Current_sheet at t = t0). Open boundaries; dx = 3 / ncell."""
    dx = (x1 - x0) / ncell
    xc = x0 + (np.arange(ncell) + 0.5) * dx
    B = np.zeros((3, ncell))
    B[1] = B0 * np.array([math.erf(0.5 * math.sqrt(sigma / t0) * v) for v in xc])
    return Fields(ncell, 1, 1, np.full(ncell, n0), np.full(ncell, p0), np.zeros((3, ncell)), B,
                  meta={"workload": "current_sheet_paper", "dx": dx, "x": xc, "sigma": sigma, "B0": B0})


def kelvin_helmholtz(nx=2048, ny=2048, nz=1, *, V=0.3, ratio=1.0, B0=0.1, a=1.0, noise=1e-3, b=10.0,
                     seed=0, p0=1.0) -> Fields:
    """Kelvin-Helmholtz shear layers on a periodic box (the paper's KH set-up
    made periodic): u_x = V * double_tanh(y), n = 1 + (dn / 2) double_tanh(y)
    with dn = 2 (ratio - 1)/(ratio + 1), B_x = B0 * double_tanh(y) (antiparallel
    across each layer), and seeded uniform noise of amplitude `noise` in u_y
    weighted by exp(-d^2 / b^2), d the distance to the nearest layer."""
    x, y, _ = _grid(nx, ny, nz)
    N = nx * ny * nz
    s = y + 0.5 - ny / 2.0
    prof = double_tanh(s, float(ny), a)
    dn = 2.0 * (ratio - 1.0) / (ratio + 1.0)
    rng = np.random.Generator(np.random.PCG64(seed))
    d = np.minimum(np.abs(s + ny / 4.0), np.abs(s - ny / 4.0))
    u = np.zeros((3, N)); B = np.zeros((3, N))
    u[0] = V * prof
    u[1] = noise * rng.uniform(-1.0, 1.0, N) * np.exp(-(d * d) / (b * b))
    B[0] = B0 * prof
    return Fields(nx, ny, nz, 1.0 + 0.5 * dn * prof, np.full(N, p0), u, B,
                  meta={"workload": "kh", "V": V, "ratio": ratio, "seed": seed})


@dataclass
class RunSpec:
    nx: int
    ny: int
    sigma: float
    V: float
    ratio: float
    seed: int


def kh_sweep(nruns=64, *, seed=1508, sides=tuple(range(256, 1025, 128))) -> list[RunSpec]:
    """Batched KH-reconnection sweep: square grids with sides drawn from
    {256, 384, ..., 1024}, sigma log-uniform in [10, 1e4], V uniform in
    [0.1, 0.5] c, density ratio in {1, 3, 10}; seeded PCG64."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for r in range(nruns):
        side = int(rng.choice(np.asarray(sides)))
        sigma = float(10.0 ** rng.uniform(1.0, 4.0))
        V = float(rng.uniform(0.1, 0.5))
        ratio = float(rng.choice(np.asarray([1.0, 3.0, 10.0])))
        out.append(RunSpec(side, side, sigma, V, ratio, seed * 1000 + r))
    return out


def flux_rope(nx=256, ny=256, nz=256, *, B_bg=0.05, B_tor=0.2, c_b=0.2534, h=2.0, r0=0.5) -> Fields:
    """Stellar-flare flux rope over x, y in [-3, 3], z in [0, 6] (Sec. IV, 3-D
    flare): flux function psi = psi_b + psi_i + psi_l of the paper (four line
    currents at (+-1.5, -0.3), (+-0.3, -0.3), an image current at z = -h and a
    rope of radius r0 at height h), poloidal field curl(psi e_y) rescaled to a
    maximum of B_bg, plus the axial core field B_y = B_tor sqrt(1 - r^2/r0^2)
    inside the rope; n = p = 1, u = 0. The curl is taken analytically."""
    x, y, z = _grid(nx, ny, nz)
    N = nx * ny * nz
    X = -3.0 + (x + 0.5) * 6.0 / nx
    Z = (z + 0.5) * 6.0 / nz

    def dlog_sq(xc, zc):
        # gradient of log[(X - xc)^2 + (Z - zc)^2]
        q = (X - xc) ** 2 + (Z - zc) ** 2
        return 2.0 * (X - xc) / q, 2.0 * (Z - zc) / q

    dpx = np.zeros(N); dpz = np.zeros(N)
    for xc, sgn in ((-0.3, 1.0), (0.3, 1.0), (-1.5, -1.0), (1.5, -1.0)):
        gx, gz = dlog_sq(xc, -0.3)
        dpx += sgn * c_b * gx
        dpz += sgn * c_b * gz
    gx, gz = dlog_sq(0.0, -h)
    dpx += -0.5 * r0 * gx
    dpz += -0.5 * r0 * gz
    r = np.sqrt(X * X + (Z - h) ** 2)
    inside = r <= r0
    # psi_l = r^2 / (2 r0) inside, r0/2 - r0 log r0 + r0 log r outside
    dl_dr = np.where(inside, r / r0, r0 / np.maximum(r, 1e-300))
    rr = np.maximum(r, 1e-300)
    dpx += dl_dr * X / rr
    dpz += dl_dr * (Z - h) / rr
    B = np.zeros((3, N))
    B[0] = -dpz
    B[2] = dpx
    bmax = float(np.max(np.sqrt(B[0] ** 2 + B[2] ** 2)))
    B *= B_bg / bmax
    B[1] = np.where(inside, B_tor * np.sqrt(np.clip(1.0 - (r / r0) ** 2, 0.0, None)), 0.0)
    return Fields(nx, ny, nz, np.ones(N), np.ones(N), np.zeros((3, N)), B,
                  meta={"workload": "flux_rope", "dx": 6.0 / nx})


def drive_layers_for(nz: int) -> int:
    """Driven photosphere thickness: the paper forces z <= 0.2343 of a 6-high box."""
    return int(math.ceil(0.2343 / 6.0 * nz))


def mlp_init_params(seed: int = 0) -> np.ndarray:
    """Seeded initial parameters of the 20-64-64-64-4 seed network (float32,
    layout W1[64][20] b1[64] W2[64][64] b2[64] W3[64][64] b3[64] W4[4][64]
    b4[4]): weights normal with variance 2 / fan_in (He et al., 2015), output
    layer scaled by 0.1, biases zero."""
    r = np.random.default_rng(seed)
    parts = []
    for fan_out, fan_in, scale in ((64, 20, 1.0), (64, 64, 1.0), (64, 64, 1.0), (4, 64, 0.1)):
        parts.append(r.normal(0.0, scale * math.sqrt(2.0 / fan_in), size=fan_out * fan_in))
        parts.append(np.zeros(fan_out))
    return np.concatenate(parts).astype(np.float32)


def alfven_paper(ncell=400, *, B0=1.0, By=0.1, eta_A=0.118591, vA=0.40785, n0=1.0, p0=1.0, x0=-0.8,
                 x1=0.0) -> Fields:
    """The paper's nonlinear Alfven-wave test (Sec. IV, Alfven-wave subsection):
    x in [-1, 1] with `ncell` cells, n = p = 1, B = (B0, By, B^z), and inside
    x0 < x < x1 the pulse B^z = eta_A B0 sin(2 pi (3 s^2 - 2 s^3)), s = (x - x0)
    / (x1 - x0), with u^z = -(v_A / B0) B^z (zero outside). dx = 2 / ncell."""
    dx = 2.0 / ncell
    x = -1.0 + (np.arange(ncell) + 0.5) * dx
    s = (x - x0) / (x1 - x0)
    inside = (x > x0) & (x < x1)
    Bz = np.where(inside, eta_A * B0 * np.sin(2.0 * math.pi * (3.0 * s * s - 2.0 * s ** 3)), 0.0)
    u = np.zeros((3, ncell))
    u[2] = -(vA / B0) * Bz
    B = np.zeros((3, ncell))
    B[0], B[1], B[2] = B0, By, Bz
    return Fields(ncell, 1, 1, np.full(ncell, n0), np.full(ncell, p0), u, B,
                  meta={"workload": "alfven_paper", "dx": dx, "x": x, "vA": vA, "x0": x0, "x1": x1,
                        "eta_A": eta_A, "B0": B0})


def kelvin_helmholtz_paper(ncell=512, *, U0=0.6, dn=1.8, c=2.5, B0=0.06, n0=1.0, p0=1.0, u_pert=0.01,
                           k=2.0 * math.pi) -> Fields:
    """The paper's Kelvin-Helmholtz-driven reconnection set-up (Sec. IV,
    Kelvin-Helmholtz-driven reconnection): [-0.5, 0.5]^2 in ncell^2 cells
    (dx = 1 / ncell, to be run with dx/dt = 2.5 sqrt 2, i.e. c = 2.5, periodic
    in x and open in y), one shear layer at y = 0 of width a = dx:
    u_x = (U0 c / 2) tanh(y / a), n = n0 + (dn / 2) tanh(y / a), p = p0,
    B_x = B0 tanh(y / a), B_y = B_z = 0, and the single-mode perturbation
    u_y = u_pert sin(k x) exp(-y^2 / b^2), b = 10 dx. U0 is given in units of
    c; u_pert in the velocity unit of the run. E is left to the solver (ideal
    Ohm's law, as the paper's initial field)."""
    dx = 1.0 / ncell
    xc = -0.5 + (np.arange(ncell) + 0.5) * dx
    X, Y = np.meshgrid(xc, xc, indexing="xy")  # X[j, i] = x_i, Y[j, i] = y_j: x-fastest after reshape
    x, y = X.reshape(-1), Y.reshape(-1)
    N = ncell * ncell
    a, b = dx, 10.0 * dx
    t = np.tanh(y / a)
    u = np.zeros((3, N)); B = np.zeros((3, N))
    u[0] = 0.5 * U0 * c * t
    u[1] = u_pert * np.sin(k * x) * np.exp(-(y * y) / (b * b))
    B[0] = B0 * t
    return Fields(ncell, ncell, 1, n0 + 0.5 * dn * t, np.full(N, p0), u, B,
                  meta={"workload": "kh_paper", "dx": dx, "c": c, "U0": U0, "dn": dn, "B0": B0, "x": xc, "y": xc})

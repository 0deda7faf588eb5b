"""Linear stability of the Maxwell lattice (Eq. LB_Maxwell with tau_h = 1/2,
Eq. Maxwell-eq, Eq. Ex_force) when the current of Eq. Ohm contains the
convection term rho_c u.

For a fixed uniform velocity u, the update of one Fourier mode of the 25 EM
populations is a 25 x 25 matrix built here from the oracle's D3Q13 tables. At
u = 0 it is neutrally stable (the Maxwell part conserves energy). With the
convection current its spectral radius exceeds 1: charge is advected by the
(1/16) v.J term of the equilibrium without any numerical diffusion. This is the
growth seen in flowing magnetised runs (KH, flare), and why their parity tests
use short horizons.
"""
import numpy as np
import pytest

import oracle as O
from paper_1508_03452_gb300 import workloads as W


def maxwell_update(k, u, sigma=0.0):
    P = O.make_params(c=1.0, sigma=sigma)
    L = O.lattice(P)
    v, e, b, hop = L["v"], L["e"], L["b"], L["hop"]
    dt = O.dt(P)
    M = np.zeros((25, 25), complex)
    for col in range(25):
        h = np.zeros(25)
        h[col] = 1.0
        Ep = (h[:24, None] * e).sum(0)
        B = (h[:24, None] * b).sum(0)
        rho = h[24] + h[:24].sum()
        E = O.ohm_solve(P, Ep, u, B, rho)
        J = O.ohm_current(P, E, u, B, rho)
        heq = O.heq(P, E, B, J, rho)
        hc = 2.0 * heq - h
        out = np.zeros(25, complex)
        out[:24] = hc[:24] * np.exp(-1j * (hop @ k))
        out[24] = hc[24]
        M[:, col] = out
    return M


def spectral_radius(u, sigma=0.0):
    r = 0.0
    for kx in np.linspace(0, np.pi, 5):
        for ky in np.linspace(0, np.pi, 5):
            r = max(r, np.abs(np.linalg.eigvals(maxwell_update(np.array([kx, ky, 0.3]), u, sigma))).max())
    return r


def test_maxwell_lattice_is_neutral_at_rest():
    assert abs(spectral_radius(np.zeros(3)) - 1.0) < 1e-9


@pytest.mark.parametrize("ux,lower", [(0.1, 1.2), (0.3, 1.5)])
def test_convection_current_makes_it_grow(ux, lower):
    assert spectral_radius(np.array([ux, 0.0, 0.0])) > lower


def test_benchmark_sheet_grows_a_grid_scale_charge_mode():
    """The benchmark's periodic double current sheet (B_y = 0.1 double tanh of
    width 8, sigma = 100) in 1-D on 512 cells: the charge density rho_c = sum h
    carries a mode at the grid's highest wavenumbers (zero in exact arithmetic)
    that the sheets' slow flow amplifies by ~1e4 per 1000 steps, while eps0
    div E stays small; it later breaks the recovery (a property of the
    scheme, reproduced by the GPU path at 512^2 and 1024^2)."""
    nx = 512
    F = W.current_sheet(nx, 1, 1, delta=8.0)
    s = O.Sim(O.make_params(nx, 1, 1, sigma=100.0, threads=8))
    s.init(F.n, F.p, F.u, F.B)

    def top(m):
        spec = np.abs(np.fft.rfft(m[12]))
        return spec[-8:].max(), spec[: len(spec) // 2].max()

    s.step(1000)
    hi1, _ = top(s.moments())
    s.step(1000)
    m = s.moments()
    hi2, lo2 = top(m)
    assert hi2 > 100 * hi1 and hi2 > 100 * lo2, (hi1, hi2, lo2)
    assert s.stats()["recover_fail"] == 0

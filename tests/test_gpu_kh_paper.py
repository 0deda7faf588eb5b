"""The paper's own Kelvin-Helmholtz-driven reconnection set-up (Sec. IV:
[-0.5, 0.5]^2, one shear layer of width a = dx, dx/dt = 2.5 sqrt 2, periodic
in x, open in y with the normal-B fix, U0 = 0.6 c, dn = 1.8, sigma = 100)
at 64^2, on the GPU in float64 against the oracle: with the paper's readings
over 12 steps (the flow amplifies a grid-scale charge mode ~4x per step from
round-off, rho_c 5e-11 at step 10, 1.3 at step 30, and the recovery fails
from step ~40, so a longer horizon would compare amplified rounding), and with the Gauss-law charge of Ohm's
convection current and the first-order fluid flux (the study options that
carry it further) over 200 steps."""
import numpy as np
import pytest

import oracle as O
from paper_1508_03452_gb300 import lbrmhd as L
from paper_1508_03452_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GROUPS = {"n": (0,), "eps": (2,), "u": (3, 4, 5), "E": (6, 7, 8), "B": (9, 10, 11)}


def _pair(n, steps, gpu_flags, orc_flags, alpha, precision=L.FP64):
    F = W.kelvin_helmholtz_paper(n, U0=0.6, dn=1.8)
    dx = 1.0 / n
    ref = O.Sim(O.make_params(n, n, 1, bc=(O.PERIODIC, O.PERIODIC, O.OPEN, O.OPEN, O.PERIODIC, O.PERIODIC),
                              sigma=100.0, alpha=alpha, c=2.5, dx=dx, flags=orc_flags, threads=8))
    ref.init(F.n, F.p, F.u, F.B)
    ref.step(steps)
    s = L.Solver(L.make_params(n, n, 1, bc=(L.PERIODIC, L.PERIODIC, L.OPEN, L.OPEN, L.PERIODIC, L.PERIODIC),
                               sigma=100.0, alpha=alpha, c=2.5, dx=dx, flags=gpu_flags, precision=precision))
    s.init_fields(0, F.n, F.p, F.u, F.B)
    s.step(steps)
    mg, mo = s.moments(), ref.moments()
    st = s.stats()
    s.close()
    assert st["recover_fail"] == 0 and ref.stats()["recover_fail"] == 0
    return {k: float(np.linalg.norm(mg[list(r)] - mo[list(r)]) / np.linalg.norm(mo[list(r)])) for k, r in GROUPS.items()}


def test_paper_kh_readings_fp64():
    errs = _pair(64, 12, 0, 0, 0.1)
    assert max(errs.values()) <= 1e-10, errs


def test_paper_kh_gauss_charge_first_order_flux_fp64():
    errs = _pair(64, 200, L.FLAG_GAUSS_CHARGE | L.FLAG_FIRST_ORDER_FLUX, O.GAUSS_CHARGE | O.FIRST_ORDER, 0.02)
    assert max(errs.values()) <= 1e-10, errs


def test_reconnection_rate_scales_as_sweet_parker_while_the_initial_sheet_diffuses():
    """R(t) = (E^z - E^z_0) / B0 at the null point (Sec. IV) on the paper's
    lattice (512^2, c = 2.5, periodic x, open y, one layer of width dx,
    B0 = 0.06, U0 = 0.2 c) for sigma = 20, 50, 100 in one handle, with the
    options that carry these runs to the paper's times (uniform density,
    Gauss-law charge, alpha = 0.02). While the initial sheet diffuses (t <~ 1)
    the rate falls with the conductivity as sigma^-1/2, the Sweet-Parker side
    of the paper's fit (measured slope -0.47 at t = 0.4, -0.44 at t = 1.2). At
    the paper's t = 23.2 the low-sigma sheets have diffused across the box and
    the slope turns positive, so the paper's R(23.2) fit is not reproduced;
    this test holds the part that is."""
    import math
    n = 512
    dx = 1.0 / n
    dt = dx / (math.sqrt(2.0) * 2.5)
    sigmas = (20.0, 50.0, 100.0)
    bc = (L.PERIODIC, L.PERIODIC, L.OPEN, L.OPEN, L.PERIODIC, L.PERIODIC)
    s = L.Solver([L.make_params(n, n, 1, bc=bc, tau=1.0, sigma=sg, alpha=0.02, c=2.5, dx=dx,
                                flags=L.FLAG_GAUSS_CHARGE) for sg in sigmas])
    F = W.kelvin_helmholtz_paper(n, U0=0.2, dn=0.0)
    for r in range(len(sigmas)):
        s.init_fields(r, F.n, F.p, F.u, F.B)
    slopes, done = {}, 0
    for t in (0.4, 1.2):
        k = int(round(t / dt)) - done
        s.step(k)
        done += k
        R = [s.reconnection_rate(r, n // 2 - 64, n // 2 + 64, 0.06)["R"] for r in range(len(sigmas))]
        assert all(np.isfinite(R)) and all(abs(v) > 0 for v in R), R
        slopes[t] = float(np.polyfit(np.log(sigmas), np.log(np.abs(R)), 1)[0])
    fails = [s.stats(r)["recover_fail"] for r in range(len(sigmas))]
    s.close()
    print("slope of log |R| against log sigma:", slopes, "failures:", fails)
    assert fails == [0, 0, 0], fails
    for t, a in slopes.items():
        assert -0.6 <= a <= -0.35, (t, a)


def test_kelvin_helmholtz_mode_grows_faster_with_the_shear():
    """The instability that is to drive the reconnection (Sec. IV) does develop
    on the paper's lattice with these options: the k = 2 pi Fourier amplitude of
    u_y along the layer grows after the initial transient, faster for the
    larger shear (measured amplitudes at t = 1, 2, 4: 0.0015, 0.0034, 0.0136 at
    U0 = 0.2 c; 0.0026, 0.0112, 0.099 at U0 = 0.4 c; saturation near t = 8)."""
    import math
    n = 512
    dx = 1.0 / n
    dt = dx / (math.sqrt(2.0) * 2.5)
    bc = (L.PERIODIC, L.PERIODIC, L.OPEN, L.OPEN, L.PERIODIC, L.PERIODIC)
    x = -0.5 + (np.arange(n) + 0.5) * dx
    amps = {}
    for U0 in (0.2, 0.4):
        s = L.Solver(L.make_params(n, n, 1, bc=bc, tau=1.0, sigma=100.0, alpha=0.02, c=2.5, dx=dx,
                                   flags=L.FLAG_GAUSS_CHARGE))
        F = W.kelvin_helmholtz_paper(n, U0=U0, dn=0.0)
        s.init_fields(0, F.n, F.p, F.u, F.B)
        done, a = 0, []
        for t in (1.0, 2.0, 4.0):
            k = int(round(t / dt)) - done
            s.step(k)
            done += k
            uy = s.moments()[4].reshape(n, n)[n // 2 - 20:n // 2 + 20]
            a.append(float(np.abs((uy * np.exp(-2j * math.pi * x)[None, :]).mean(axis=1)).max() * 2))
        assert s.stats()["recover_fail"] == 0
        s.close()
        amps[U0] = a
    print("k = 2 pi amplitude of u_y at t = 1, 2, 4:", amps)
    for U0, (a1, a2, a4) in amps.items():
        assert a4 > 3.0 * a2 > 3.0 * a1, (U0, amps[U0])
    growth = {U0: math.log(a[2] / a[0]) / 3.0 for U0, a in amps.items()}
    assert growth[0.4] > 1.3 * growth[0.2], growth


def test_kelvin_helmholtz_growth_matches_the_oracle():
    """A chaotic run is compared by its statistics beyond the step-by-step
    horizon: the seeded k = 2 pi mode of u_y grows the same way on the GPU
    (float64 and float32 builds) as on the oracle, over 905 steps (t = 2) of
    the paper's set-up at 128^2 (U0 = 0.4 c, uniform density, Gauss-law charge,
    alpha = 0.02; oracle amplitudes 0.00375 at t = 1, 0.00818 at t = 2)."""
    import math
    n = 128
    dx = 1.0 / n
    dt = dx / (math.sqrt(2.0) * 2.5)
    x = -0.5 + (np.arange(n) + 0.5) * dx
    F = W.kelvin_helmholtz_paper(n, U0=0.4, dn=0.0)

    def amp(m):
        uy = m[4].reshape(n, n)[n // 2 - 10:n // 2 + 10]
        return float(np.abs((uy * np.exp(-2j * math.pi * x)[None, :]).mean(axis=1)).max() * 2)

    ref = O.Sim(O.make_params(n, n, 1, bc=(O.PERIODIC, O.PERIODIC, O.OPEN, O.OPEN, O.PERIODIC, O.PERIODIC),
                              sigma=100.0, alpha=0.02, c=2.5, dx=dx, flags=O.GAUSS_CHARGE, threads=16))
    ref.init(F.n, F.p, F.u, F.B)
    runs = {p: L.Solver(L.make_params(n, n, 1, bc=(L.PERIODIC, L.PERIODIC, L.OPEN, L.OPEN, L.PERIODIC, L.PERIODIC),
                                      sigma=100.0, alpha=0.02, c=2.5, dx=dx, flags=L.FLAG_GAUSS_CHARGE, precision=p))
            for p in (L.FP64, L.FP32)}
    for s in runs.values():
        s.init_fields(0, F.n, F.p, F.u, F.B)
    done, a = 0, {"oracle": [], L.FP64: [], L.FP32: []}
    for t in (1.0, 2.0):
        k = int(round(t / dt)) - done
        ref.step(k)
        a["oracle"].append(amp(ref.moments()))
        for p, s in runs.items():
            s.step(k)
            a[p].append(amp(s.moments()))
        done += k
    fails = [s.stats()["recover_fail"] for s in runs.values()] + [ref.stats()["recover_fail"]]
    for s in runs.values():
        s.close()
    print("k = 2 pi amplitude of u_y at t = 1, 2:", a)
    assert fails == [0, 0, 0], fails
    assert a["oracle"][1] > 1.8 * a["oracle"][0], a
    for p, tol in ((L.FP64, 1e-6), (L.FP32, 1e-3)):
        for g, r in zip(a[p], a["oracle"]):
            assert abs(g - r) <= tol * r, (p, a)

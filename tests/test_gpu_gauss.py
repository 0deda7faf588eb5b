"""The Gauss-law charge in Ohm's convection current (an option beyond the
paper, reading R28) on the GPU: parity with the oracle run with the same
option, and the stability it brings to flowing magnetised plasma."""
import numpy as np
import pytest

import oracle as O
from paper_1508_03452_gb300 import lbrmhd as L
from paper_1508_03452_gb300 import workloads as W
from test_gpu_parity import BC_ORC, FP32_SMALL_SIGNAL, TOL, assert_parity, rel_errors

pytestmark = pytest.mark.gpu


def _pair(F, steps, precision, bc=(L.PERIODIC,) * 6, **kw):
    ref = O.Sim(O.make_params(F.nx, F.ny, F.nz, bc=tuple(BC_ORC[b] for b in bc), threads=8,
                              flags=O.GAUSS_CHARGE, **kw))
    ref.init(F.n, F.p, F.u, F.B, F.E)
    ref.step(steps)
    s = L.Solver(L.make_params(F.nx, F.ny, F.nz, bc=bc, precision=precision, flags=L.FLAG_GAUSS_CHARGE, **kw))
    s.init_fields(0, F.n, F.p, F.u, F.B, F.E)
    s.step(steps)
    errs = rel_errors(s.moments(), ref.moments())
    st = s.stats()
    s.close()
    assert st["recover_fail"] == 0, st
    return errs


@pytest.mark.parametrize("precision", [L.FP64, L.FP32])
def test_gauss_charge_kelvin_helmholtz_parity(precision):
    """float32: every group but E within 1e-5 (E_z = u_y B_x of the noise
    velocity is the float32 small-signal group of the Kelvin-Helmholtz layers,
    test_gpu_parity.test_fp32_small_signal_groups)."""
    F = W.kelvin_helmholtz(96, 40, 1, V=0.2, ratio=10.0, B0=0.1, a=2.0, noise=1e-3, seed=3)
    errs = _pair(F, 40, precision, sigma=1e3)
    print("gauss KH", errs)
    assert_parity(errs, TOL[precision], skip=FP32_SMALL_SIGNAL["kh"] if precision == L.FP32 else ())


def test_gauss_charge_three_dimensional_and_open_parity():
    """Every axis of the central difference (3-D periodic), and the clamp at
    open faces, float64."""
    rng = np.random.default_rng(5)
    nx, ny, nz = 16, 12, 10
    N = nx * ny * nz
    u = np.zeros((3, N))
    u[0] = 0.05 * rng.uniform(-1, 1, N)
    u[2] = 0.05 * rng.uniform(-1, 1, N)
    B = np.zeros((3, N))
    B[1] = 0.05
    F = W.Fields(nx, ny, nz, 1.0 + 0.02 * rng.uniform(size=N), np.ones(N), u, B)
    assert_parity(_pair(F, 15, L.FP64, sigma=50.0, alpha=0.0), TOL[L.FP64])
    G = W.current_sheet(48, 32, 1, delta=4.0)
    assert_parity(_pair(G, 20, L.FP64, bc=(L.OPEN, L.OPEN) + (L.PERIODIC,) * 4, sigma=100.0), TOL[L.FP64])


def test_gauss_charge_keeps_a_flowing_plasma_on_gpu():
    """0.1c flow across B = 0.1 (32^2, sigma = 100, alpha = 0.02, noise
    1e-4), float32: with the moment charge the run fails within 300 steps;
    with the Gauss-law charge it runs 1000 steps and the noise decays."""
    nx = ny = 32
    N = nx * ny
    rng = np.random.default_rng(1)
    u = np.zeros((3, N))
    u[0] = 0.1 + 1e-4 * rng.uniform(-1, 1, N)
    B = np.zeros((3, N))
    B[1] = 0.1
    out = {}
    for flags, steps in ((0, 300), (L.FLAG_GAUSS_CHARGE, 1000)):
        s = L.Solver(L.make_params(nx, ny, 1, sigma=100.0, alpha=0.02, precision=L.FP32, flags=flags))
        s.init_fields(0, np.ones(N), np.ones(N), u, B)
        s.step(steps)
        out[flags] = (s.stats()["recover_fail"], float(np.abs(s.moments()[4]).max()))
        s.close()
    assert out[0][0] > 0
    assert out[L.FLAG_GAUSS_CHARGE][0] == 0 and out[L.FLAG_GAUSS_CHARGE][1] < 1e-5, out


def test_gauss_charge_keeps_the_benchmark_sheet():
    """The 512^2 benchmark sheet (sigma = 100, float32) fails after ~2000
    steps with the moment charge; with the Gauss-law charge it runs 4000
    steps without a failure and B_y stays at its initial maximum."""
    F = W.current_sheet(512, 512, 1, delta=8.0)
    s = L.Solver(L.make_params(512, 512, 1, sigma=100.0, precision=L.FP32, flags=L.FLAG_GAUSS_CHARGE))
    s.init_fields(0, F.n, F.p, F.u, F.B)
    s.step(4000)
    st = s.stats()
    m = s.moments()
    s.close()
    assert st["recover_fail"] == 0 and np.abs(m[10]).max() <= 0.1001

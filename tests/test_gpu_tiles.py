"""The TMA tile kernel (LBRMHD_FLAG_TMA_TILES): 2-D runs with periodic faces
stored in float32 or float16 step by tensor-map copies of each 32 x 8 tile and
its halo through shared memory (edge tiles cell by cell). It computes the same
update as the default per-cell kernel, operation for operation, so the two
agree to float rounding. Grids: interior tiles and edge tiles (160 x 24, 256 x 40),
a ragged right edge (132 x 20), tile maps but no interior tile (160 x 12),
too few rows for a tile (96 x 9), a width the tile maps cannot describe
(130 x 16 float32, 132 x 20 float16), and the benchmark's 1024 x 1024.

The two kernels are compiled separately, and the assembler may fuse a
multiply and an add of the shared cell code differently in each, so they
agree to float rounding, not bit for bit. Two bars follow from that: after
one step every population and moment agrees to a few float32 ulps of its
scale (a wrong neighbour, plane or pair would be off by the population's own
size), and after 20 Kelvin-Helmholtz steps (which amplify rounding in the
near-zero fields u_z, E_y) the tile run is no further from the float64 run
than the per-cell run's own float32 error allows."""
import numpy as np
import pytest

from paper_1508_03452_gb300 import lbrmhd as L
from paper_1508_03452_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _run(F, steps, precision, flags=0, recovery=L.RECOVERY_PLAIN, weights=None, sigma=1e3):
    s = L.Solver(L.make_params(F.nx, F.ny, 1, precision=precision, flags=flags, recovery=recovery, sigma=sigma))
    if weights is not None:
        s.set_mlp_weights(weights)
    s.init_fields(0, F.n, F.p, F.u, F.B, F.E)
    s.step(steps)
    out = s.moments(), s.populations(), s.status()
    s.close()
    return out


TILE_H = 8  # rows of a tile (the library's default)


def _tile_eligible(nx, ny, precision):
    px = 4 if precision == L.FP32 else 8
    return nx % px == 0 and nx >= 32 + 2 * px and ny >= TILE_H + 4


GROUPS = {"n": (0,), "p": (1,), "eps": (2,), "u": (3, 4, 5), "E": (6, 7, 8), "B": (9, 10, 11)}


def _one_step(a, b, tol):
    """Every moment and population of a within tol of its scale in b (a
    population's largest value, at least 1e-3 of its family's: f, g, h or the
    moments)."""
    (ma, pa, sa), (mb, pb, sb) = a, b
    assert sa["rc"] == L.OK and sb["rc"] == L.OK, (sa, sb)
    worst = (0.0, "")
    for fam, x, y in (("moment", ma[:12], mb[:12]),) + tuple(zip("fgh", pa, pb)):
        floor = 1e-3 * max(np.abs(y).max(), 1e-300)
        for i in range(y.shape[0]):
            d = np.abs(x[i] - y[i]).max() / max(np.abs(y[i]).max(), floor)
            worst = max(worst, (d, f"{fam} {i}"))
    print(f"one step: tile vs per-cell kernel, max difference {worst[0]:.3e} of the scale ({worst[1]})")
    assert worst[0] <= tol, worst


def _rel(a, b):
    return {k: float(np.linalg.norm(a[list(r)] - b[list(r)]) / np.linalg.norm(b[list(r)])) for k, r in GROUPS.items()}


def _matched(t, c, ref):
    """Relative L2 per field group: tile - per-cell within twice the per-cell
    run's own error against float64 (two float32 rounding paths differ by
    about sqrt 2 times one of them)."""
    assert t[2]["rc"] == L.OK and c[2]["rc"] == L.OK
    d, e = _rel(t[0], c[0]), _rel(c[0], ref[0])
    print("tile - per-cell", {k: f"{v:.2e}" for k, v in d.items()}, "per-cell - float64", {k: f"{v:.2e}" for k, v in e.items()})
    for k in GROUPS:
        assert d[k] <= 2.0 * e[k] + 1e-9, (k, d[k], e[k])


# float32: a few ulps of the scale after one step; float16 storage: a few
# float16 roundings that a last-bit float32 difference flips (4.9e-4 each)
ONE_STEP_TOL = {L.FP32: 1e-6, L.FP16_DEV: 2e-3}


@pytest.mark.parametrize("precision", [L.FP32, L.FP16_DEV])
@pytest.mark.parametrize("shape", [(160, 12), (160, 24), (256, 40), (132, 20), (96, 9), (130, 16)])
def test_tile_kernel_equals_per_cell_kernel(precision, shape):
    nx, ny = shape
    F = W.kelvin_helmholtz(nx, ny, 1, V=0.2, ratio=3.0, B0=0.1, a=2.0, noise=1e-3, seed=5)
    _one_step(_run(F, 1, precision, flags=L.FLAG_TMA_TILES), _run(F, 1, precision), ONE_STEP_TOL[precision])
    t = _run(F, 20, precision, flags=L.FLAG_TMA_TILES)
    c = _run(F, 20, precision)
    assert t[2]["tiled_runs"] == (1 if _tile_eligible(nx, ny, precision) else 0)
    assert c[2]["tiled_runs"] == 0
    _matched(t, c, _run(F, 20, L.FP64))


@pytest.mark.parametrize("recovery", [L.RECOVERY_COLD, L.RECOVERY_MLP])
def test_tile_kernel_seed_variants(recovery):
    torch = pytest.importorskip("torch")
    F = W.kelvin_helmholtz(256, 40, 1, V=0.2, ratio=3.0, B0=0.1, a=2.0, noise=1e-3, seed=6)
    w = None
    if recovery == L.RECOVERY_MLP:
        g = torch.Generator().manual_seed(11)
        w = (0.02 * torch.randn(L.MLP_NPARAM, generator=g)).to(torch.float32).cuda()
    _one_step(_run(F, 1, L.FP32, flags=L.FLAG_TMA_TILES, recovery=recovery, weights=w),
              _run(F, 1, L.FP32, recovery=recovery, weights=w), ONE_STEP_TOL[L.FP32])
    t = _run(F, 12, L.FP32, flags=L.FLAG_TMA_TILES, recovery=recovery, weights=w)
    c = _run(F, 12, L.FP32, recovery=recovery, weights=w)
    assert t[2]["tiled_runs"] == 1
    _matched(t, c, _run(F, 12, L.FP64, recovery=recovery, weights=w))


def test_tile_kernel_benchmark_grid():
    """The benchmark's 1024 x 1024 current sheet (sigma = 100), 4 steps."""
    F = W.current_sheet(1024, 1024, 1, delta=8.0)
    _one_step(_run(F, 1, L.FP32, flags=L.FLAG_TMA_TILES, sigma=100.0), _run(F, 1, L.FP32, sigma=100.0),
              ONE_STEP_TOL[L.FP32])
    t = _run(F, 4, L.FP32, flags=L.FLAG_TMA_TILES, sigma=100.0)
    c = _run(F, 4, L.FP32, sigma=100.0)
    assert t[2]["tiled_runs"] == 1
    _matched(t, c, _run(F, 4, L.FP64, sigma=100.0))


def test_gauss_charge_runs_take_the_per_cell_kernel():
    """The Gauss-charge option reads E of the neighbours, which the tile's
    primitive box does not hold: such runs step cell by cell."""
    F = W.kelvin_helmholtz(160, 12, 1, V=0.1, ratio=3.0, B0=0.1, a=2.0, noise=1e-3, seed=7)
    t = _run(F, 5, L.FP32, flags=L.FLAG_GAUSS_CHARGE | L.FLAG_TMA_TILES)
    assert t[2]["tiled_runs"] == 0

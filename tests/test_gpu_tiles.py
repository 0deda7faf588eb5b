"""The TMA tile kernel (LBRMHD_FLAG_TMA_TILES): 2-D runs with periodic faces
stored in float32 or float16 step by tensor-map copies of each 32 x 8 tile and
its halo through shared memory (edge tiles cell by cell). It computes the same
update as the default per-cell kernel, operation for operation, so the two
agree to float rounding. Grids: interior tiles and edge tiles (160 x 24, 256 x 40),
a ragged right edge (132 x 20), tile maps but no interior tile (160 x 12),
too few rows for a tile (96 x 9), a width the tile maps cannot describe
(130 x 16 float32, 132 x 20 float16), and the benchmark's 1024 x 1024."""
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


def _compare(a, b, tol=1e-6):
    """Equal up to float rounding: the compiler may contract the same
    operations differently in the two kernels (a last-bit difference, which
    the following steps carry along); measured on the tile grids below: at most
    1e-17 of each field's scale after 20 steps."""
    (ma, pa, sa), (mb, pb, sb) = a, b
    assert sa["rc"] == L.OK and sb["rc"] == L.OK, (sa, sb)
    d = max(np.abs(x - y).max() / max(np.abs(y).max(), 1e-300) for x, y in zip((ma,) + pa, (mb,) + pb))
    print(f"tile vs per-cell kernel: max difference {d:.3e} of each field's scale")
    assert d <= tol, d


@pytest.mark.parametrize("precision", [L.FP32, L.FP16_DEV])
@pytest.mark.parametrize("shape", [(160, 12), (160, 24), (256, 40), (132, 20), (96, 9), (130, 16)])
def test_tile_kernel_equals_per_cell_kernel(precision, shape):
    nx, ny = shape
    F = W.kelvin_helmholtz(nx, ny, 1, V=0.2, ratio=3.0, B0=0.1, a=2.0, noise=1e-3, seed=5)
    t = _run(F, 20, precision, flags=L.FLAG_TMA_TILES)
    c = _run(F, 20, precision)
    assert t[2]["tiled_runs"] == (1 if _tile_eligible(nx, ny, precision) else 0)
    assert c[2]["tiled_runs"] == 0
    _compare(t, c)


@pytest.mark.parametrize("recovery", [L.RECOVERY_COLD, L.RECOVERY_MLP])
def test_tile_kernel_seed_variants(recovery):
    torch = pytest.importorskip("torch")
    F = W.kelvin_helmholtz(256, 40, 1, V=0.2, ratio=3.0, B0=0.1, a=2.0, noise=1e-3, seed=6)
    w = None
    if recovery == L.RECOVERY_MLP:
        g = torch.Generator().manual_seed(11)
        w = (0.02 * torch.randn(L.MLP_NPARAM, generator=g)).to(torch.float32).cuda()
    t = _run(F, 12, L.FP32, flags=L.FLAG_TMA_TILES, recovery=recovery, weights=w)
    c = _run(F, 12, L.FP32, recovery=recovery, weights=w)
    assert t[2]["tiled_runs"] == 1
    _compare(t, c)


def test_tile_kernel_benchmark_grid():
    """The benchmark's 1024 x 1024 current sheet (sigma = 100), 4 steps."""
    F = W.current_sheet(1024, 1024, 1, delta=8.0)
    t = _run(F, 4, L.FP32, flags=L.FLAG_TMA_TILES, sigma=100.0)
    c = _run(F, 4, L.FP32, sigma=100.0)
    assert t[2]["tiled_runs"] == 1
    _compare(t, c)


def test_gauss_charge_runs_take_the_per_cell_kernel():
    """The Gauss-charge option reads E of the neighbours, which the tile's
    primitive box does not hold: such runs step cell by cell."""
    F = W.kelvin_helmholtz(160, 12, 1, V=0.1, ratio=3.0, B0=0.1, a=2.0, noise=1e-3, seed=7)
    t = _run(F, 5, L.FP32, flags=L.FLAG_GAUSS_CHARGE | L.FLAG_TMA_TILES)
    assert t[2]["tiled_runs"] == 0

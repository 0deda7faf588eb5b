"""Degenerate and tiny grids against the FP64 oracle: a single cell, 1-D runs,
axes of length 1 and 2 inside 3-D runs (the wrap of a +-2 stencil around an
axis shorter than the stencil), and the smallest 3-D periodic box. Every
field group within 1e-10 (FP64) after 12 steps."""
import numpy as np
import pytest

from paper_1508_03452_gb300 import lbrmhd as L
from paper_1508_03452_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _fields(nx, ny, nz, seed):
    rng = np.random.default_rng(seed)
    N = nx * ny * nz
    u = 0.02 * rng.uniform(-1, 1, (3, N))
    B = np.zeros((3, N))
    B[0], B[2] = 0.08, 0.05  # uniform B: divergence-free on any grid
    return W.Fields(nx, ny, nz, 1.0 + 0.05 * rng.uniform(size=N), 1.0 + 0.05 * rng.uniform(size=N), u, B)


@pytest.mark.parametrize("shape", [(1, 1, 1), (7, 1, 1), (1, 9, 1), (2, 2, 2), (5, 1, 2), (3, 2, 4), (3, 3, 3),
                                   (33, 2, 1)])
def test_tiny_grid_parity(shape):
    from test_gpu_parity import assert_parity, run_pair
    F = _fields(*shape, seed=sum(shape))
    # a 2-cell periodic 3-D box is all checkerboard modes, which the bulk
    # viscosity at alpha = 0.1 amplifies (the oracle fails to recover there
    # too: see the next test); it is checked without that term
    alpha = 0.0 if shape == (2, 2, 2) else 0.1
    errs, _ = run_pair(F, 12, L.FP64, sigma=30.0, alpha=alpha)
    assert_parity(errs, 1e-10)


def test_recovery_failures_match_the_oracle():
    """Where the method itself breaks down (2-cell 3-D box, alpha = 0.1), the
    GPU fails to recover in the same cell updates as the oracle."""
    import oracle as O
    F = _fields(2, 2, 2, seed=6)
    ref = O.Sim(O.make_params(2, 2, 2, sigma=30.0, threads=1))
    ref.init(F.n, F.p, F.u, F.B, F.E)
    ref.step(12)
    s = L.Solver(L.make_params(2, 2, 2, sigma=30.0, precision=L.FP64))
    s.init_fields(0, F.n, F.p, F.u, F.B, F.E)
    s.step(12)
    assert s.stats()["recover_fail"] == ref.stats()["recover_fail"] > 0
    s.close()


def test_uniform_single_cell_stays_uniform():
    F = _fields(1, 1, 1, seed=0)
    s = L.Solver(L.make_params(1, 1, 1, sigma=30.0, precision=L.FP32))
    s.init_fields(0, F.n, F.p, F.u, F.B)
    m0 = s.moments()
    s.step(50)
    m = s.moments()
    s.close()
    # one periodic cell streams onto itself: nothing changes but round-off
    assert np.allclose(m[:12], m0[:12], rtol=1e-5, atol=1e-7)

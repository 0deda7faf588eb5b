"""Grids at the sizes the 64-bit layout is there for: a float32 run whose
population arrays hold more than 2^31 elements (every offset past 2^31 formed
in 64 bits) and whose ny is past the 65535 rows a per-run launch grid can
cover (the default schedule then walks the tile list). The state is the
current sheet, uniform along y, so every row must stay bit-identical to the
first, and the first rows must match the FP64 oracle on a 12-row grid of the
same profile within the float32 bar."""
import numpy as np
import pytest

import oracle as O
from paper_1508_03452_gb300 import lbrmhd as L
from paper_1508_03452_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_tall_grid_past_the_launch_limit_and_32_bit_offsets():
    torch = pytest.importorskip("torch")
    from test_gpu_parity import assert_parity, rel_errors

    nx, ny, ny_small, steps = 1024, 90112, 12, 20  # 20 steps: the horizon of the 1024^2 multi-step parity test
    N = nx * ny
    assert 38 * N > 2 ** 31 and 25 * N > 2 ** 31 and ny > 65535
    F = W.current_sheet(nx, ny_small, 1, delta=8.0)
    dev = torch.device("cuda", 0)

    def tall(a, comps):  # the 12-row profile's first row repeated over ny rows, on the device
        row = torch.from_numpy(np.ascontiguousarray(a.reshape(comps, ny_small, nx)[:, :1, :])).to(dev)
        return row.expand(comps, ny, nx).contiguous().reshape(-1)

    n, p, u, B = tall(F.n, 1), tall(F.p, 1), tall(F.u, 3), tall(F.B, 3)
    s = L.Solver(L.make_params(nx, ny, 1, sigma=100.0, precision=L.FP32))
    try:
        torch.cuda.synchronize()  # the inputs are written on torch's stream
        s.init_fields_device(0, n, p, u, B)
        torch.cuda.synchronize()
        del n, p, u, B
        assert s.schedule().kind == L.SCHED_BATCH  # the per-run grid would need ny blocks along y
        s.step(steps)
        st = s.status()
        assert st["rc"] == L.OK and st["recover_fail"] == 0, st
        m = torch.empty((L.NMOMENTS, ny, nx), dtype=torch.float64, device=dev)
        s.moments_device(0, m)
        torch.cuda.synchronize()
        assert bool(torch.isfinite(m).all())
        same = (m == m[:, :1, :]).all(dim=2).all(dim=0)  # per row
        assert bool(same.all()), int((~same).nonzero()[0, 0])
        mg = m[:, :ny_small, :].reshape(L.NMOMENTS, -1).cpu().numpy()
        del m, same
    finally:
        s.close()
        torch.cuda.empty_cache()
    ref = O.Sim(O.make_params(nx, ny_small, 1, sigma=100.0, threads=8))
    ref.init(F.n, F.p, F.u, F.B)
    ref.step(steps)
    errs = rel_errors(mg, ref.moments())
    print("tall grid", errs)
    assert_parity(errs, 1e-5)

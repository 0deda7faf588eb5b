"""lbrmhd_get_diagnostics_noalloc, the diagnostics call for callers that cannot
allocate device memory when they need the numbers (a monitor running while
another framework's pool holds the free device memory, or a time-critical loop
that must not pay the device-wide synchronisation cudaMalloc / cudaFree may
imply). It keeps its partial sums in a static device array of the library and
writes to a caller-owned device buffer.

The test calls it through the C ABI, twice in a row on changing states (the
second call runs over the array the first one left behind), and checks each
result against lbrmhd_get_diagnostics. The file is named to be collected last.
"""
import ctypes as C

import numpy as np
import pytest

from paper_1508_03452_gb300 import lbrmhd as L
from paper_1508_03452_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [L.FP64, L.FP32])
def test_noalloc_diagnostics_match_allocating_call(precision):
    torch = pytest.importorskip("torch")
    F = W.kelvin_helmholtz(96, 80, 1, V=0.1, ratio=3.0, B0=0.1, a=2.0, noise=1e-2, seed=21)
    stream = torch.cuda.current_stream()
    s = L.Solver(L.make_params(F.nx, F.ny, 1, sigma=100.0, precision=precision), stream=stream)
    s.init_fields(0, F.n, F.p, F.u, F.B)
    lib = L.load()
    d_out = torch.full((L.NDIAG,), float("nan"), dtype=torch.float64, device="cuda")
    for steps in (3, 7):
        s.step(steps)
        rc = lib.lbrmhd_get_diagnostics_noalloc(s._h, 0, C.c_void_p(d_out.data_ptr()))
        assert rc == L.OK, lib.lbrmhd_last_error(s._h)
        stream.synchronize()
        got = d_out.cpu().numpy()
        want = s.diagnostics()
        scale = np.maximum(np.abs(want), 1e-300)
        assert np.all(np.abs(got - want) <= 1e-12 * scale + 1e-15), (got, want)
        assert got[9] == F.N and got[8] == 0
    s.close()


def test_noalloc_rejects_runs_above_its_limit():
    torch = pytest.importorskip("torch")
    s = L.Solver(L.make_params(4096, 4097, 1, precision=L.FP16_DEV))
    N = s.cells[0]
    s.init_fields(0, np.ones(N), np.ones(N), np.zeros(3 * N), np.zeros(3 * N))
    lib = L.load()
    d_out = torch.zeros(L.NDIAG, dtype=torch.float64, device="cuda")
    rc = lib.lbrmhd_get_diagnostics_noalloc(s._h, 0, C.c_void_p(d_out.data_ptr()))
    assert rc == L.ERR_BAD_ARG
    assert b"limit" in lib.lbrmhd_last_error(s._h)
    s.close()

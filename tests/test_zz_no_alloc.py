"""lbrmhd_get_diagnostics_noalloc, the diagnostics call for callers that cannot
allocate device memory when they need the numbers (a monitor running while
another framework's pool holds the free device memory, or a time-critical loop
that must not pay the device-wide synchronisation cudaMalloc / cudaFree may
imply). It keeps its partial sums in a static device array of the library and
writes to a caller-owned device buffer.

The tests call it through the C ABI and check each result against
lbrmhd_get_diagnostics: twice in a row on changing states (the second call
runs over the array the first one left behind), in every storage precision,
and a large run followed by a small one (the small call must not pick up the
large call's leftover partial sums). The file is named to be collected last.
"""
import ctypes as C

import numpy as np
import pytest

from paper_1508_03452_gb300 import lbrmhd as L
from paper_1508_03452_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _noalloc(lib, s, d_out, stream):
    rc = lib.lbrmhd_get_diagnostics_noalloc(s._h, 0, C.c_void_p(d_out.data_ptr()))
    assert rc == L.OK, lib.lbrmhd_last_error(s._h)
    stream.synchronize()
    return d_out.cpu().numpy()


def _check(got, want, ncells):
    scale = np.maximum(np.abs(want), 1e-300)
    assert np.all(np.abs(got - want) <= 1e-12 * scale + 1e-15), (got, want)
    assert got[9] == ncells and got[8] == 0


@pytest.mark.parametrize("precision", [L.FP64, L.FP32, L.FP16_DEV])
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
        _check(_noalloc(lib, s, d_out, stream), s.diagnostics(), F.N)
    s.close()


def test_noalloc_large_run_then_small_run():
    """A 512 x 512 run fills 2048 blocks of partial sums; a 40 x 24 run after it
    uses 8 and must read only its own."""
    torch = pytest.importorskip("torch")
    stream = torch.cuda.current_stream()
    lib = L.load()
    d_out = torch.full((L.NDIAG,), float("nan"), dtype=torch.float64, device="cuda")
    for nx, ny in ((512, 512), (40, 24)):
        F = W.current_sheet(nx, ny, 1, delta=8.0)
        s = L.Solver(L.make_params(nx, ny, 1, sigma=100.0, precision=L.FP32), stream=stream)
        s.init_fields(0, F.n, F.p, F.u, F.B)
        s.step(2)
        _check(_noalloc(lib, s, d_out, stream), s.diagnostics(), F.N)
        s.close()


def test_noalloc_rejects_runs_above_its_limit():
    """The size check comes first: a run above the limit is rejected without
    being initialised."""
    torch = pytest.importorskip("torch")
    s = L.Solver(L.make_params(4096, 4097, 1, precision=L.FP16_DEV))
    lib = L.load()
    d_out = torch.zeros(L.NDIAG, dtype=torch.float64, device="cuda")
    rc = lib.lbrmhd_get_diagnostics_noalloc(s._h, 0, C.c_void_p(d_out.data_ptr()))
    assert rc == L.ERR_BAD_ARG
    assert b"limit" in lib.lbrmhd_last_error(s._h)
    s.close()

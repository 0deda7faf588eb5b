"""The reconnection-rate diagnostic on the GPU against its float64 reference
(oracle/diagnostics_ref.py): exactly on the GPU's own fields, and against the
FP64 oracle's run (the null is unique only up to the parity tolerance, so
the GPU's null point is checked to be a null of the oracle's field and R is
compared there)."""
import numpy as np
import pytest

import oracle as O
from oracle import diagnostics_ref as D
from paper_1508_03452_gb300 import lbrmhd as L
from paper_1508_03452_gb300 import workloads as W

pytestmark = pytest.mark.gpu

NX, NY, B0 = 96, 64, 0.1
BAND = (8, 24)  # rows around the layer at y = NY / 4


def _fields():
    return W.kelvin_helmholtz(NX, NY, 1, V=0.2, ratio=3.0, B0=B0, a=2.0, noise=1e-3, seed=4)


@pytest.mark.parametrize("precision", [L.FP64, L.FP32])
def test_reconnection_rate_matches_reference_on_gpu_fields(precision):
    F = _fields()
    s = L.Solver(L.make_params(NX, NY, 1, sigma=1e3, precision=precision))
    s.init_fields(0, F.n, F.p, F.u, F.B)
    m0 = s.moments()
    for steps in (0, 10, 25):
        s.step(steps)
        m = s.moments()
        r = s.reconnection_rate(0, *BAND, B0)
        R, x, y, b = D.reconnection_rate(m[8], m0[8], m[9], m[10], NX, NY, B0, *BAND)
        assert (r["x"], r["y"]) == (x, y)
        assert r["R"] == pytest.approx(R, rel=1e-12, abs=1e-300) and r["B"] == pytest.approx(b, rel=1e-12, abs=0)
    s.close()


def test_reconnection_rate_against_oracle_and_checkpoint():
    F = _fields()
    steps = 25
    s = L.Solver(L.make_params(NX, NY, 1, sigma=1e3, precision=L.FP64))
    s.init_fields(0, F.n, F.p, F.u, F.B)
    s.step(steps)
    r = s.reconnection_rate(0, *BAND, B0)
    ref = O.Sim(O.make_params(NX, NY, 1, sigma=1e3, threads=8))
    ref.init(F.n, F.p, F.u, F.B)
    mo0 = ref.moments()
    ref.step(steps)
    mo = ref.moments()
    _, _, _, bmin = D.reconnection_rate(mo[8], mo0[8], mo[9], mo[10], NX, NY, B0, *BAND)
    c = r["y"] * NX + r["x"]
    b_at = np.hypot(mo[9][c], mo[10][c])
    assert b_at <= bmin + 1e-10 * B0  # the GPU's null is a null of the oracle's field
    assert r["R"] == pytest.approx((mo[8][c] - mo0[8][c]) / B0, rel=1e-8, abs=1e-12)
    # E^z_0 travels with a checkpoint
    blob = s.get_state()
    t = L.Solver(L.make_params(NX, NY, 1, sigma=1e3, precision=L.FP64))
    t.set_state(blob)
    assert t.reconnection_rate(0, *BAND, B0) == r
    with pytest.raises(L.LbrmhdError):
        t.reconnection_rate(0, 10, 10, B0)
    with pytest.raises(L.LbrmhdError):
        t.reconnection_rate(0, 0, NY + 1, B0)
    s.close()
    t.close()

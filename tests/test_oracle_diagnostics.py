"""Pins of the reconnection-rate reference (oracle/diagnostics_ref.py) against
fields whose null point and rate are known in closed form."""
import numpy as np

from oracle import diagnostics_ref as D


def _xpoint(nx, ny, x0, y0, scale=1.0):
    """B = (y - y0, x - x0) (an X-point at (x0, y0)), sampled at cell centres."""
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    return (scale * (y - y0)).ravel(), (scale * (x - x0)).ravel()


def test_single_xpoint_position_and_rate():
    nx, ny = 40, 30
    Bx, By = _xpoint(nx, ny, 17, 11, scale=0.01)
    Ez0 = np.full(nx * ny, 0.3)
    Ez = Ez0.copy()
    Ez[11 * nx + 17] = 0.3 + 0.004  # the generated field at the null
    R, x, y, b = D.reconnection_rate(Ez, Ez0, Bx, By, nx, ny, 0.1, 0, ny)
    assert (x, y) == (17, 11) and b == 0.0
    assert R == (0.3 + 0.004 - 0.3) / 0.1


def test_band_selects_the_named_layer_and_ties_go_low():
    nx, ny = 32, 40
    Bx1, By1 = _xpoint(nx, ny, 5, 9)
    Bx2, By2 = _xpoint(nx, ny, 20, 30)
    # two X-points: the field vanishes at both; each band finds its own
    b2 = np.minimum(Bx1 ** 2 + By1 ** 2, Bx2 ** 2 + By2 ** 2)
    Bx, By = np.sqrt(b2), np.zeros_like(b2)
    Ez = np.arange(nx * ny, dtype=np.float64)
    Ez0 = np.zeros(nx * ny)
    R, x, y, _ = D.reconnection_rate(Ez, Ez0, Bx, By, nx, ny, 2.0, 0, 20)
    assert (x, y) == (5, 9) and R == (9 * nx + 5) / 2.0
    R, x, y, _ = D.reconnection_rate(Ez, Ez0, Bx, By, nx, ny, 2.0, 20, 40)
    assert (x, y) == (20, 30)
    # a uniform band: every cell ties, the lowest index wins
    c, _ = D.null_point(np.ones(nx * ny), np.zeros(nx * ny), nx, ny, 7, 12)
    assert c == 7 * nx

"""Float64 reference of the reconnection-rate diagnostic, written out plainly.

TEST INFRASTRUCTURE ONLY (like the rest of this package).

The paper (Sec. IV, Kelvin-Helmholtz-driven reconnection) measures the
reconnection rate as the out-of-plane electric field generated at the null
point, normalised by the field strength: R(t) = (E^z - E^z_0) / B0 taken at the
null point, E^z_0 being the initial out-of-plane field there. The null point
moves as the instability evolves; it is located here as the cell of smallest
in-plane field magnitude B_x^2 + B_y^2 within a band of rows (the periodic
set-ups hold two current layers, so the caller names the layer's rows). Ties
go to the lowest cell index (x fastest).

Pins (tests/test_oracle_diagnostics.py): a field with a single X-point of known
position and a known E^z change gives that position and R exactly; the band
restriction picks the null of the named layer.
"""
from __future__ import annotations

import numpy as np


def null_point(Bx, By, nx, ny, y_lo, y_hi):
    """(cell index, |B_in-plane|) of the smallest in-plane field in rows
    y_lo <= y < y_hi of a 2-D run (fields of nx * ny values, x fastest)."""
    b2 = (np.asarray(Bx, dtype=np.float64) ** 2 + np.asarray(By, dtype=np.float64) ** 2).reshape(ny, nx)
    band = b2[y_lo:y_hi]
    k = int(np.argmin(band))  # first occurrence: the lowest index
    y, x = divmod(k, nx)
    return (y + y_lo) * nx + x, float(np.sqrt(band.flat[k]))


def reconnection_rate(Ez, Ez0, Bx, By, nx, ny, B0, y_lo, y_hi):
    """R = (E^z - E^z_0) / B0 at the null point of rows [y_lo, y_hi); returns
    (R, x, y, |B| at the null)."""
    c, bmag = null_point(Bx, By, nx, ny, y_lo, y_hi)
    R = (float(np.asarray(Ez, dtype=np.float64).reshape(-1)[c]) -
         float(np.asarray(Ez0, dtype=np.float64).reshape(-1)[c])) / B0
    return R, c % nx, c // nx, bmag

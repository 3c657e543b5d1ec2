"""Sound-speed derivative grids and bilinear sampling (TEST INFRASTRUCTURE ONLY).

The ray equations (Eikonal, Eq. 6; Transport via dynamic ray tracing, Eq. 7)
need c, grad c and the Hessian of c along each ray.  The paper gives no
discretisation; the reading taken here:
  * first derivatives by central differences over the index-clamped
    neighbours, c_x(i) = (c(i+1') - c(i-1')) / ((i+1' - (i-1')) h), which is
    one-sided at the grid edge;
  * second derivatives c_xx(i) = (c(i*+1) - 2 c(i*) + c(i*-1)) / h^2 with
    i* = clamp(i, 1, nx-2) (an edge pixel takes its inner neighbour's
    stencil), likewise c_yy; and the mixed
    c_xy = (c(i+1',j+1') - c(i+1',j-1') - c(i-1',j+1') + c(i-1',j-1'))
           / ((i+1' - (i-1')) h (j+1' - (j-1')) h);
  * each of the 7 grids (c, c_x, c_y, c_xx, c_xy, c_yy, alpha0) is sampled by
    bilinear interpolation of its pixel-centre values, with the query
    clamped to the grid.
For a linear c these give exact gradients and zero second derivatives
everywhere; for a quadratic c the second derivatives are exact everywhere.
"""
from __future__ import annotations

import numpy as np

from .geometry import Geom

FIELD_NAMES = ("c", "c_x", "c_y", "c_xx", "c_xy", "c_yy", "alpha0")


def fields(g: Geom, c: np.ndarray, alpha0: np.ndarray) -> np.ndarray:
    """F[7, ny, nx] float64 in the order of FIELD_NAMES."""
    c = np.asarray(c, dtype=np.float64).reshape(g.ny, g.nx)
    a0 = np.asarray(alpha0, dtype=np.float64).reshape(g.ny, g.nx)
    h = g.h
    ix = np.arange(g.nx)
    iy = np.arange(g.ny)
    ip, im = np.minimum(ix + 1, g.nx - 1), np.maximum(ix - 1, 0)
    jp, jm = np.minimum(iy + 1, g.ny - 1), np.maximum(iy - 1, 0)
    dxs = ((ip - im) * h)[None, :]
    dys = ((jp - jm) * h)[:, None]
    F = np.empty((7, g.ny, g.nx))
    F[0] = c
    F[1] = (c[:, ip] - c[:, im]) / dxs
    F[2] = (c[jp, :] - c[jm, :]) / dys
    ic = np.clip(ix, 1, g.nx - 2)
    jc = np.clip(iy, 1, g.ny - 2)
    F[3] = (c[:, ic + 1] - 2.0 * c[:, ic] + c[:, ic - 1]) / (h * h)
    F[4] = (c[jp][:, ip] - c[jm][:, ip] - c[jp][:, im] + c[jm][:, im]) / (dxs * dys)
    F[5] = (c[jc + 1, :] - 2.0 * c[jc, :] + c[jc - 1, :]) / (h * h)
    F[6] = a0
    return F


def bilinear(g: Geom, grid: np.ndarray, x, y) -> np.ndarray:
    """Bilinear sample of one [ny, nx] grid at points (x, y), query clamped to the grid."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    u = np.clip(x / g.h + 0.5 * (g.nx - 1), 0.0, g.nx - 1)
    v = np.clip(y / g.h + 0.5 * (g.ny - 1), 0.0, g.ny - 1)
    i0 = np.minimum(np.floor(u).astype(np.int64), g.nx - 2)
    j0 = np.minimum(np.floor(v).astype(np.int64), g.ny - 2)
    fu = u - i0
    fv = v - j0
    return ((1 - fu) * (1 - fv) * grid[j0, i0] + fu * (1 - fv) * grid[j0, i0 + 1]
            + (1 - fu) * fv * grid[j0 + 1, i0] + fu * fv * grid[j0 + 1, i0 + 1])

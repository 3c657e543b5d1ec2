"""High-frequency 2-D Green's function on the grid (TEST INFRASTRUCTURE ONLY).

Eq. 4 writes g ~ A exp(i [phi + pi/4]) with A = A_geom A_abs (Eq. 5); phi = omega T
solves the Eikonal equation (Eq. 6) and A_geom the Transport equation
(Eq. 7).  Written out (time convention exp(-i omega t), matching the +i of
Eq. 4):

  G_t(x, w) = sqrt(c(x) / (8 pi w J)) * exp(-K_a f_MHz^y L)
              * exp(i [w T + dphi(w, L) + pi/4 - kappa pi/2])

* A_geom: the Transport equation keeps A^2 (w/c) J constant along a ray
  tube; matching the 2-D Green's function (i/4) H0(kr) near the source,
  whose far field is sqrt(1/(8 pi k r)) exp(i (k r + pi/4)), fixes the
  constant, so A_geom = sqrt(c(x)/(8 pi w J)).  J = |Q| is floored at h/4
  (caustic guard, a reading).
* A_abs: alpha(f) = alpha0 f_MHz^y dB/cm; K_a = 100 ln(10)/20 turns dB/cm into
  Np/m; L is the ray integral of alpha0.
* dphi: power-law (Kramers-Kronig, time-causal) dispersion relative to the
  reference frequency f_ref at which c is the phase speed (a reading: the
  paper names dispersion, Sec. 1, without its law):
    y != 1: dphi = w tan(pi y/2) (w^(y-1) - w_ref^(y-1)) K_a L (2 pi 1e6)^(-y)
    y == 1: dphi = -(2/pi) w ln(w/w_ref) K_a L (2 pi 1e6)^(-1)
* kappa: KMAH index, a -pi/2 phase shift per caustic crossed.
* s(w) = 1 (point source of unit amplitude).
"""
from __future__ import annotations

import math

import numpy as np

from .geometry import Geom, element_positions, pixel_centres

K_A = 100.0 * math.log(10.0) / 20.0  # dB/cm -> Np/m


def dispersion_phase(f_hz: float, L, y: float, f_ref: float) -> np.ndarray:
    L = np.asarray(L, dtype=np.float64)
    w = 2.0 * math.pi * f_hz
    wr = 2.0 * math.pi * f_ref
    if y == 1.0:
        return -(2.0 / math.pi) * w * math.log(w / wr) * K_A * L / (2.0 * math.pi * 1e6)
    diff = wr ** (y - 1.0) * math.expm1((y - 1.0) * math.log(w / wr))  # w^(y-1) - wr^(y-1)
    return w * math.tan(0.5 * math.pi * y) * diff * K_A * L * (2.0 * math.pi * 1e6) ** (-y)


def green_value(g: Geom, f_hz: float, T, Q, L, kappa, c_local) -> np.ndarray:
    """Eq. 4-5 evaluated from ray quantities (traveltime T, tube width Q, absorption
    integral L, KMAH index kappa) and the local sound speed."""
    w = 2.0 * math.pi * f_hz
    J = np.maximum(np.abs(Q), 0.25 * g.h)
    amp = np.sqrt(np.asarray(c_local, dtype=np.float64) / (8.0 * math.pi * w * J))
    amp = amp * np.exp(-K_A * (f_hz / 1e6) ** g.power_y * np.asarray(L))
    ph = w * np.asarray(T) + dispersion_phase(f_hz, L, g.power_y, g.f_ref) + 0.25 * math.pi \
        - 0.5 * math.pi * np.asarray(kappa)
    return amp * np.exp(1j * ph)


def gridded_traveltime(g: Geom, tables) -> np.ndarray:
    """T(p) = |p - x_t|/c_ref + T_res(p), [n_elem, npix]."""
    xe, ye = element_positions(g)
    X, Y = pixel_centres(g)
    D = np.hypot(X.ravel()[None, :] - xe[:, None], Y.ravel()[None, :] - ye[:, None])
    return D / g.c_ref + tables.t_res


def green(g: Geom, tables, c: np.ndarray, f_hz: float, pix=None) -> np.ndarray:
    """G[n_elem, npix] complex128 from full tables; or, with pix, G[n_elem, len(pix)] at those flat
    pixel indices from tables that hold exactly those pixels (grid.grid_pixels); zero at holes."""
    c = np.asarray(c, dtype=np.float64).ravel()
    xe, ye = element_positions(g)
    X, Y = pixel_centres(g)
    X, Y = X.ravel(), Y.ravel()
    sl = slice(None) if pix is None else np.asarray(pix)
    D = np.hypot(X[sl][None, :] - xe[:, None], Y[sl][None, :] - ye[:, None])
    T = D / g.c_ref + tables.t_res
    G = green_value(g, f_hz, T, tables.q, tables.l, tables.kappa, c[sl][None, :])
    return np.where(tables.hit, G, 0.0)

"""Born forward operator, adjoint and Gauss-Newton Hessian diagonal
(TEST INFRASTRUCTURE ONLY).

The linearised subproblem (Eqs. 9-10) is, per the paper's Sec. 1, a form of
the Born approximation whose Green's functions come from rays.  Perturbing
k^2 = w^2/c^2 in Eq. 1 by dc gives d(k^2) = -2 w^2 dc / c^3; with the pixel area
h^2 as quadrature weight the scattered data are

  d[e, r] = w^2 sum_x G_e(x) G_r(x) m(x),     m = -2 h^2 dc / c^3,

using reciprocity G(x_r, x) = G_r(x).  For real m and data weights W the
misfit F(m) = 1/2 sum W |R + B m|^2 has gradient (at m = 0)

  g(x) = w^2 sum_{e,r} conj(G_e(x) G_r(x)) W[e,r] R[e,r]   (use Re g),

and Gauss-Newton Hessian diagonal

  H(x) = w^4 sum_{e,r} W[e,r] |G_e(x)|^2 |G_r(x)|^2.

Straight NumPy complex128 matrix products; no blocking or reordering.
"""
from __future__ import annotations

import math

import numpy as np


def born_forward(G: np.ndarray, m: np.ndarray, f_hz: float) -> np.ndarray:
    """d[e, r] = w^2 sum_x G_e(x) G_r(x) m(x).  G[n_elem, npix], m[npix] (real or complex)."""
    w = 2.0 * math.pi * f_hz
    return (w * w) * ((G * m[None, :]) @ G.T)


def born_adjoint(G: np.ndarray, S: np.ndarray, f_hz: float) -> np.ndarray:
    """g(x) = w^2 sum_{e,r} conj(G_e(x) G_r(x)) S[e, r], with S = W * R (complex [npix])."""
    w = 2.0 * math.pi * f_hz
    Gc = np.conj(G)
    U = S @ Gc                       # U[e, x] = sum_r S[e, r] conj(G_r(x))
    return (w * w) * np.sum(Gc * U, axis=0)


def hess_diag(G: np.ndarray, W: np.ndarray, f_hz: float) -> np.ndarray:
    """H(x) = w^4 sum_{e,r} W[e, r] |G_e(x)|^2 |G_r(x)|^2 (real [npix])."""
    w = 2.0 * math.pi * f_hz
    A = np.abs(G) ** 2
    V = np.asarray(W, dtype=np.float64) @ A
    return (w ** 4) * np.sum(A * V, axis=0)

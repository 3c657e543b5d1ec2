"""Ray fans through the current sound speed (TEST INFRASTRUCTURE ONLY).

Python front end of rb_oracle.c.  What a fan is (readings where the paper,
Sec. 2 and the ray-tracing remarks of Sec. 5, is silent):
  * element t emits N_ray rays with take-off angle th_0 = phi_t + pi + psi_i,
    psi_i = -pi/2 + (i + 1/2) pi / N_ray: the inward half-plane, never exactly
    along the tangent;
  * initial state T = 0, Q = 0, P = 1/c(x_t), L = 0; with this P the dynamic
    ray-tracing Q is the ray-tube width per radian of take-off angle, so
    J = |Q| is the geometric spreading of the Transport equation (Eq. 7);
  * classical RK4 in arclength with fixed step ds (half a pixel), stopping at
    the first step k >= 1 with |x_k| >= R and closing with the linearly
    interpolated crossing of the ring; a ray still inside after max_steps is
    "lost";
  * KMAH index kappa: the number of sign changes of Q between consecutive
    vertices from the second step on (caustic crossings).

Vertex records hold (x, y, th, T, Q, P, L, kappa, s).
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _clib
from .fields import fields
from .geometry import Geom

NV = 9
VX, VY, VTH, VT, VQ, VP, VL, VK, VS = range(NV)


def _cgeom(g: Geom) -> _clib.OrcGeom:
    return _clib.OrcGeom(g.n_elem, g.ring_radius, g.nx, g.ny, g.h, g.n_rays, g.ds, g.max_steps,
                         g.support_margin, g.c_ref)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def trace_fan(g: Geom, c: np.ndarray, alpha0: np.ndarray, t: int, F: np.ndarray | None = None):
    """All rays of element t: (V[n_rays, max_steps+1, NV], nvert[n_rays], n_lost)."""
    if F is None:
        F = fields(g, c, alpha0)
    F = np.ascontiguousarray(F, dtype=np.float64)
    V = np.zeros((g.n_rays, g.max_steps + 1, NV))
    nvert = np.zeros(g.n_rays, dtype=np.int32)
    cg = _cgeom(g)
    nl = _clib.lib().orc_trace_fan(ctypes.byref(cg), _ptr(F), int(t), _ptr(V), _ptr(nvert))
    return V, nvert, int(nl)


def trace_endpoints(g: Geom, c: np.ndarray, alpha0: np.ndarray, F: np.ndarray | None = None):
    """Last vertex of every ray: (E[n_elem, n_rays, NV], nvert[n_elem, n_rays], lost[n_elem, n_rays])."""
    if F is None:
        F = fields(g, c, alpha0)
    F = np.ascontiguousarray(F, dtype=np.float64)
    E = np.zeros((g.n_elem, g.n_rays, NV))
    nvert = np.zeros((g.n_elem, g.n_rays), dtype=np.int32)
    lost = np.zeros((g.n_elem, g.n_rays), dtype=np.int32)
    cg = _cgeom(g)
    _clib.lib().orc_trace_endpoints(ctypes.byref(cg), _ptr(F), _ptr(E), _ptr(nvert), _ptr(lost))
    return E, nvert, lost

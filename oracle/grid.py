"""First-arrival gridding of ray fans onto pixels (TEST INFRASTRUCTURE ONLY).

The paper names "back-propagation of ray parameters" onto the grid as a
step of the method (Sec. 5) without giving it.  The reading implemented in
rb_oracle.c:
  * rays i and i+1 of a fan and steps k, k+1 bound a quad, split along
    (i,k)-(i+1,k+1) into triangles {(i,k),(i+1,k),(i+1,k+1)} and
    {(i,k),(i+1,k+1),(i,k+1)}; a ray that has already reached the ring keeps
    its exit vertex (vertex indices clamp at the last one), which closes the
    tube up to the ring; zero-area triangles are skipped;
  * a support pixel lies in a triangle when all barycentric weights are
    >= -1e-12;
  * the traveltime is interpolated as a residual against the straight water
    time, T(p) = |p - x_t|/c_ref + sum_j w_j (T_j - |v_j - x_t|/c_ref); Q and
    L are interpolated linearly, J = |Q|; kappa comes from the vertex with
    the largest weight;
  * where several triangles contain the pixel the smallest T wins (first
    arrival); ties keep the earliest triangle (i, k, half) in that order;
  * an uncovered support pixel is a hole: its Green's function is zero.
"""
from __future__ import annotations

import ctypes
import dataclasses

import numpy as np

from . import _clib
from .fields import fields
from .geometry import Geom, r2max
from .rays import _cgeom, _ptr


@dataclasses.dataclass
class Tables:
    t_res: np.ndarray   # [n_elem, npix] s
    q: np.ndarray       # [n_elem, npix] signed tube width (J = |q|)
    l: np.ndarray       # [n_elem, npix] integral of alpha0 along the ray
    kappa: np.ndarray   # [n_elem, npix] int
    tri: np.ndarray     # [n_elem, npix] int64 winning triangle id, -1 for holes
    hit: np.ndarray     # [n_elem, npix] bool
    n_lost: int = 0


def grid(g: Geom, c: np.ndarray, alpha0: np.ndarray, F: np.ndarray | None = None) -> Tables:
    if F is None:
        F = fields(g, c, alpha0)
    F = np.ascontiguousarray(F, dtype=np.float64)
    out = np.zeros((g.n_elem, g.npix, 6))
    cg = _cgeom(g)
    nl = _clib.lib().orc_grid(ctypes.byref(cg), _ptr(F), ctypes.c_int64(r2max(g)), _ptr(out))
    return Tables(t_res=out[..., 0].copy(), q=out[..., 1].copy(), l=out[..., 2].copy(),
                  kappa=out[..., 3].astype(np.int64), tri=out[..., 4].astype(np.int64),
                  hit=out[..., 5] > 0.5, n_lost=int(nl))


def grid_pixels(g: Geom, c: np.ndarray, alpha0: np.ndarray, pix: np.ndarray, F: np.ndarray | None = None) -> Tables:
    """The same tables as grid(), kept only at the listed flat pixel indices ([n_elem, len(pix)])."""
    if F is None:
        F = fields(g, c, alpha0)
    F = np.ascontiguousarray(F, dtype=np.float64)
    sel = np.ascontiguousarray(pix, dtype=np.int64)
    out = np.zeros((g.n_elem, sel.size, 6))
    cg = _cgeom(g)
    nl = _clib.lib().orc_grid_pixels(ctypes.byref(cg), _ptr(F), ctypes.c_int64(r2max(g)), _ptr(sel),
                                     ctypes.c_int64(sel.size), _ptr(out))
    return Tables(t_res=out[..., 0].copy(), q=out[..., 1].copy(), l=out[..., 2].copy(),
                  kappa=out[..., 3].astype(np.int64), tri=out[..., 4].astype(np.int64),
                  hit=out[..., 5] > 0.5, n_lost=int(nl))


def triangles_of_fan(g: Geom, V: np.ndarray, nvert: np.ndarray):
    """Every triangle of one fan as arrays (ids, vertex records [n, 3, NV]), in id order.
    Used by tests to brute-force the first arrival."""
    ids, tris = [], []
    KQ = g.max_steps + 1
    for i in range(g.n_rays - 1):
        na, nb = int(nvert[i]), int(nvert[i + 1])
        for k in range(max(na, nb) - 1):
            A0 = V[i, min(k, na - 1)]
            A1 = V[i, min(k + 1, na - 1)]
            B0 = V[i + 1, min(k, nb - 1)]
            B1 = V[i + 1, min(k + 1, nb - 1)]
            tris.append((A0, B0, B1))
            ids.append((i * KQ + k) * 2)
            tris.append((A0, B1, A1))
            ids.append((i * KQ + k) * 2 + 1)
    return np.array(ids, dtype=np.int64), np.array(tris)

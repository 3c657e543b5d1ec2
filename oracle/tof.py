"""Time-of-flight initial guess (TEST INFRASTRUCTURE ONLY).

Sec. 4: the ray-Born sweep starts from a smooth, low-contrast image obtained by a
few (three) linearisations of a time-of-flight reconstruction, which minimises the
misfit between measured times of flight and times of flight along rays.  The paper
gives no more detail; the readings taken here:

* ToF of the pair (e, r): the first-arrival traveltime of the ray linking
  (``link.link``): T_er = chord/c_ref + (1 - lam) tres_i + lam tres_(i+1) over the
  winning interval (rays i, i + 1) of fan e.
* Linearisation in slowness s = 1/c along fixed rays (Fermat): dT_er =
  (1 - lam) int_(ray i) ds dl + lam int_(ray i+1) ds dl.  A ray is the polyline of
  its RK4 vertices; int f dl = sum over segments of |x_(k+1) - x_k| f(midpoint),
  and f on the grid is the bilinear interpolant of pixel values (the basis the
  fields use).  This is the operator L (rows: pairs, columns: pixels).
* Rows used: receivers on the opposite ~75 % of the ring (as the data weights),
  pairs linked both in the measured data and in the current medium.
* One linearisation = one SIRT step (simultaneous iterative reconstruction,
  Gilbert 1972): ds = D_col^-1 L^T D_row^-1 dT with dT = T_obs - T(c), D_row the
  row sums of L (interpolated ray lengths), D_col its column sums; the per-row
  mean slowness error dT / D_row is clamped to +-2e-3 s/m; ds is applied on the
  support where D_col > 0; c <- 1 / (1/c + ds).  Rays and links are recomputed
  in the updated medium before the next linearisation.

Pinned by closed forms on straight rays (the ray integral of a linear field is the
ray length times its value at the ray's midpoint), the adjoint identity of the
projection and back-projection (a dot-product test), exact recovery of a uniform
slowness shift from linear data in one SIRT step, and a decreasing ToF residual.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List

import numpy as np

from . import link, rays
from .fields import fields
from .geometry import Geom, receiver_mask, support_mask

A_MAX = 2e-3   # clamp of the per-row mean slowness error [s/m]


@dataclasses.dataclass
class Paths:
    """Ray segments of every fan: for ray (t, i), pixel indices [.., 4], bilinear weights
    times segment length [.., 4], flattened, with the ray id of each segment."""
    ray: np.ndarray       # [n_seg] t * n_rays + i
    pix: np.ndarray       # [n_seg, 4]
    wl: np.ndarray        # [n_seg, 4] phi_p(midpoint) * segment length
    length: np.ndarray    # [n_elem, n_rays] sum of segment lengths (0 for a lost ray)


def bilinear_basis(g: Geom, x: np.ndarray, y: np.ndarray):
    """Pixel indices and weights of the bilinear interpolant at (x, y) (query clamped)."""
    u = np.clip(x / g.h + 0.5 * (g.nx - 1), 0.0, g.nx - 1.0)
    v = np.clip(y / g.h + 0.5 * (g.ny - 1), 0.0, g.ny - 1.0)
    i0 = np.minimum(np.floor(u).astype(np.int64), g.nx - 2)
    j0 = np.minimum(np.floor(v).astype(np.int64), g.ny - 2)
    fu, fv = u - i0, v - j0
    p00 = j0 * g.nx + i0
    pix = np.stack([p00, p00 + 1, p00 + g.nx, p00 + g.nx + 1], axis=-1)
    w = np.stack([(1 - fu) * (1 - fv), fu * (1 - fv), (1 - fu) * fv, fu * fv], axis=-1)
    return pix, w


def ray_paths(g: Geom, c: np.ndarray, alpha0: np.ndarray, F=None) -> Paths:
    if F is None:
        F = fields(g, c, alpha0)
    R_, P_, W_ = [], [], []
    length = np.zeros((g.n_elem, g.n_rays))
    for t in range(g.n_elem):
        V, nvert, _ = rays.trace_fan(g, c, alpha0, t, F)
        x, y = V[:, :, rays.VX], V[:, :, rays.VY]
        seg_len = np.hypot(x[:, 1:] - x[:, :-1], y[:, 1:] - y[:, :-1])
        k = np.arange(g.max_steps)[None, :]
        valid = (nvert[:, None] > 0) & (k < nvert[:, None] - 1)
        seg_len = np.where(valid, seg_len, 0.0)
        length[t] = seg_len.sum(axis=1)
        ii, kk = np.nonzero(valid)
        mx = 0.5 * (x[ii, kk] + x[ii, kk + 1])
        my = 0.5 * (y[ii, kk] + y[ii, kk + 1])
        pix, w = bilinear_basis(g, mx, my)
        R_.append(t * g.n_rays + ii)
        P_.append(pix)
        W_.append(w * seg_len[ii, kk][:, None])
    return Paths(np.concatenate(R_), np.concatenate(P_), np.concatenate(W_), length)


def ray_integrals(g: Geom, P: Paths, s: np.ndarray) -> np.ndarray:
    """int_(ray) s dl for every ray: [n_elem, n_rays]."""
    per_seg = np.sum(P.wl * np.asarray(s, dtype=np.float64).ravel()[P.pix], axis=1)
    out = np.zeros(g.n_elem * g.n_rays)
    np.add.at(out, P.ray, per_seg)
    return out.reshape(g.n_elem, g.n_rays)


def project(g: Geom, P: Paths, lk: link.Links, rows: np.ndarray, s: np.ndarray) -> np.ndarray:
    """(L s)[e, r] on the rows (zero elsewhere)."""
    I = ray_integrals(g, P, s)
    b = np.where(rows, lk.best, 0)
    e = np.arange(g.n_elem)[:, None]
    val = (1.0 - lk.lam) * I[e, b] + lk.lam * I[e, np.minimum(b + 1, g.n_rays - 1)]
    return np.where(rows, val, 0.0)


def backproject(g: Geom, P: Paths, lk: link.Links, rows: np.ndarray, d: np.ndarray) -> np.ndarray:
    """(L^T d)[pixel] for row values d[e, r] (rows outside ``rows`` ignored)."""
    a = np.zeros((g.n_elem, g.n_rays))
    e, r = np.nonzero(rows)
    b = lk.best[e, r]
    lam = lk.lam[e, r]
    np.add.at(a, (e, b), (1.0 - lam) * d[e, r])
    np.add.at(a, (e, b + 1), lam * d[e, r])
    out = np.zeros(g.npix)
    np.add.at(out, P.pix.ravel(), (P.wl * a.ravel()[P.ray][:, None]).ravel())
    return out


@dataclasses.dataclass
class TofState:
    T: np.ndarray
    linked: np.ndarray
    lk: link.Links
    paths: Paths


def tof_state(g: Geom, c: np.ndarray, alpha0: np.ndarray) -> TofState:
    c = np.asarray(c, dtype=np.float64).reshape(g.ny, g.nx)
    F = fields(g, c, alpha0)
    E, _, lost = rays.trace_endpoints(g, c, alpha0, F)
    lk = link.link(g, E, lost, c)
    return TofState(lk.T, lk.linked, lk, ray_paths(g, c, alpha0, F))


def tof_times(g: Geom, c: np.ndarray, alpha0: np.ndarray):
    """Linked first-arrival times of flight T[e, r] and the linked mask."""
    c = np.asarray(c, dtype=np.float64).reshape(g.ny, g.nx)
    E, _, lost = rays.trace_endpoints(g, c, alpha0)
    lk = link.link(g, E, lost, c)
    return lk.T, lk.linked


def sirt_step(g: Geom, S: TofState, T_obs: np.ndarray, obs_linked: np.ndarray):
    """Slowness update ds[npix] of one linearisation, and the RMS ToF residual of its rows."""
    rows = receiver_mask(g) & S.linked & obs_linked
    dT = np.where(rows, T_obs - S.T, 0.0)
    b = np.where(rows, S.lk.best, 0)
    e = np.arange(g.n_elem)[:, None]
    d_row = (1.0 - S.lk.lam) * S.paths.length[e, b] + S.lk.lam * S.paths.length[e, np.minimum(b + 1, g.n_rays - 1)]
    ok = rows & (d_row > 0.0)
    mean_err = np.where(ok, np.clip(dT / np.where(ok, d_row, 1.0), -A_MAX, A_MAX), 0.0)
    num = backproject(g, S.paths, S.lk, ok, mean_err)
    den = backproject(g, S.paths, S.lk, ok, np.ones_like(mean_err))
    upd = support_mask(g).ravel() & (den > 0.0)
    ds = np.where(upd, num / np.where(den > 0.0, den, 1.0), 0.0)
    n = int(rows.sum())
    rms = math.sqrt(float(np.sum(dT[rows] ** 2)) / n) if n else 0.0
    return ds, rms


def tof_invert(g: Geom, c0: np.ndarray, alpha0: np.ndarray, T_obs: np.ndarray, obs_linked: np.ndarray,
               n_iter: int = 3):
    """n_iter linearisations from c0; returns (c, [RMS ToF residual before each one and after the last])."""
    c = np.asarray(c0, dtype=np.float64).reshape(g.ny, g.nx).copy()
    hist: List[float] = []
    for _ in range(n_iter):
        S = tof_state(g, c, alpha0)
        ds, rms = sirt_step(g, S, T_obs, obs_linked)
        hist.append(rms)
        c = (1.0 / (1.0 / c.ravel() + ds)).reshape(g.ny, g.nx)
    T, linked = tof_times(g, c, alpha0)
    rows = receiver_mask(g) & linked & obs_linked
    dT = T_obs - T
    hist.append(math.sqrt(float(np.sum(dT[rows] ** 2)) / max(int(rows.sum()), 1)))
    return c, hist

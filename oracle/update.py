"""Data weighting, the Hessian-free one-step update and the frequency sweep
(TEST INFRASTRUCTURE ONLY).

Sec. 3 (Eqs. 8-10) and Sec. 4 give the method; the paper defers the exact
weights to its reference [Javaherian 2022], so these are readings:

* Objective (Eq. 8): F = 1/2 sum_w sum_{e,r} W |R|^2, R = p_ray(c) - p_obs, the
  frequency integral taken as a sum over the set.
* Data-space weight W (Sec. 4.1): receivers on the opposite ~75 % of the ring
  (circular index distance >= ceil(N_t/8)) and linked by a ray; then "the
  largest 1 % of values set to zero" per frequency set, read as: over all
  kept entries (w, e, r) of the set, zero the floor(frac * count) entries of
  largest |R|, ties to the smallest flat index (w, e, r).
* Solution-space weight and one step (Eq. 10 with a diagonal Hessian):
  W_m = 1 / (sum_w H_w + eps), eps = eps_rel * mean over the support of
  sum_w H_w;  direction p = -W_m sum_w Re g_w on the support, 0 outside.
  Step mode "diag": dm = p.  Step mode "exact" (default): dm = alpha p with
  the scalar alpha that minimises the linearised objective of Eq. 10 along
  p, alpha = -<sum_w Re g_w, p> / sum_w sum_{e,r} W |B_w p|^2 (zero if the
  denominator is zero).  The scalar is read as the normalisation of the
  solution-space weight: the bare diagonal overshoots by roughly the area of
  the Hessian's point-spread function in pixels (about 9x on the tiny
  phantom), which the paper's weighting must remove.
  dc = -dm c^3 / (2 h^2);  c <- c + dc;  report ||dc||_2 over the support.
* Sweep (Secs. 1, 3, 4): sets of consecutive frequencies, low to high; the
  image after one set seeds the next; rays and tables are recomputed per set.
* Synthetic data: p_obs_w = p_ray_w(c0) + B_w(c0) m_true + noise,
  m_true = -2 h^2 (c_true - c0)/c0^3 on the support, noise =
  level * rms_masked |p_obs_w| * (n1 + i n2)/sqrt(2) with the seeded draws.

* CG variant (``cg_solve``, ``cg_update``): the same linearised objective solved by
  conjugate gradients instead of the diagonal Hessian (readings beside the code);
  pinned by Krylov optimality, finite termination, the first iteration equal to the
  one-step update, and a decreasing objective.

``sweep`` has no printed values to match (the paper's figures are absent); it is
pinned by the fixed point of the true medium under its own noise-free data and by
the error to the phantom falling set by set.  The one-step solve is pinned by a
least-squares check on a single-pixel support.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence

import numpy as np

from . import born, green, link, rays
from .fields import fields
from .geometry import Geom, receiver_mask, support_mask
from .grid import grid


def outlier_weights(base: np.ndarray, R: np.ndarray, frac: float):
    """W[nw, e, r] as uint8 from the kept-entry mask base[nw, e, r] and residuals R.
    Zeroes floor(frac * count) kept entries of largest |R| (ties: smallest flat index)."""
    W = base.astype(np.uint8).copy()
    flat = np.flatnonzero(base.ravel())
    k = int(math.floor(frac * flat.size))
    if k > 0:
        mag = np.abs(R.ravel()[flat]) ** 2
        order = np.lexsort((flat, -mag))   # primary: largest |R|^2, then smallest index
        W.ravel()[flat[order[:k]]] = 0
    return W, flat.size, k


@dataclasses.dataclass
class UpdateResult:
    c_new: np.ndarray
    dc: np.ndarray
    dc_norm: float
    g_sum: np.ndarray
    h_sum: np.ndarray
    R: np.ndarray
    W: np.ndarray
    p_ray: np.ndarray
    n_kept: int
    n_zeroed: int
    n_holes: int
    n_unlinked: int
    n_lost: int
    alpha: float


def hf_update(g: Geom, c: np.ndarray, alpha0: np.ndarray, freqs: Sequence[float], p_obs: np.ndarray,
              outlier_frac: float = 0.01, eps_rel: float = 1e-3, step: str = "exact") -> UpdateResult:
    """One frequency-set update.  p_obs[nw, e, r] complex; c, alpha0 [ny, nx]."""
    c = np.asarray(c, dtype=np.float64).reshape(g.ny, g.nx)
    F = fields(g, c, alpha0)
    tabs = grid(g, c, alpha0, F)
    E, nvert, lost = rays.trace_endpoints(g, c, alpha0, F)
    lk = link.link(g, E, lost, c)
    nw = len(freqs)
    p_ray = np.stack([link.ray_data(g, lk, f) for f in freqs])
    R = p_ray - p_obs
    base = np.broadcast_to(receiver_mask(g) & lk.linked, R.shape)
    W, n_kept, n_zero = outlier_weights(base, R, outlier_frac)
    g_sum = np.zeros(g.npix)
    h_sum = np.zeros(g.npix)
    for j, f in enumerate(freqs):
        G = green.green(g, tabs, c, f)
        g_sum += np.real(born.born_adjoint(G, W[j] * R[j], f))
        h_sum += born.hess_diag(G, W[j], f)
    sup = support_mask(g).ravel()
    eps = eps_rel * float(np.mean(h_sum[sup]))
    pdir = np.where(sup, -g_sum / (h_sum + eps), 0.0)
    alpha = 1.0
    if step == "exact":
        num = -float(pdir @ g_sum)
        den = 0.0
        for j, f in enumerate(freqs):
            G = green.green(g, tabs, c, f)
            d = born.born_forward(G, pdir, f)
            den += float(np.sum(W[j] * np.abs(d) ** 2))
        alpha = num / den if den > 0.0 else 0.0
    elif step != "diag":
        raise ValueError(step)
    dm = alpha * pdir
    cf = c.ravel()
    dc = -dm * cf ** 3 / (2.0 * g.h * g.h)
    holes = int(np.sum(~tabs.hit[:, sup]))
    return UpdateResult(c_new=(cf + dc).reshape(g.ny, g.nx), dc=dc.reshape(g.ny, g.nx),
                        dc_norm=float(np.sqrt(np.sum(dc[sup] ** 2))), g_sum=g_sum, h_sum=h_sum,
                        R=R, W=W, p_ray=p_ray, n_kept=n_kept, n_zeroed=n_zero, n_holes=holes,
                        n_unlinked=int(np.sum(~lk.linked & receiver_mask(g))), n_lost=int(lost.sum()),
                        alpha=alpha)


def sweep(g: Geom, c0: np.ndarray, alpha0: np.ndarray, freqs: Sequence[float],
          sets: Sequence[Sequence[int]], p_obs_all: np.ndarray, outlier_frac: float = 0.01,
          eps_rel: float = 1e-3, step: str = "exact"):
    """Run every set in order; returns (c_final, [||dc|| per set])."""
    c = np.asarray(c0, dtype=np.float64).reshape(g.ny, g.nx)
    norms: List[float] = []
    for s in sets:
        fs = [freqs[i] for i in s]
        r = hf_update(g, c, alpha0, fs, p_obs_all[list(s)], outlier_frac, eps_rel, step)
        c = r.c_new
        norms.append(r.dc_norm)
    return c, norms


def synth_data(g: Geom, c0: np.ndarray, c_true: np.ndarray, alpha0: np.ndarray, freqs: Sequence[float],
               noise_re: np.ndarray | None = None, noise_im: np.ndarray | None = None,
               level: float = 0.01) -> np.ndarray:
    """p_obs[nw, e, r] from the ray-Born forward model about c0 (see module docstring)."""
    c0 = np.asarray(c0, dtype=np.float64).reshape(g.ny, g.nx)
    ct = np.asarray(c_true, dtype=np.float64).reshape(g.ny, g.nx)
    F = fields(g, c0, alpha0)
    tabs = grid(g, c0, alpha0, F)
    E, nvert, lost = rays.trace_endpoints(g, c0, alpha0, F)
    lk = link.link(g, E, lost, c0)
    sup = support_mask(g).ravel()
    m = np.where(sup, -2.0 * g.h * g.h * (ct - c0).ravel() / c0.ravel() ** 3, 0.0)
    mask = receiver_mask(g)
    out = []
    for j, f in enumerate(freqs):
        G = green.green(g, tabs, c0, f)
        p = link.ray_data(g, lk, f) + born.born_forward(G, m, f)
        if noise_re is not None and level > 0:
            rms = math.sqrt(float(np.mean(np.abs(p[mask]) ** 2)))
            p = p + level * rms * (noise_re[j] + 1j * noise_im[j]) / math.sqrt(2.0)
        out.append(p)
    return np.stack(out)


# ---------------------------------------------------------------------------
# CG variant (Sec. 3: the linear equation of Eq. 10 solved iteratively, as in
# the earlier ray-Born method the paper contrasts with; 10-15 iterations).
#
# Readings: the linearised objective is the one of ``hf_update``,
#   phi(dm) = 1/2 sum_w sum_{e,r} W |R_w + B_w dm|^2  over real dm on the support,
# whose normal equations are  A dm = b,  A = sum_w Re(B_w^H W B_w),  b = -sum_w Re g_w.
# The paper does not say whether its CG is preconditioned; ``precond`` selects the
# plain method (M = I) or the diagonal-Hessian preconditioner M^-1 = 1/(sum_w H_w + eps)
# on the support (the one-step update's solution-space weight), under which a single
# iteration is exactly the one-step update with the exact step.  The iteration is
# Hestenes and Stiefel's conjugate gradients (1952) with a preconditioner, started at 0.
# ---------------------------------------------------------------------------
def cg_solve(apply_A, b: np.ndarray, minv: np.ndarray | None, iters: int):
    """Preconditioned conjugate gradients for A x = b from x = 0.

    apply_A(p) returns A p; minv is the diagonal of M^-1 (None: M = I).  Returns x after
    ``iters`` iterations and the list rho_k = <r_k, M^-1 r_k>, k = 0..iters.  An iteration
    whose curvature <p, A p> is not positive leaves x unchanged from then on."""
    x = np.zeros_like(b, dtype=np.float64)
    r = np.array(b, dtype=np.float64)
    z = r * minv if minv is not None else r.copy()
    p = z.copy()
    rho = float(r @ z)
    hist = [rho]
    for _ in range(iters):
        q = apply_A(p)
        curv = float(p @ q)
        a = rho / curv if curv > 0.0 else 0.0
        x = x + a * p
        r = r - a * q
        z = r * minv if minv is not None else r.copy()
        rho_new = float(r @ z)
        beta = rho_new / rho if rho != 0.0 else 0.0
        p = z + beta * p
        rho = rho_new
        hist.append(rho)
    return x, hist


@dataclasses.dataclass
class CGResult:
    c_new: np.ndarray
    dc: np.ndarray
    dm: np.ndarray
    dc_norm: float
    rho: List[float]
    phi: float            # the linearised objective at dm, minus its value at 0


def cg_update(g: Geom, c: np.ndarray, alpha0: np.ndarray, freqs: Sequence[float], p_obs: np.ndarray, iters: int,
              precond: bool = True, outlier_frac: float = 0.01, eps_rel: float = 1e-3) -> CGResult:
    """One frequency-set update with dm from ``iters`` CG iterations on the normal equations
    of the linearised objective (data, weights and eps exactly as in ``hf_update``)."""
    c = np.asarray(c, dtype=np.float64).reshape(g.ny, g.nx)
    F = fields(g, c, alpha0)
    tabs = grid(g, c, alpha0, F)
    E, nvert, lost = rays.trace_endpoints(g, c, alpha0, F)
    lk = link.link(g, E, lost, c)
    p_ray = np.stack([link.ray_data(g, lk, f) for f in freqs])
    R = p_ray - p_obs
    base = np.broadcast_to(receiver_mask(g) & lk.linked, R.shape)
    W, _, _ = outlier_weights(base, R, outlier_frac)
    Gs = [green.green(g, tabs, c, f) for f in freqs]
    sup = support_mask(g).ravel()
    g_sum = np.zeros(g.npix)
    h_sum = np.zeros(g.npix)
    for j, f in enumerate(freqs):
        g_sum += np.real(born.born_adjoint(Gs[j], W[j] * R[j], f))
        h_sum += born.hess_diag(Gs[j], W[j], f)
    eps = eps_rel * float(np.mean(h_sum[sup]))

    def apply_A(p):
        q = np.zeros(g.npix)
        for j, f in enumerate(freqs):
            q += np.real(born.born_adjoint(Gs[j], W[j] * born.born_forward(Gs[j], p, f), f))
        return np.where(sup, q, 0.0)

    b = np.where(sup, -g_sum, 0.0)
    minv = np.where(sup, 1.0 / (h_sum + eps), 0.0) if precond else None
    dm, hist = cg_solve(apply_A, b, minv, iters)
    phi = 0.5 * float(dm @ apply_A(dm)) - float(b @ dm)
    cf = c.ravel()
    dc = -dm * cf ** 3 / (2.0 * g.h * g.h)
    return CGResult(c_new=(cf + dc).reshape(g.ny, g.nx), dc=dc.reshape(g.ny, g.nx), dm=dm,
                    dc_norm=float(np.sqrt(np.sum(dc[sup] ** 2))), rho=hist, phi=phi)

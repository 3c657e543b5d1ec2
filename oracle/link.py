"""Ray linking: the ray-model data p(c) at the receivers (TEST INFRASTRUCTURE ONLY).

Eq. 8 compares measured data with p_(w,r,e)(c), the pressure "approximated
using the ray-based forward model at receiver r after excitation from
emitter e"; the paper lists ray linking among the method's steps (Sec. 5).
Reading taken here:
  * each ray of fan e ends on the ring at angle vartheta_i = atan2(end) - phi_e,
    wrapped into [0, 2 pi); receiver r sits at vartheta_r = 2 pi ((r-e) mod N_t)/N_t;
  * an interval of neighbouring rays (i, i+1), both reaching the ring, with
    |vartheta_{i+1} - vartheta_i| <= pi (wrap guard), brackets r when
    vartheta_r lies between its ends; T (as a residual against the straight
    water time of the chord), Q and L are interpolated linearly in
    vartheta, kappa is taken from the nearer ray (the lower on a tie);
  * several brackets: the smallest T wins (first arrival), ties to the lowest
    i; none: the pair is unlinked (its data weight is zero);
  * p_ray = G of Eq. 4-5 at x_r with the bilinearly sampled c(x_r).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from .fields import bilinear
from .geometry import Geom, element_angles, element_positions
from .green import green_value
from .rays import VQ, VL, VK, VT, VX, VY


@dataclasses.dataclass
class Links:
    linked: np.ndarray  # [e, r] bool
    T: np.ndarray       # [e, r] traveltime at the receiver
    Q: np.ndarray
    L: np.ndarray
    kappa: np.ndarray
    c_rx: np.ndarray    # [r] sound speed sampled at each receiver
    best: np.ndarray    # [e, r] winning interval i (rays i, i + 1); -1 if unlinked
    lam: np.ndarray     # [e, r] its interpolation weight of ray i + 1


def link(g: Geom, E: np.ndarray, lost: np.ndarray, c: np.ndarray) -> Links:
    n = g.n_elem
    phi = element_angles(g)
    xe, ye = element_positions(g)
    c2 = np.asarray(c, dtype=np.float64).reshape(g.ny, g.nx)
    linked = np.zeros((n, n), dtype=bool)
    T = np.zeros((n, n))
    Q = np.zeros((n, n))
    L = np.zeros((n, n))
    K = np.zeros((n, n), dtype=np.int64)
    BI = np.full((n, n), -1, dtype=np.int64)
    LM = np.zeros((n, n))
    two_pi = 2.0 * math.pi
    for e in range(n):
        ex, ey = E[e, :, VX], E[e, :, VY]
        th = np.mod(np.arctan2(ey, ex) - phi[e], two_pi)
        tres = E[e, :, VT] - np.hypot(ex - xe[e], ey - ye[e]) / g.c_ref
        ok = lost[e] == 0
        a, b = th[:-1], th[1:]
        valid = ok[:-1] & ok[1:] & (np.abs(b - a) <= math.pi)
        lo, hi = np.minimum(a, b), np.maximum(a, b)
        r = np.arange(n)
        thr = two_pi * np.mod(r - e, n) / n                           # [r]
        inside = valid[None, :] & (thr[:, None] >= lo[None, :]) & (thr[:, None] <= hi[None, :])
        den = (b - a)[None, :]
        lam = np.where(den != 0.0, (thr[:, None] - a[None, :]) / np.where(den != 0.0, den, 1.0), 0.0)
        chord = np.hypot(xe - xe[e], ye - ye[e])                       # [r]
        Tr = chord[:, None] / g.c_ref + (1 - lam) * tres[None, :-1] + lam * tres[None, 1:]
        Tm = np.where(inside, Tr, np.inf)
        best = np.argmin(Tm, axis=1)
        has = np.isfinite(Tm[np.arange(n), best])
        lb = lam[np.arange(n), best]
        linked[e] = has
        T[e] = np.where(has, Tm[np.arange(n), best], 0.0)
        q0, q1 = E[e, best, VQ], E[e, best + 1, VQ]
        l0, l1 = E[e, best, VL], E[e, best + 1, VL]
        k0, k1 = E[e, best, VK], E[e, best + 1, VK]
        Q[e] = np.where(has, (1 - lb) * q0 + lb * q1, 0.0)
        L[e] = np.where(has, (1 - lb) * l0 + lb * l1, 0.0)
        K[e] = np.where(has, np.where(lb <= 0.5, k0, k1), 0).astype(np.int64)
        BI[e] = np.where(has, best, -1)
        LM[e] = np.where(has, lb, 0.0)
    c_rx = bilinear(g, c2, xe, ye)
    return Links(linked, T, Q, L, K, c_rx, BI, LM)


def ray_data(g: Geom, links: Links, f_hz: float) -> np.ndarray:
    """p_ray[e, r] for one frequency; zero for unlinked pairs."""
    p = green_value(g, f_hz, links.T, links.Q, links.L, links.kappa, links.c_rx[None, :])
    return np.where(links.linked, p, 0.0)

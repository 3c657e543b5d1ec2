"""Ring, pixel grid and support (TEST INFRASTRUCTURE ONLY, see oracle/__init__.py).

The acquisition is a circular ring of N_t transducers, each one emitter and
receiver (Sec. 4.1: 256 elements on a ring of radius 11 cm).  Readings where
the paper is silent:
  * element t sits at angle phi_t = 2 pi t / N_t, counter-clockwise from +x;
  * pixel (ix, iy) has centre ((ix - (nx-1)/2) h, (iy - (ny-1)/2) h) and flat
    index iy*nx + ix;
  * the support is the disc |x| <= R - margin (margin = max(2 mm, 2 h) unless
    given): the update is zero outside it.  A pixel is inside iff
    (2ix-(nx-1))^2 + (2iy-(ny-1))^2 <= floor((2 (R - margin) / h)^2), an
    integer test that both implementations evaluate identically.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass(frozen=True)
class Geom:
    n_elem: int
    ring_radius: float
    nx: int
    ny: int
    h: float
    n_rays: int
    ds: float
    max_steps: int
    support_margin: float
    c_ref: float
    f_ref: float = 1.0e6
    power_y: float = 1.0

    @property
    def npix(self) -> int:
        return self.nx * self.ny


def from_config(cfg, **over) -> Geom:
    d = dict(n_elem=cfg.n_elem, ring_radius=cfg.ring_radius, nx=cfg.nx, ny=cfg.ny, h=cfg.h,
             n_rays=cfg.n_rays, ds=cfg.ds, max_steps=cfg.max_steps, support_margin=cfg.support_margin,
             c_ref=cfg.c_water, f_ref=1.0e6, power_y=cfg.power_y)
    d.update(over)
    return Geom(**d)


def element_angles(g: Geom) -> np.ndarray:
    return 2.0 * np.pi * np.arange(g.n_elem) / g.n_elem


def element_positions(g: Geom):
    phi = element_angles(g)
    return g.ring_radius * np.cos(phi), g.ring_radius * np.sin(phi)


def pixel_centres(g: Geom):
    x = (np.arange(g.nx) - 0.5 * (g.nx - 1)) * g.h
    y = (np.arange(g.ny) - 0.5 * (g.ny - 1)) * g.h
    return np.meshgrid(x, y)


def r2max(g: Geom) -> int:
    q = 2.0 * (g.ring_radius - g.support_margin) / g.h
    return int(math.floor(q * q))


def support_mask(g: Geom) -> np.ndarray:
    jx = 2 * np.arange(g.nx, dtype=np.int64) - (g.nx - 1)
    jy = 2 * np.arange(g.ny, dtype=np.int64) - (g.ny - 1)
    JX, JY = np.meshgrid(jx, jy)
    return (JX * JX + JY * JY) <= r2max(g)


def receiver_mask(g: Geom) -> np.ndarray:
    """Keep receiver r for emitter e iff the circular index distance is at least
    ceil(N_t/8): the receivers on the opposite ~75 % of the ring (Sec. 4.1)."""
    e = np.arange(g.n_elem)
    d = np.abs(e[:, None] - e[None, :])
    d = np.minimum(d, g.n_elem - d)
    return d >= int(math.ceil(g.n_elem / 8))

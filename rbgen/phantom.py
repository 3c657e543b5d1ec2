"""Seeded sound-speed / absorption phantoms, initial guess and noise draws.

Recipe (stand-ins for the paper's URMC in-vitro and in-vivo data):

* ``ellipses`` (tiny workload): water at 1480 m/s with 3 ellipses whose centres
  are uniform in the disc of radius 0.6 R, semi-axes uniform in 5-15 mm, random
  rotation, speed uniform in 1450-1560 m/s; the whole map is smoothed by a
  Gaussian of sigma = 2 px.  Absorption 0.5 dB/(MHz cm) inside the ellipses
  (same smoothing), 0 in water.
* ``breast`` (256- and 512-grid workloads): a centred breast ellipse with
  semi-axes uniform in 60-85 mm and one fat speed uniform in 1440-1470 m/s; a
  fibroglandular region made of 3-8 smooth blobs inside 0.7x the breast, speed
  1500-1560 m/s; 5-15 lesion ellipses with semi-axes 2-8 mm and speed
  1520-1600 m/s.  Absorption uniform in 0.5-1.0 dB/(MHz^y cm) per tissue class,
  water 0.  Gaussian smoothing of sigma = 2 px.
* Initial guess (stand-in for the paper's three-iteration time-of-flight image):
  c_init = c_w + 0.5 (G_{10 mm} * c_true - c_w).
* Noise: standard-normal draws n1, n2 of shape [n_freq, n_elem, n_elem]; the
  data builder scales them by 1 % of the masked RMS data amplitude.

Every array is float32 (the dtype the CUDA path consumes); pixel (ix, iy) sits
at ((ix - (nx-1)/2) h, (iy - (ny-1)/2) h) and is stored at flat index iy*nx+ix.
"""
from __future__ import annotations

import dataclasses

import numpy as np
from scipy.ndimage import gaussian_filter

from .configs import Config


@dataclasses.dataclass
class Inputs:
    cfg: Config
    c_true: np.ndarray    # [ny, nx] float32, m/s
    alpha0: np.ndarray    # [ny, nx] float32, dB/(MHz^y cm)
    c_init: np.ndarray    # [ny, nx] float32, m/s
    noise_re: np.ndarray  # [n_freq, n_elem, n_elem] float64 standard normal
    noise_im: np.ndarray


def _grid(cfg: Config):
    x = (np.arange(cfg.nx) - (cfg.nx - 1) / 2.0) * cfg.h
    y = (np.arange(cfg.ny) - (cfg.ny - 1) / 2.0) * cfg.h
    return np.meshgrid(x, y)  # X[iy, ix], Y[iy, ix]


def _ellipse(X, Y, cx, cy, a, b, rot):
    cr, sr = np.cos(rot), np.sin(rot)
    u = (X - cx) * cr + (Y - cy) * sr
    v = -(X - cx) * sr + (Y - cy) * cr
    return (u / a) ** 2 + (v / b) ** 2 <= 1.0


def ellipse_phantom(cfg: Config, rng: np.random.Generator):
    X, Y = _grid(cfg)
    c = np.full(X.shape, cfg.c_water)
    a0 = np.zeros(X.shape)
    for _ in range(3):
        r = 0.6 * cfg.ring_radius * np.sqrt(rng.uniform())
        ang = rng.uniform(0, 2 * np.pi)
        a, b = rng.uniform(5e-3, 15e-3, size=2)
        rot = rng.uniform(0, np.pi)
        sp = rng.uniform(1450.0, 1560.0)
        m = _ellipse(X, Y, r * np.cos(ang), r * np.sin(ang), a, b, rot)
        c[m] = sp
        a0[m] = 0.5
    return gaussian_filter(c, 2.0, mode="nearest"), gaussian_filter(a0, 2.0, mode="nearest")


def breast_phantom(cfg: Config, rng: np.random.Generator):
    X, Y = _grid(cfg)
    c = np.full(X.shape, cfg.c_water)
    a0 = np.zeros(X.shape)
    A, B = rng.uniform(60e-3, 85e-3, size=2)
    rot = rng.uniform(0, np.pi)
    breast = _ellipse(X, Y, 0.0, 0.0, A, B, rot)
    fat_c = rng.uniform(1440.0, 1470.0)
    a_fat, a_fib, a_les = rng.uniform(0.5, 1.0, size=3)
    c[breast] = fat_c
    a0[breast] = a_fat
    # fibroglandular: union of smooth blobs inside 0.7x the breast
    fib = np.zeros(X.shape, dtype=bool)
    for _ in range(int(rng.integers(3, 9))):
        rr = 0.7 * np.sqrt(rng.uniform())
        ang = rng.uniform(0, 2 * np.pi)
        cx = rr * A * np.cos(ang) * np.cos(rot) - rr * B * np.sin(ang) * np.sin(rot)
        cy = rr * A * np.cos(ang) * np.sin(rot) + rr * B * np.sin(ang) * np.cos(rot)
        a, b = rng.uniform(8e-3, 25e-3, size=2)
        fib |= _ellipse(X, Y, cx, cy, a, b, rng.uniform(0, np.pi))
    fib &= _ellipse(X, Y, 0.0, 0.0, 0.7 * A, 0.7 * B, rot)
    c[fib] = rng.uniform(1500.0, 1560.0)
    a0[fib] = a_fib
    for _ in range(int(rng.integers(5, 16))):
        rr = 0.8 * np.sqrt(rng.uniform())
        ang = rng.uniform(0, 2 * np.pi)
        cx = rr * A * np.cos(ang) * np.cos(rot) - rr * B * np.sin(ang) * np.sin(rot)
        cy = rr * A * np.cos(ang) * np.sin(rot) + rr * B * np.sin(ang) * np.cos(rot)
        a, b = rng.uniform(2e-3, 8e-3, size=2)
        m = _ellipse(X, Y, cx, cy, a, b, rng.uniform(0, np.pi))
        c[m] = rng.uniform(1520.0, 1600.0)
        a0[m] = a_les
    return gaussian_filter(c, 2.0, mode="nearest"), gaussian_filter(a0, 2.0, mode="nearest")


def initial_guess(cfg: Config, c_true: np.ndarray) -> np.ndarray:
    sig_px = 10e-3 / cfg.h
    sm = gaussian_filter(c_true.astype(np.float64), sig_px, mode="nearest")
    return cfg.c_water + 0.5 * (sm - cfg.c_water)


def noise_draws(cfg: Config, rng: np.random.Generator):
    shape = (len(cfg.freqs_hz), cfg.n_elem, cfg.n_elem)
    return rng.standard_normal(shape), rng.standard_normal(shape)


def make_inputs(cfg: Config) -> Inputs:
    rng = np.random.Generator(np.random.PCG64(cfg.seed))
    if cfg.kind == "ellipses":
        c, a0 = ellipse_phantom(cfg, rng)
    elif cfg.kind == "breast":
        c, a0 = breast_phantom(cfg, rng)
    elif cfg.kind == "water":
        c, a0 = np.full((cfg.ny, cfg.nx), cfg.c_water), np.zeros((cfg.ny, cfg.nx))
    else:
        raise ValueError(cfg.kind)
    ci = initial_guess(cfg, c)
    n1, n2 = noise_draws(cfg, rng)
    return Inputs(cfg, c.astype(np.float32), a0.astype(np.float32), ci.astype(np.float32), n1, n2)

"""Pins for the oracle's Green's function, absorption and dispersion (CPU only).

* Homogeneous medium: the ray Green's function must approach the exact 2-D
  Helmholtz Green's function (i/4) H0^(1)(k r) (SciPy's Hankel routine) with the
  asymptotic error of its leading term, about 1/(8 k r).
* Uniform absorption: amplitude decay exp(-K_a alpha0 f^y r).
* Dispersion: the complex wavenumber  dphi/L + i alpha  must be, up to a term
  linear in w, the boundary value of the function analytic in the upper
  half-plane  i a (-i w)^y / cos(pi y / 2)  (causality, Kramers-Kronig); the
  y = 1 branch must be the limit of the general one.
"""
import math

import numpy as np
import pytest
from scipy.special import hankel1

import rbgen
from oracle import geometry, green, grid


def _homog_tables(c0=1480.0, a0=0.0, **kw):
    cfg = rbgen.tiny(**kw)
    g = geometry.from_config(cfg)
    c = np.full((g.ny, g.nx), c0)
    al = np.full((g.ny, g.nx), a0)
    return g, c, grid.grid(g, c, al)


def test_db_to_neper_constant():
    # 1 dB/cm over 1 cm is an amplitude ratio of 10^(-1/20)
    assert abs(math.exp(-green.K_A * 1.0 * 0.01) - 10 ** (-1 / 20)) < 1e-15


@pytest.mark.parametrize("f", [0.3e6, 0.8e6])
def test_green_matches_hankel_far_field(f):
    g, c, tabs = _homog_tables(n_rays=256)
    G = green.green(g, tabs, c, f)
    xe, ye = geometry.element_positions(g)
    X, Y = geometry.pixel_centres(g)
    k = 2 * math.pi * f / 1480.0
    sup = geometry.support_mask(g).ravel()
    checked = 0
    for t in (0, 9, 40):
        r = np.hypot(X.ravel() - xe[t], Y.ravel() - ye[t])
        sel = sup & (k * r >= 20)
        ex = 0.25j * hankel1(0, k * r[sel])
        rel = np.abs(G[t, sel] / ex - 1.0)
        bound = 1.0 / (8 * k * r[sel]) + 2e-3
        assert np.all(rel <= bound), float(np.max(rel - bound))
        checked += sel.sum()
    assert checked > 1000


def test_uniform_absorption_decay():
    a0, f = 0.6, 0.5e6
    g, c, tabs = _homog_tables(a0=a0, n_rays=256)
    G = green.green(g, tabs, c, f)
    G0 = green.green(g, grid.grid(g, c, np.zeros_like(c)), c, f)
    xe, ye = geometry.element_positions(g)
    X, Y = geometry.pixel_centres(g)
    r = np.hypot(X.ravel() - xe[3], Y.ravel() - ye[3])
    sup = geometry.support_mask(g).ravel() & (r > 5e-3)
    ratio = np.abs(G[3, sup]) / np.abs(G0[3, sup])
    expect = np.exp(-green.K_A * a0 * (f / 1e6) ** g.power_y * r[sup])
    assert np.max(np.abs(ratio / expect - 1)) < 2e-3


@pytest.mark.parametrize("y", [1.05, 1.1, 1.3, 1.5, 1.8])
def test_dispersion_is_causal_power_law(y):
    fr = 1.0e6
    fs = np.array([0.2e6, 0.5e6, 0.9e6, 1.3e6, 2.0e6])
    # dispersion phase per unit absorption integral, and the attenuation, in the same units
    disp = np.array([green.dispersion_phase(f, 1.0, y, fr) for f in fs])
    att = green.K_A * (fs / 1e6) ** y
    w = 2 * np.pi * fs
    a = green.K_A * (2 * np.pi * 1e6) ** (-y)
    K = 1j * a * (-1j * w) ** y / math.cos(math.pi * y / 2)     # analytic in Im w > 0
    assert np.allclose(K.imag, att, rtol=1e-12)
    # real parts agree up to a term linear in w (absorbed in c at f_ref)
    lin = K.real - disp
    slope = lin / w
    assert np.allclose(slope, slope[0], rtol=1e-9)
    assert abs(green.dispersion_phase(fr, 1.0, y, fr)) < 1e-12


def test_dispersion_limits():
    fr = 1.0e6
    for f in (0.3e6, 1.7e6):
        d1 = green.dispersion_phase(f, 2.0, 1.0, fr)
        for eps in (1e-6, -1e-6):
            assert abs(green.dispersion_phase(f, 2.0, 1.0 + eps, fr) - d1) <= 1e-5 * abs(d1)
        assert green.dispersion_phase(f, 0.0, 1.1, fr) == 0.0

"""Pins of the oracle's time-of-flight initial guess (ray-path projection, its
back-projection and the SIRT linearisation)."""
import math

import numpy as np
import pytest

import rbgen
from oracle import geometry as ogeom
from oracle import link as olink
from oracle import rays as orays
from oracle import tof


@pytest.fixture(scope="module")
def water():
    cfg = rbgen.tiny()
    g = ogeom.from_config(cfg)
    c = np.full((g.ny, g.nx), g.c_ref)
    a0 = np.zeros((g.ny, g.nx))
    return cfg, g, c, a0, tof.tof_state(g, c, a0)


def test_straight_ray_integrals(water):
    """Homogeneous medium: rays are straight, so the integral of 1 is the distance from the
    emitter to the ring crossing, and the integral of a linear field is that length times the
    field at the ray's midpoint (bilinear interpolation and the midpoint rule are exact)."""
    cfg, g, c, a0, S = water
    E, nvert, lost = orays.trace_endpoints(g, c, a0)
    xe, ye = ogeom.element_positions(g)
    dist = np.hypot(E[:, :, orays.VX] - xe[:, None], E[:, :, orays.VY] - ye[:, None])
    assert np.all(lost == 0)
    assert np.allclose(S.paths.length, dist, rtol=1e-10, atol=0)
    X, Y = np.meshgrid((np.arange(g.nx) - 0.5 * (g.nx - 1)) * g.h, (np.arange(g.ny) - 0.5 * (g.ny - 1)) * g.h)
    a, bx, by = 6.7e-4, 3e-4, -2e-4
    I = tof.ray_integrals(g, S.paths, a + bx * X + by * Y)
    mx = 0.5 * (E[:, :, orays.VX] + xe[:, None])
    my = 0.5 * (E[:, :, orays.VY] + ye[:, None])
    assert np.allclose(I, dist * (a + bx * mx + by * my), rtol=1e-10, atol=0)


def test_projection_adjoint_identity(water):
    cfg, g, c, a0, S = water
    rows = ogeom.receiver_mask(g) & S.linked
    rng = np.random.default_rng(3)
    s = rng.standard_normal(g.npix)
    d = rng.standard_normal((g.n_elem, g.n_elem))
    lhs = float(np.sum(tof.project(g, S.paths, S.lk, rows, s) * d))
    rhs = float(s @ tof.backproject(g, S.paths, S.lk, rows, d))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_sirt_recovers_uniform_shift_from_linear_data(water):
    """dT = L (ds0 everywhere): every row's mean slowness error is ds0, so one SIRT step
    returns ds0 on every updated pixel."""
    cfg, g, c, a0, S = water
    ds0 = 1.5e-5
    rows = ogeom.receiver_mask(g) & S.linked
    T_obs = S.T + tof.project(g, S.paths, S.lk, rows, np.full(g.npix, ds0))
    ds, rms = tof.sirt_step(g, S, T_obs, S.linked)
    upd = ds != 0.0
    assert upd.sum() >= 0.9 * ogeom.support_mask(g).sum()
    assert np.allclose(ds[upd], ds0, rtol=1e-10, atol=0)
    assert rms > 0.0


def test_water_times_are_chord_times(water):
    cfg, g, c, a0, S = water
    T, linked = tof.tof_times(g, c, a0)
    xe, ye = ogeom.element_positions(g)
    chord = np.hypot(xe[:, None] - xe[None, :], ye[:, None] - ye[None, :])
    rows = ogeom.receiver_mask(g) & linked
    assert np.allclose(T[rows], chord[rows] / g.c_ref, rtol=1e-9, atol=0)


def test_tof_inversion_reduces_misfit():
    cfg = rbgen.tiny()
    g = ogeom.from_config(cfg)
    inp = rbgen.make_inputs(cfg)
    T_obs, obs_linked = tof.tof_times(g, inp.c_true, inp.alpha0)
    c0 = np.full((g.ny, g.nx), g.c_ref)
    c, hist = tof.tof_invert(g, c0, inp.alpha0, T_obs, obs_linked, 3)
    sup = ogeom.support_mask(g)
    e0 = math.sqrt(float(np.mean((c0 - inp.c_true)[sup] ** 2)))
    e3 = math.sqrt(float(np.mean((c - inp.c_true)[sup] ** 2)))
    assert hist[1] < hist[0] and hist[2] < hist[1] and hist[3] < hist[2], hist
    assert e3 < e0, (e0, e3)


def test_projection_is_the_linearised_traveltime(water):
    """A weak smooth slowness perturbation: the change of the linked first-arrival times
    (rays re-traced in the perturbed medium) equals L ds to second order in its amplitude
    (Fermat: the rays' bending changes the times only to second order)."""
    cfg, g, c, a0, S = water
    X, Y = np.meshgrid((np.arange(g.nx) - 0.5 * (g.nx - 1)) * g.h, (np.arange(g.ny) - 0.5 * (g.ny - 1)) * g.h)
    errs = []
    for amp in (2.0, 0.5):
        c1 = c + amp * np.exp(-((X - 0.01) ** 2 + (Y + 0.005) ** 2) / (2 * 0.012 ** 2))
        T1, l1 = tof.tof_times(g, c1, a0)
        rows = ogeom.receiver_mask(g) & S.linked & l1
        dT = np.where(rows, T1 - S.T, 0.0)
        lin = tof.project(g, S.paths, S.lk, rows, (1.0 / c1 - 1.0 / c).ravel())
        errs.append(np.linalg.norm(lin - dT) / np.linalg.norm(dT))
    assert errs[0] <= 2e-3 and errs[1] <= 0.5 * errs[0], errs

"""Pins for the oracle's gridding and ray linking (CPU only).

* Homogeneous medium: no holes in the support, gridded traveltime equal to
  |p - x_t|/c0 within the linear-interpolation bound of the fan triangles,
  J equal to the distance within the same kind of bound.
* Caustic medium: the first-arrival winner at sampled pixels equals a brute
  force over every triangle of the fan (no bounding boxes, no early exits).
* The sampled-pixel tables and Green's functions (the oracle of the full-size GPU
  tests) equal the full ones at the listed pixels, bit for bit.
* Linking: exact reciprocity p[e,r] = p[r,e] in a homogeneous medium (the
  fan geometry is mirror-symmetric), the linked traveltime equal to the chord
  time, and in a heterogeneous medium a reciprocity error that falls as the
  fans are refined.
* Ray data in water: the linked p[e,r] against SciPy's exact 2-D Green's function
  (i/4) H0^(1)(k r) over the chord, within its leading asymptotic error, and the
  uniform-absorption decay along the chord.
* The receiver mask keeps the "opposite 75 %" of the ring the paper uses
  (Sec. 4.1), with the paper's element counts read from tests/golden.
"""
import json
import math
import os

import numpy as np
import pytest

import rbgen
from oracle import geometry, green, grid, link, rays
from oracle.rays import VQ, VT, VX, VY

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "acquisition.json")


def test_homogeneous_grid_coverage_and_traveltime():
    cfg = rbgen.tiny()
    g = geometry.from_config(cfg)
    c0 = 1530.0   # != c_ref so the interpolated residual is non-zero
    c = np.full((g.ny, g.nx), c0)
    tabs = grid.grid(g, c, np.zeros_like(c))
    sup = geometry.support_mask(g).ravel()
    assert tabs.hit[:, sup].all()
    assert not tabs.hit[:, ~sup].any()
    xe, ye = geometry.element_positions(g)
    X, Y = geometry.pixel_centres(g)
    for t in (0, 21, 50):
        D = np.hypot(X.ravel() - xe[t], Y.ravel() - ye[t])[sup]
        T = D / g.c_ref + tabs.t_res[t, sup]
        # |T - D/c0| <= |1/c0 - 1/c_ref| * (interpolation error of D over a triangle);
        # triangles are at most ~ds by the ray spacing pi*D/n_rays, D's Hessian ~ 1/D
        span = np.maximum(g.ds, math.pi * D / g.n_rays) + g.ds
        bound = abs(1 / c0 - 1 / g.c_ref) * span ** 2 / (2 * np.maximum(D - 2 * g.ds, 1e-4)) + 1e-15
        assert np.all(np.abs(T - D / c0) <= bound)
        J = np.abs(tabs.q[t, sup])
        assert np.all(np.abs(J - D) <= span ** 2 / np.maximum(D - 2 * g.ds, 1e-4) + 1e-12)


def _brute_first_arrival(g, V, nvert, t, pix):
    """Smallest interpolated T_res over every triangle containing each pixel."""
    ids, tri = grid.triangles_of_fan(g, V, nvert)
    xe, ye = geometry.element_positions(g)
    X, Y = geometry.pixel_centres(g)
    ax, ay = tri[:, 0, VX], tri[:, 0, VY]
    bx, by = tri[:, 1, VX], tri[:, 1, VY]
    cx, cy = tri[:, 2, VX], tri[:, 2, VY]
    area = (bx - ax) * (cy - ay) - (by - ay) * (cx - ax)
    ok = area != 0
    tres = tri[:, :, VT] - np.hypot(tri[:, :, VX] - xe[t], tri[:, :, VY] - ye[t]) / g.c_ref
    out = []
    for p in pix:
        px, py = X.ravel()[p], Y.ravel()[p]
        with np.errstate(divide="ignore", invalid="ignore"):
            wb = ((px - ax) * (cy - ay) - (py - ay) * (cx - ax)) / area
            wc = ((bx - ax) * (py - ay) - (by - ay) * (px - ax)) / area
        wa = 1 - wb - wc
        inside = ok & (wa >= -1e-12) & (wb >= -1e-12) & (wc >= -1e-12)
        if not inside.any():
            out.append((None, None))
            continue
        tv = wa * tres[:, 0] + wb * tres[:, 1] + wc * tres[:, 2]
        tv = np.where(inside, tv, np.inf)
        j = int(np.argmin(tv))          # first index among equal minima = earliest id
        out.append((tv[j], ids[j]))
    return out


def test_first_arrival_matches_brute_force_in_caustic_medium():
    cfg = rbgen.tiny()
    g = geometry.from_config(cfg)
    X, Y = geometry.pixel_centres(g)
    c = 1480.0 - 300.0 * np.exp(-((X - 0.004) ** 2 + (Y + 0.003) ** 2) / (2 * 0.008 ** 2))
    al = np.zeros_like(c)
    tabs = grid.grid(g, c, al)
    rng = np.random.default_rng(7)
    sup = np.flatnonzero(geometry.support_mask(g).ravel())
    multi = 0
    for t in (0, 13):
        V, nvert, _ = rays.trace_fan(g, c, al, t)
        assert V[:, :, 7].max() >= 1, "fan should cross a caustic"
        pix = rng.choice(sup, 150, replace=False)
        for p, (tv, tid) in zip(pix, _brute_first_arrival(g, V, nvert, t, pix)):
            if tv is None:
                assert not tabs.hit[t, p]
                continue
            assert tabs.hit[t, p]
            assert tabs.tri[t, p] == tid
            assert abs(tabs.t_res[t, p] - tv) <= 1e-18   # residual seconds, rounding level
        multi += 1
    assert multi == 2


def test_sampled_pixel_tables_and_green_equal_the_full_ones():
    """grid_pixels and green(..., pix) (the sampled forms the full-size GPU tests use as
    their oracle) select from the full first-arrival tables exactly: same winner, Q, L,
    kappa, triangle and hole flag at every listed pixel, in the listed order."""
    cfg = rbgen.tiny()
    g = geometry.from_config(cfg)
    X, Y = geometry.pixel_centres(g)
    c = 1480.0 - 300.0 * np.exp(-((X - 0.004) ** 2 + (Y + 0.003) ** 2) / (2 * 0.008 ** 2))
    al = np.zeros_like(c)
    full = grid.grid(g, c, al)
    npix = g.nx * g.ny
    rng = np.random.default_rng(11)
    pix = np.concatenate([[npix - 1, 0], rng.choice(npix, 97, replace=False), [npix // 2, npix // 2]])
    part = grid.grid_pixels(g, c, al, pix)
    assert part.n_lost == full.n_lost
    for name in ("t_res", "q", "l", "kappa", "tri", "hit"):
        assert np.array_equal(getattr(part, name), getattr(full, name)[:, pix]), name
    assert part.hit.any() and not part.hit.all()   # support and outside both sampled
    f = cfg.freqs_hz[0]
    assert np.array_equal(green.green(g, part, c, f, pix=pix), green.green(g, full, c, f)[:, pix])


def test_link_reciprocity_homogeneous_exact():
    cfg = rbgen.tiny()
    g = geometry.from_config(cfg)
    c0 = 1500.0
    c = np.full((g.ny, g.nx), c0)
    al = np.full((g.ny, g.nx), 0.4)
    E, nv, lost = rays.trace_endpoints(g, c, al)
    lk = link.link(g, E, lost, c)
    mask = geometry.receiver_mask(g)
    assert lk.linked[mask].all()
    for f in (0.3e6, 0.5e6):
        p = link.ray_data(g, lk, f)
        assert np.max(np.abs(p - p.T)[mask]) <= 1e-12 * np.max(np.abs(p[mask]))
    xe, ye = geometry.element_positions(g)
    chord = np.hypot(xe[:, None] - xe[None, :], ye[:, None] - ye[None, :])
    # c0 != c_ref: the residual (1/c0 - 1/c_ref) * chord is interpolated linearly in angle
    assert np.max(np.abs(lk.T - chord / c0)[mask] / (chord / c0)[mask]) < 1e-5
    assert np.max(np.abs(lk.Q - chord)[mask] / chord[mask]) < 5e-3
    # c0 == c_ref: the residual vanishes and the chord time is exact
    cw = np.full((g.ny, g.nx), g.c_ref)
    E, nv, lost = rays.trace_endpoints(g, cw, al)
    lk = link.link(g, E, lost, cw)
    assert np.max(np.abs(lk.T - chord / g.c_ref)[mask] / (chord / g.c_ref)[mask]) < 1e-13


def test_link_reciprocity_converges_heterogeneous():
    base = rbgen.tiny()
    inp = rbgen.make_inputs(base)
    errs = []
    for nr in (64, 256):
        g = geometry.from_config(base, n_rays=nr)
        E, nv, lost = rays.trace_endpoints(g, inp.c_true, inp.alpha0)
        lk = link.link(g, E, lost, inp.c_true)
        p = link.ray_data(g, lk, 0.4e6)
        m = geometry.receiver_mask(g) & lk.linked & lk.linked.T
        errs.append(np.sqrt(np.mean(np.abs(p - p.T)[m] ** 2) / np.mean(np.abs(p[m]) ** 2)))
    assert errs[1] < 0.5 * errs[0], errs


def test_receiver_mask_matches_paper_fraction():
    facts = json.load(open(GOLDEN))
    for key in ("in_vitro", "in_vivo_cyst"):
        n = facts[key]["n_elem"]
        g = geometry.Geom(n, 0.11, 8, 8, 1e-3, 8, 5e-4, 10, 2e-3, 1480.0)
        m = geometry.receiver_mask(g)
        frac = m.sum(axis=1) / n
        assert np.all(frac == frac[0])
        assert abs(frac[0] - facts[key]["receiver_fraction_kept"]) < 0.01
        assert np.array_equal(m, m.T)


@pytest.mark.parametrize("f", [0.3e6, 0.8e6])
def test_ray_data_in_water_is_the_hankel_green_function(f):
    """The linked ray data between two elements in homogeneous water must approach the
    exact 2-D Green's function (i/4) H0^(1)(k r) over the chord (SciPy's Hankel routine),
    within the leading asymptotic error 1/(8 k r); with uniform absorption its modulus
    falls by exp(-K_a alpha0 f^y r) along the chord."""
    from scipy.special import hankel1

    cfg = rbgen.tiny(n_rays=256)
    g = geometry.from_config(cfg)
    c = np.full((g.ny, g.nx), g.c_ref)
    mask = geometry.receiver_mask(g)
    xe, ye = geometry.element_positions(g)
    chord = np.hypot(xe[:, None] - xe[None, :], ye[:, None] - ye[None, :])
    k = 2 * math.pi * f / g.c_ref
    out = {}
    for a0 in (0.0, 0.5):
        al = np.full((g.ny, g.nx), a0)
        E, nv, lost = rays.trace_endpoints(g, c, al)
        lk = link.link(g, E, lost, c)
        assert lk.linked[mask].all()
        out[a0] = link.ray_data(g, lk, f)
    ex = 0.25j * hankel1(0, k * chord[mask])
    rel = np.abs(out[0.0][mask] / ex - 1.0)
    assert np.all(rel <= 1.0 / (8 * k * chord[mask]) + 2e-3), float(np.max(rel))
    ratio = np.abs(out[0.5][mask]) / np.abs(out[0.0][mask])
    expect = np.exp(-green.K_A * 0.5 * (f / 1e6) ** g.power_y * chord[mask])
    assert np.max(np.abs(ratio / expect - 1.0)) < 2e-3

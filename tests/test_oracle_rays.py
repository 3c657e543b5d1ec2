"""Pins for the oracle's fields, ray fans and KMAH counting (CPU only).

Each pin comes from outside the oracle: straight rays and closed-form
traveltimes in homogeneous and constant-gradient media (textbook ray
theory), circular ray paths in a constant-gradient medium, and the
ray-tube width Q checked against the finite-difference separation of
neighbouring rays (which does not use the dynamic ray-tracing equations).
"""
import math

import numpy as np
import pytest

import rbgen
from oracle import fields as ofields
from oracle import geometry, rays
from oracle.rays import VK, VL, VQ, VT, VTH, VX, VY


def _geom(**kw):
    cfg = rbgen.tiny()
    return geometry.from_config(cfg, **kw)


def _grid_xy(g):
    X, Y = geometry.pixel_centres(g)
    return X, Y


def test_fields_linear_exact():
    g = _geom()
    X, Y = _grid_xy(g)
    c = 1500.0 + 300.0 * X - 200.0 * Y
    F = ofields.fields(g, c, np.zeros_like(c))
    assert np.allclose(F[1], 300.0, rtol=0, atol=1e-9)
    assert np.allclose(F[2], -200.0, rtol=0, atol=1e-9)
    assert np.allclose(F[3:6], 0.0, atol=1e-6)
    # bilinear sampling reproduces the linear field anywhere inside the grid
    rng = np.random.default_rng(1)
    px, py = rng.uniform(-0.045, 0.045, 50), rng.uniform(-0.045, 0.045, 50)
    v = ofields.bilinear(g, c, px, py)
    assert np.allclose(v, 1500.0 + 300.0 * px - 200.0 * py, rtol=1e-14)


def test_fields_quadratic_interior_exact():
    g = _geom()
    X, Y = _grid_xy(g)
    a, b, cc = 40.0, -25.0, 70.0
    c = 1500.0 + a * X * X + b * X * Y + cc * Y * Y
    F = ofields.fields(g, c, np.zeros_like(c))
    inner = (slice(1, -1), slice(1, -1))
    assert np.allclose(F[3], 2 * a, rtol=1e-8)
    assert np.allclose(F[4][inner], b, rtol=1e-8)
    assert np.allclose(F[5], 2 * cc, rtol=1e-8)
    assert np.allclose(F[1][inner], (2 * a * X + b * Y)[inner], rtol=1e-9, atol=1e-9)


@pytest.mark.parametrize("t", [0, 5, 17])
def test_homogeneous_fan_straight(t):
    """c = c0, alpha0 = a uniform: straight chords, T = chord/c0, Q = arclength,
    L = a * arclength, kappa = 0, exit on the ring where the chord ends."""
    g = _geom()
    c0, a = 1510.0, 0.37
    c = np.full((g.ny, g.nx), c0)
    al = np.full((g.ny, g.nx), a)
    V, nvert, nlost = rays.trace_fan(g, c, al, t)
    assert nlost == 0
    phi = 2 * math.pi * t / g.n_elem
    R = g.ring_radius
    for i in range(g.n_rays):
        psi = -math.pi / 2 + (i + 0.5) * math.pi / g.n_rays
        chord = 2 * R * math.cos(psi)
        end = V[i, nvert[i] - 1]
        ang = phi + math.pi + 2 * psi           # inscribed-angle theorem
        assert abs(end[VX] - R * math.cos(ang)) < 1e-12 * R
        assert abs(end[VY] - R * math.sin(ang)) < 1e-12 * R
        assert abs(end[VT] - chord / c0) < 1e-12 * chord / c0
        assert abs(end[VQ] - chord) < 1e-12 * chord
        assert abs(end[VL] - a * chord) < 1e-12 * a * chord
        assert end[VK] == 0
        # vertex k (inside the ring) lies at arclength k*ds on the chord
        k = nvert[i] // 2
        assert abs(V[i, k, VX] - (R * math.cos(phi) + k * g.ds * math.cos(phi + math.pi + psi))) < 1e-12
        assert nvert[i] == int(math.floor(chord / g.ds - 1e-12)) + 2


def test_constant_gradient_medium_traveltime_and_circle():
    """c = c1 + gy*y: rays are circular arcs and the traveltime between two points is
    (1/|g|) arccosh(1 + g^2 |dx|^2 / (2 c(x1) c(x2))) (textbook closed form)."""
    g = _geom()
    X, Y = _grid_xy(g)
    c1, gy = 1500.0, 600.0
    c = c1 + gy * Y
    al = np.zeros_like(c)
    t = 3
    V, nvert, nlost = rays.trace_fan(g, c, al, t)
    assert nlost == 0
    x0, y0 = V[0, 0, VX], V[0, 0, VY]
    checked = 0
    for i in range(0, g.n_rays, 5):
        n = nvert[i]
        end = V[i, n - 1]
        d2 = (end[VX] - x0) ** 2 + (end[VY] - y0) ** 2
        ca, cb = c1 + gy * y0, c1 + gy * end[VY]
        T = _acosh1p(gy * gy * d2 / (2 * ca * cb)) / abs(gy)
        # the exit vertex is a linear interpolation between two steps: O(ds^2) error
        assert abs(end[VT] - T) < 1e-5 * T
        # interior vertices are RK4 states: O(ds^4)
        for k in range(1, n - 1):
            v = V[i, k]
            d2 = (v[VX] - x0) ** 2 + (v[VY] - y0) ** 2
            Tk = _acosh1p(gy * gy * d2 / (2 * ca * (c1 + gy * v[VY]))) / abs(gy)
            assert abs(v[VT] - Tk) < 1e-9 * Tk
        # circle: horizontal slowness cos(th)/c is conserved; centre on y = -c1/gy
        th0 = V[i, 0, VTH]
        if abs(math.cos(th0)) > 0.05:
            rho = ca / (abs(gy) * abs(math.cos(th0)))
            yc = -c1 / gy
            pts = V[i, 1:n - 1]
            # the centre sits at distance rho along the normal at the source, on the line y = yc;
            # every inner vertex must be at distance rho from it
            nrm = np.array([-math.sin(th0), math.cos(th0)])
            cand = [np.array([x0, y0]) + s * rho * nrm for s in (1.0, -1.0)]
            cen = min(cand, key=lambda q: abs(q[1] - yc))
            assert abs(cen[1] - yc) < 1e-9 * rho
            dist = np.hypot(pts[:, 0] - cen[0], pts[:, 1] - cen[1])
            assert np.max(np.abs(dist / rho - 1.0)) < 1e-10
            checked += 1
    assert checked > 5


def _acosh1p(x):
    """arccosh(1 + x) without the cancellation of forming 1 + x for small x."""
    return math.log1p(x + math.sqrt(x * (x + 2.0)))


def _lens(g, dc=-300.0, sig=0.008, off=(0.004, -0.003)):
    X, Y = _grid_xy(g)
    return 1480.0 + dc * np.exp(-((X - off[0]) ** 2 + (Y - off[1]) ** 2) / (2 * sig * sig))


def _q_vs_fd(g, c, t, rays_idx, tol):
    V, nvert, nlost = rays.trace_fan(g, c, np.zeros_like(c), t)
    assert nlost == 0
    d = math.pi / g.n_rays
    kmax = 0
    for i in rays_idx:
        n = min(nvert[i - 1], nvert[i], nvert[i + 1]) - 1
        ks = np.arange(2, n)
        th = V[i, ks, VTH]
        nrm = np.stack([-np.sin(th), np.cos(th)], axis=1)
        sep = (V[i + 1, ks, :2] - V[i - 1, ks, :2]) / (2 * d)
        qfd = np.sum(sep * nrm, axis=1)
        q = V[i, ks, VQ]
        scale = np.max(np.abs(q))
        assert np.max(np.abs(qfd - q)) < tol * scale
        # KMAH: kappa steps where Q changes sign; away from the zeros it must track
        # the sign changes of the geometric separation
        well = np.abs(qfd) > 0.05 * scale
        flips = np.cumsum(np.r_[0, (np.sign(qfd[1:]) != np.sign(qfd[:-1])).astype(int)])
        kap = V[i, ks, VK]
        assert np.all((kap[well] - flips[well]) == (kap[well][0] - flips[well][0]))
        kmax = max(kmax, int(kap.max()))
    return kmax


def test_Q_matches_neighbour_ray_separation_quadratic_medium():
    """Dynamic ray tracing against geometry: Q(s) equals the normal component of
    (x(psi + d, s) - x(psi - d, s)) / (2 d) up to O(d^2).  The gradient and Hessian
    grids are exact for a quadratic c; only the bilinear c itself is not (an O(h^2)
    inconsistency of about 1e-3 here)."""
    g = _geom(n_rays=2001)
    X, Y = _grid_xy(g)
    c = 1480.0 + 5.0e5 * X * X + 1.0e5 * X * Y + 3.5e5 * Y * Y
    _q_vs_fd(g, c, 0, (600, 1000, 1300, 1500), 2e-3)


def test_Q_matches_neighbour_ray_separation_linear_medium():
    """In a linear medium every grid (c, its gradient, its zero Hessian) is exact, and
    Q still evolves non-trivially through the ray curvature: tight match."""
    g = _geom(n_rays=2001)
    X, Y = _grid_xy(g)
    c = 1480.0 + 2.0e3 * X - 3.0e3 * Y
    _q_vs_fd(g, c, 7, (300, 1000, 1700), 2e-5)


def test_Q_and_kappa_through_a_gaussian_lens():
    """Smooth low-speed lens: Q against neighbouring rays within the O(h^2) mismatch of
    the discrete gradient and Hessian grids, and kappa following the sign changes."""
    g = _geom(n_rays=2001)
    c = _lens(g)
    kmax = _q_vs_fd(g, c, 0, (700, 990, 1040, 1100, 1290), 6e-2)
    assert kmax >= 1


def test_lost_ray_flag():
    g = _geom(max_steps=20)
    c = np.full((g.ny, g.nx), 1480.0)
    V, nvert, nlost = rays.trace_fan(g, c, np.zeros_like(c), 0)
    assert nlost > 0
    assert np.all(nvert <= 21)

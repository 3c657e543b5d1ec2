"""Pins for the oracle's caustic handling: the KMAH phase of Eq. 4 and the KMAH index
the gridding carries (CPU only).

* Phase past a caustic.  Behind a strong low-speed lens the fan of a point source
  folds: inside the caustic three rays reach each point, one of which has touched the
  caustic once (kappa = 1, Q changed sign).  Eq. 3 (the Helmholtz equation for g with a
  point source) is solved here independently by a fourth-order compact finite-difference
  scheme with an absorbing sponge (scipy.sparse LU), checked first against the exact
  Hankel function in water.  The sum of the oracle's ray Green's function
  (green.green_value, Eq. 4-5) over the three arrivals of its own ray fan must match
  that full-wave solution where the arrivals are separated in phase (away from the
  caustic lines, where the geometric sum is not valid).  With a +pi/2 shift per caustic
  instead of -pi/2, or none, the same sum is off by O(1): the pin has the power to tell.
  The first-arrival tables alone cannot pin this phase: a minimum-time ray has passed
  no caustic (a ray beyond a conjugate point is not a minimum of traveltime), so kappa
  reaches the tables only at the odd pixel next to a fold.
* KMAH index of a gridded pixel: the index of the winning triangle's vertex with the
  largest barycentric weight, checked at every covered pixel of every fan in a caustic
  medium, where some winning triangles straddle a caustic (their vertices' indices
  differ, so another vertex choice changes the table).
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spl
from scipy.special import hankel1

import rbgen
from oracle import geometry, green, grid, rays
from oracle.rays import VK, VQ, VT, VX, VY


# --------------------------------------------------------------------------------------
# Independent full-wave solver of Eq. 3: [lap + k^2] g = -delta(x - x_s)
# --------------------------------------------------------------------------------------
def _helmholtz_fd(cfun, f, h, nxh, nyh, src, sponge):
    """Fourth-order compact 9-point scheme (variable k) on the grid x = i h, |i| <= nxh,
    y = j h, |j| <= nyh, with g = 0 on the outer edge and a sponge (k^2 -> k^2 (1 + i s),
    s rising quadratically to 1 over the outer ``sponge`` metres) that absorbs outgoing
    waves.  The scheme, from the PDE's own fourth derivatives:
        D_xx g + D_yy g + h^2/6 D_xx D_yy g + k^2 g + h^2/12 lap_h(k^2 g) = q + h^2/12 lap_h q
    with q = -1/h^2 at the source node.  Returns (x, y, g[ny, nx])."""
    x = h * np.arange(-nxh, nxh + 1)
    y = h * np.arange(-nyh, nyh + 1)
    nx, ny = x.size, y.size
    X, Y = np.meshgrid(x, y)
    k2 = (2.0 * math.pi * f / cfun(X, Y)) ** 2
    ex = np.maximum(0.0, np.abs(X) - (x[-1] - sponge)) / sponge
    ey = np.maximum(0.0, np.abs(Y) - (y[-1] - sponge)) / sponge
    k2 = k2 * (1.0 + 1j * np.maximum(ex, ey) ** 2)
    idx = np.arange(nx * ny).reshape(ny, nx)
    h2 = h * h
    I = idx[1:-1, 1:-1]
    k2c = k2[1:-1, 1:-1]
    rows, cols, vals = [], [], []
    for dj in (-1, 0, 1):
        for di in (-1, 0, 1):
            J = idx[1 + dj:ny - 1 + dj, 1 + di:nx - 1 + di]
            kk = k2[1 + dj:ny - 1 + dj, 1 + di:nx - 1 + di]
            if dj == 0 and di == 0:
                v = -4.0 / h2 + (4.0 / 6.0) / h2 + k2c - (4.0 / 12.0) * k2c
            elif dj == 0 or di == 0:
                v = 1.0 / h2 - (2.0 / 6.0) / h2 + kk / 12.0
            else:
                v = np.full(I.shape, (1.0 / 6.0) / h2)
            rows.append(I.ravel())
            cols.append(J.ravel())
            vals.append(np.asarray(v, dtype=complex).ravel())
    edge = np.ones((ny, nx), bool)
    edge[1:-1, 1:-1] = False
    rows.append(idx[edge])
    cols.append(idx[edge])
    vals.append(np.ones(int(edge.sum()), complex))
    A = sp.csc_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(nx * ny, nx * ny))
    i0 = int(round(src[0] / h)) + nxh
    j0 = int(round(src[1] / h)) + nyh
    assert abs(x[i0] - src[0]) < 1e-12 and abs(y[j0] - src[1]) < 1e-12
    q = np.zeros((ny, nx), complex)
    q[j0, i0] = -1.0 / h2 + (h2 / 12.0) * (-4.0 / h2) * (-1.0 / h2)
    for dj, di in ((0, 1), (0, -1), (1, 0), (-1, 0)):
        q[j0 + dj, i0 + di] += (h2 / 12.0) * (1.0 / h2) * (-1.0 / h2)
    return x, y, spl.spsolve(A, q.ravel()).reshape(ny, nx)


# --------------------------------------------------------------------------------------
# Every arrival of a traced fan at a point (all ray-tube triangles that contain it)
# --------------------------------------------------------------------------------------
def _fan_triangles(V, nvert):
    """Triangles of neighbouring rays (i, i+1) and steps (k, k+1), vertex indices clamped
    at each ray's exit vertex, as vertex records [n, 3, NV]."""
    n_rays = V.shape[0]
    tris = []
    for i in range(n_rays - 1):
        na, nb = int(nvert[i]), int(nvert[i + 1])
        k = np.arange(max(na, nb) - 1)
        A0 = V[i, np.minimum(k, na - 1)]
        A1 = V[i, np.minimum(k + 1, na - 1)]
        B0 = V[i + 1, np.minimum(k, nb - 1)]
        B1 = V[i + 1, np.minimum(k + 1, nb - 1)]
        tris.append(np.stack([A0, B0, B1], 1))
        tris.append(np.stack([A0, B1, A1], 1))
    return np.concatenate(tris)


def _arrivals_on_lattice(tri, xs, ys):
    """Every arrival at the lattice points (xs[a], ys[b]) (uniform spacings): a dict
    (a, b) -> [(T, Q, kappa of the heaviest vertex)] over all triangles holding the point."""
    dx, dy = xs[1] - xs[0], ys[1] - ys[0]
    lo_a = np.ceil((tri[:, :, VX].min(1) - xs[0]) / dx - 1e-9).astype(np.int64)
    hi_a = np.floor((tri[:, :, VX].max(1) - xs[0]) / dx + 1e-9).astype(np.int64)
    lo_b = np.ceil((tri[:, :, VY].min(1) - ys[0]) / dy - 1e-9).astype(np.int64)
    hi_b = np.floor((tri[:, :, VY].max(1) - ys[0]) / dy + 1e-9).astype(np.int64)
    out = {}
    span = int(max(1, (hi_a - lo_a).max(initial=0), (hi_b - lo_b).max(initial=0)))
    for da in range(span + 1):
        for db in range(span + 1):
            a, b = lo_a + da, lo_b + db
            j = np.flatnonzero((a <= hi_a) & (b <= hi_b) & (a >= 0) & (a < xs.size) & (b >= 0) & (b < ys.size))
            if j.size == 0:
                continue
            px, py = xs[a[j]], ys[b[j]]
            t = tri[j]
            ax, ay, bx, by = t[:, 0, VX], t[:, 0, VY], t[:, 1, VX], t[:, 1, VY]
            cx, cy = t[:, 2, VX], t[:, 2, VY]
            area = (bx - ax) * (cy - ay) - (by - ay) * (cx - ax)
            with np.errstate(divide="ignore", invalid="ignore"):
                wb = ((px - ax) * (cy - ay) - (py - ay) * (cx - ax)) / area
                wc = ((bx - ax) * (py - ay) - (by - ay) * (px - ax)) / area
            wa = 1.0 - wb - wc
            ok = (area != 0) & (wa >= -1e-12) & (wb >= -1e-12) & (wc >= -1e-12)
            for q in np.flatnonzero(ok):
                w = np.array([wa[q], wb[q], wc[q]])
                out.setdefault((int(a[j[q]]), int(b[j[q]])), []).append(
                    (float(w @ t[q, :, VT]), float(w @ t[q, :, VQ]), int(t[q, int(np.argmax(w)), VK])))
    return out


def test_fd_solver_reproduces_the_hankel_function_in_water():
    """The full-wave reference itself: in water the FD solution is (i/4) H0^(1)(k r)."""
    f, h = 1.0e6, 1.25e-4
    x, y, u = _helmholtz_fd(lambda X, Y: 1480.0 + 0.0 * X, f, h, 296, 200, (0.03, 0.0), 0.008)
    X, Y = np.meshgrid(x, y)
    r = np.hypot(X - 0.03, Y)
    sel = (np.abs(X) <= 0.027) & (np.abs(Y) <= 0.012) & (r >= 0.015)
    k = 2.0 * math.pi * f / 1480.0
    rel = np.abs(u[sel] / (0.25j * hankel1(0, k * r[sel])) - 1.0)
    # measured: median 0.020, max 0.039 (the scheme's dispersion over up to 40 wavelengths)
    assert np.median(rel) < 0.03 and np.max(rel) < 0.06, (np.median(rel), np.max(rel))


@pytest.mark.slow
def test_kmah_phase_past_a_caustic_matches_the_helmholtz_solution():
    R, f = 0.03, 1.0e6
    sig, dip = 0.006, 400.0          # Gaussian low-speed lens, 1480 -> 1080 m/s at its centre

    def cfun(X, Y):
        return 1480.0 - dip * np.exp(-(X ** 2 + Y ** 2) / (2.0 * sig ** 2))

    # the oracle's ray fan of an element at (R, 0), on a fine grid of the same medium
    hr = 1.0e-4
    n = int(round(2 * R / hr)) + 3
    g = geometry.Geom(4, R, n, n, hr, 2048, hr / 2, int(math.ceil(4 * R / (hr / 2))), 0.002, 1480.0, 1.0e6, 1.0)
    X, Y = geometry.pixel_centres(g)
    c = cfun(X, Y)
    V, nvert, lost = rays.trace_fan(g, c, np.zeros_like(c), 0)
    assert lost == 0 and V[:, :, VK].max() == 1
    tri = _fan_triangles(V, nvert)
    fh = 1.25e-4
    x, y, u = _helmholtz_fd(cfun, f, fh, 296, 200, (R, 0.0), 0.008)
    # observation lattice behind the lens: every third FD node of the window
    ix = np.flatnonzero((x >= -0.027) & (x <= -0.012))[::3]
    jy = np.flatnonzero(np.abs(y) <= 0.006)[::3]
    arrivals = _arrivals_on_lattice(tri, x[ix], y[jy])
    w = 2.0 * math.pi * f
    errs = {"paper": [], "plus": [], "none": []}
    for (a, b), arr in arrivals.items():
        if len(arr) != 3 or sorted(q[2] for q in arr) != [0, 0, 1]:
            continue
        T = sorted(q[0] for q in arr)
        if w * min(T[1] - T[0], T[2] - T[1]) < 1.0:
            continue                 # arrivals about to coalesce at a caustic
        cl = float(cfun(x[ix[a]], y[jy[b]]))
        for key, kap in (("paper", lambda k: k), ("plus", lambda k: -k), ("none", lambda k: 0)):
            s = sum(green.green_value(g, f, q[0], q[1], 0.0, kap(q[2]), cl) for q in arr)
            errs[key].append(abs(s / u[jy[b], ix[a]] - 1.0))
    e = {k: np.array(v) for k, v in errs.items()}
    assert e["paper"].size >= 30, e["paper"].size
    # measured: 46 points, median 0.073 (+pi/2: 1.29, none: 0.87) (FD dispersion and the ray
    # approximation a few wavelengths from the caustic)
    assert np.median(e["paper"]) < 0.15 and np.percentile(e["paper"], 90) < 0.25, e["paper"]
    # the test tells the sign: +pi/2 per caustic, or no shift, misses by O(1)
    assert np.median(e["plus"]) > 0.6 and np.median(e["none"]) > 0.4, (np.median(e["plus"]), np.median(e["none"]))


def test_gridded_kmah_index_is_that_of_the_heaviest_vertex():
    cfg = rbgen.tiny()
    g = geometry.from_config(cfg)
    X, Y = geometry.pixel_centres(g)
    c = 1480.0 - 300.0 * np.exp(-((X - 0.004) ** 2 + (Y + 0.003) ** 2) / (2 * 0.008 ** 2))
    al = np.zeros_like(c)
    tabs = grid.grid(g, c, al)
    KQ = g.max_steps + 1
    Xf, Yf = X.ravel(), Y.ravel()
    straddle = 0
    for t in range(g.n_elem):
        V, nv, _ = rays.trace_fan(g, c, al, t)
        p = np.flatnonzero(tabs.hit[t])
        tid = tabs.tri[t, p]
        half, k, i = tid % 2, (tid // 2) % KQ, (tid // 2) // KQ
        na, nb = nv[i], nv[i + 1]
        A0, A1 = V[i, np.minimum(k, na - 1)], V[i, np.minimum(k + 1, na - 1)]
        B0, B1 = V[i + 1, np.minimum(k, nb - 1)], V[i + 1, np.minimum(k + 1, nb - 1)]
        P = [A0, np.where(half[:, None] == 0, B0, B1), np.where(half[:, None] == 0, B1, A1)]
        ax, ay, bx, by, cx, cy = P[0][:, VX], P[0][:, VY], P[1][:, VX], P[1][:, VY], P[2][:, VX], P[2][:, VY]
        area = (bx - ax) * (cy - ay) - (by - ay) * (cx - ax)
        wb = ((Xf[p] - ax) * (cy - ay) - (Yf[p] - ay) * (cx - ax)) / area
        wc = ((bx - ax) * (Yf[p] - ay) - (by - ay) * (Xf[p] - ax)) / area
        Wt = np.stack([1.0 - wb - wc, wb, wc], 1)
        K = np.stack([P[0][:, VK], P[1][:, VK], P[2][:, VK]], 1)
        rows = np.arange(p.size)
        heavy = K[rows, np.argmax(Wt, 1)]
        assert np.array_equal(tabs.kappa[t, p], heavy.astype(np.int64)), t
        straddle += int(np.sum(heavy != K[rows, np.argmin(Wt, 1)]))
    # some winners straddle a caustic with the heaviest and the lightest vertex on
    # different sides of it, so the vertex choice is exercised
    assert straddle >= 5, straddle

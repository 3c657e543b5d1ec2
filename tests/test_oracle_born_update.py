"""Pins for the oracle's Born operators, data weights and one-step update (CPU only).

* Adjoint identity <B m, S> = <m, B* S> to 1e-12 for complex m and data.
* Brute force on small grids: B applied to every unit vector gives
  w^2 G_e(x_j) G_r(x_j); the Hessian diagonal equals ||W^(1/2) B e_j||^2; the
  gradient equals central finite differences of 1/2 ||W^(1/2)(B m + R)||^2.
* The Born data of a weak smooth perturbation equal the first-order change of the
  linked ray data (central difference of p(c) at c0 +- dc) to 2 %.
* One-step update on a support of a few pixels equals, pixel by pixel, the
  least-squares solution (numpy.linalg.lstsq) of that 1-unknown problem, damped by
  H_j / (H_j + eps) with eps from the mean of H over the support (eps_rel 0 and 0.5).
* Outlier zeroing: invariants of a top-k selection and its tie rule.
* Sweep (no printed values exist to match): the true medium is a fixed point under
  its own noise-free data (zero residual, zero update, in every set); on noise-free
  data the error to the phantom falls set by set, each set seeded by the last.
"""
import math

import numpy as np
import pytest

import rbgen
from oracle import born, geometry, green, grid, update


def _small_problem(n_elem=12, n=10, seed=3):
    rng = np.random.default_rng(seed)
    G = (rng.standard_normal((n_elem, n * n)) + 1j * rng.standard_normal((n_elem, n * n))) * 1e-2
    return rng, G


def test_adjoint_identity_complex():
    rng, G = _small_problem()
    f = 0.4e6
    m = rng.standard_normal(G.shape[1]) + 1j * rng.standard_normal(G.shape[1])
    S = rng.standard_normal((12, 12)) + 1j * rng.standard_normal((12, 12))
    lhs = np.vdot(born.born_forward(G, m, f), S)                  # <B m, S>
    rhs = np.vdot(m, born.born_adjoint(G, S, f))                  # <m, B* S>
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_adjoint_identity_real_m_on_ray_tables():
    cfg = rbgen.tiny()
    g = geometry.from_config(cfg)
    inp = rbgen.make_inputs(cfg)
    tabs = grid.grid(g, inp.c_init, inp.alpha0)
    G = green.green(g, tabs, inp.c_init, 0.4e6)
    rng = np.random.default_rng(0)
    m = rng.standard_normal(g.npix)
    S = rng.standard_normal((g.n_elem, g.n_elem)) + 1j * rng.standard_normal((g.n_elem, g.n_elem))
    lhs = np.real(np.vdot(born.born_forward(G, m, 0.4e6), S))
    rhs = float(m @ np.real(born.born_adjoint(G, S, 0.4e6)))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_brute_force_columns_hessian_and_gradient():
    rng, G = _small_problem(n_elem=8, n=8)
    f = 0.3e6
    w = 2 * math.pi * f
    npix = G.shape[1]
    W = (rng.uniform(size=(8, 8)) > 0.3).astype(np.uint8)
    R = rng.standard_normal((8, 8)) + 1j * rng.standard_normal((8, 8))
    Bcols = []
    for j in range(npix):
        e = np.zeros(npix)
        e[j] = 1.0
        d = born.born_forward(G, e, f)
        assert np.allclose(d, w * w * np.outer(G[:, j], G[:, j]), rtol=1e-13, atol=0)
        Bcols.append(d)
    H = born.hess_diag(G, W, f)
    Hb = np.array([np.sum(W * np.abs(b) ** 2) for b in Bcols])
    assert np.allclose(H, Hb, rtol=1e-12)
    # gradient of F(m) = 1/2 sum W |R + B m|^2 at m = 0 by central differences
    gr = np.real(born.born_adjoint(G, W * R, f))
    F = lambda m: 0.5 * np.sum(W * np.abs(R + born.born_forward(G, m, f)) ** 2)
    hstep = 1e-3 / (w * w * 1e-4)
    for j in (0, 17, 40, 63):
        e = np.zeros(npix)
        e[j] = hstep
        fd = (F(e) - F(-e)) / (2 * hstep)
        assert abs(fd - gr[j]) <= 1e-7 * (abs(gr[j]) + 1e-30) + 1e-9 * np.max(np.abs(gr))


@pytest.mark.parametrize("eps_rel", [0.0, 0.5])
def test_one_step_single_pixel_equals_least_squares(eps_rel):
    """On a support of a few pixels the diagonal step of each pixel is that pixel's own
    least-squares solution (numpy.linalg.lstsq over its brute-force Born column), damped
    by the solution-space weight's eps: dm_j = dm_ls_j H_j / (H_j + eps), with
    H_j = ||W^(1/2) b_j||^2 from the same column and eps = eps_rel x the mean of H over
    the support pixels (not over the whole grid, where H is zero outside the support)."""
    cfg = rbgen.tiny()
    # margin so large that the support holds the 4 central pixels only
    g = geometry.from_config(cfg, support_margin=cfg.ring_radius - 1.2 * cfg.h)
    sup = geometry.support_mask(g).ravel()
    assert 2 <= sup.sum() <= 4
    inp = rbgen.make_inputs(cfg)
    rng = np.random.default_rng(5)
    fr = [0.3e6, 0.35e6]
    p_obs = 0.01 * (rng.standard_normal((2, g.n_elem, g.n_elem)) + 1j * rng.standard_normal((2, g.n_elem, g.n_elem)))
    r = update.hf_update(g, inp.c_init, inp.alpha0, fr, p_obs, outlier_frac=0.0, eps_rel=eps_rel, step="diag")
    # least squares for each support pixel alone: min_dm sum_w ||W^(1/2) (R_w + b_w dm)||^2
    tabs = grid.grid(g, inp.c_init, inp.alpha0)
    dm_ls, hj = {}, {}
    for j in np.flatnonzero(sup):
        rows, rhs = [], []
        for k, f in enumerate(fr):
            G = green.green(g, tabs, inp.c_init, f)
            b = (2 * math.pi * f) ** 2 * np.outer(G[:, j], G[:, j])
            sw = np.sqrt(r.W[k].astype(float))
            rows += [(sw * b).real.ravel(), (sw * b).imag.ravel()]
            rhs += [-(sw * r.R[k]).real.ravel(), -(sw * r.R[k]).imag.ravel()]
        A = np.concatenate(rows)[:, None]
        y = np.concatenate(rhs)
        dm_ls[j] = np.linalg.lstsq(A, y, rcond=None)[0][0]
        hj[j] = float(A[:, 0] @ A[:, 0])
    eps = eps_rel * np.mean(list(hj.values()))
    for j in dm_ls:
        dm = r.dc.ravel()[j] * (-2 * g.h * g.h) / np.asarray(inp.c_init, float).ravel()[j] ** 3
        # with several support pixels the diagonal step for pixel j is still that pixel's
        # own least-squares solution (off-diagonal couplings are ignored by construction)
        expect = dm_ls[j] * hj[j] / (hj[j] + eps)
        assert abs(dm - expect) <= 1e-10 * abs(expect)


def test_outlier_selection_invariants_and_ties():
    rng = np.random.default_rng(11)
    base = rng.uniform(size=(3, 16, 16)) > 0.2
    R = rng.standard_normal((3, 16, 16)) + 1j * rng.standard_normal((3, 16, 16))
    W, n, k = update.outlier_weights(base, R, 0.05)
    assert n == base.sum() and k == int(math.floor(0.05 * n))
    zeroed = base & (W == 0)
    assert zeroed.sum() == k
    kept = base & (W == 1)
    assert np.abs(R[zeroed]).min() >= np.abs(R[kept]).max()
    # ties: equal magnitudes go by smallest flat index
    R2 = np.ones((2, 4, 4), dtype=complex)
    b2 = np.ones((2, 4, 4), dtype=bool)
    W2, n2, k2 = update.outlier_weights(b2, R2, 0.1)
    assert k2 == 3
    assert list(np.flatnonzero(W2.ravel() == 0)) == [0, 1, 2]


@pytest.mark.parametrize("step", ["exact", "diag"])
def test_sweep_smoke_noise_free(step):
    cfg = rbgen.tiny()
    g = geometry.from_config(cfg)
    inp = rbgen.make_inputs(cfg)
    p = update.synth_data(g, inp.c_init, inp.c_true, inp.alpha0, cfg.freqs_hz, level=0.0)
    sup = geometry.support_mask(g)
    e0 = np.sqrt(np.mean((inp.c_init.astype(float) - inp.c_true)[sup] ** 2))
    r = update.hf_update(g, inp.c_init, inp.alpha0, [cfg.freqs_hz[0]], p[[0]], 0.0, 1e-3, step)
    assert np.isfinite(r.dc_norm)
    e1 = np.sqrt(np.mean((r.c_new - inp.c_true)[sup] ** 2))
    corr = np.sum(r.dc[sup] * (inp.c_true - inp.c_init)[sup])
    assert corr > 0          # the step points toward the truth
    if step == "exact":
        assert e1 < e0


def test_sweep_true_medium_is_a_fixed_point():
    """Noise-free data made about the true medium leave it unchanged through the whole
    sweep: every set's residual vanishes, so its gradient and update do (Eqs. 8-10).
    The same data handed to the sets in the wrong frequency order move it."""
    cfg = rbgen.tiny()
    g = geometry.from_config(cfg)
    inp = rbgen.make_inputs(cfg)
    p = update.synth_data(g, inp.c_true, inp.c_true, inp.alpha0, cfg.freqs_hz, level=0.0)
    c, norms = update.sweep(g, inp.c_true, inp.alpha0, cfg.freqs_hz, cfg.sets, p)
    assert norms == [0.0] * len(cfg.sets)
    assert np.array_equal(c, inp.c_true.reshape(g.ny, g.nx).astype(np.float64))
    # planted mistake: each set sees the data of the next frequency
    c_bad, norms_bad = update.sweep(g, inp.c_true, inp.alpha0, cfg.freqs_hz, cfg.sets, np.roll(p, 1, axis=0))
    assert min(norms_bad) > 0.0


def test_sweep_error_falls_set_by_set():
    """On noise-free data the image after each set is closer to the phantom than the one
    that seeded it (the sweep's low-to-high refinement, Secs. 3-4): each set starts from
    the previous set's image, so seeding every set from the start image would fail."""
    cfg = rbgen.tiny()
    g = geometry.from_config(cfg)
    inp = rbgen.make_inputs(cfg)
    p = update.synth_data(g, inp.c_init, inp.c_true, inp.alpha0, cfg.freqs_hz, level=0.0)
    sup = geometry.support_mask(g)
    ct = inp.c_true.reshape(g.ny, g.nx)
    errs = [np.sqrt(np.mean((inp.c_init.reshape(g.ny, g.nx) - ct)[sup] ** 2))]
    for k in range(1, len(cfg.sets) + 1):
        c, norms = update.sweep(g, inp.c_init, inp.alpha0, cfg.freqs_hz, cfg.sets[:k], p)
        assert len(norms) == k and all(n > 0 for n in norms)
        errs.append(np.sqrt(np.mean((c - ct)[sup] ** 2)))
    assert all(b < 0.9 * a for a, b in zip(errs, errs[1:])), errs
    # the last set alone, from the start image, lands further from the phantom
    last, _ = update.sweep(g, inp.c_init, inp.alpha0, cfg.freqs_hz, cfg.sets[-1:], p)
    assert np.sqrt(np.mean((last - ct)[sup] ** 2)) > errs[-1] * 1.2


def test_born_forward_is_the_first_order_change_of_the_ray_data():
    """Sec. 1 / Eq. 10: the Born data of a weak, smooth perturbation dc (m = -2 h^2 dc / c^3,
    d = w^2 sum_x G_e G_r m) must equal the first-order change of the ray-model data p(c)
    of Eq. 8, here the central difference of the linked ray data at c0 +- dc.  The two
    sides share no code (Green's function tables and the Born sum against traced and
    linked rays), so the scaling, sign and phase convention of m and of B are pinned.
    A 12 mm Gaussian at 0.3 MHz (wavelength 4.9 mm, 3 pixels per wavelength) agrees to
    0.5 %; the bar is 2 %."""
    from oracle import link, rays
    cfg = rbgen.tiny(n_rays=256)
    g = geometry.from_config(cfg)
    X, Y = geometry.pixel_centres(g)
    sup = geometry.support_mask(g)
    c0 = np.full((g.ny, g.nx), g.c_ref)
    al = np.zeros_like(c0)
    dc = np.exp(-((X - 0.005) ** 2 + (Y + 0.008) ** 2) / (2 * 0.012 ** 2)).reshape(g.ny, g.nx)
    dc = np.where(sup, dc, 0.0)          # 1 m/s peak
    f = 0.3e6
    ps = []
    for c in (c0 - dc, c0 + dc):
        E, nv, lost = rays.trace_endpoints(g, c, al)
        lk = link.link(g, E, lost, c)
        ps.append(link.ray_data(g, lk, f))
    dp = (ps[1] - ps[0]) / 2.0
    G = green.green(g, grid.grid(g, c0, al), c0, f)
    m = np.where(sup.ravel(), -2.0 * g.h * g.h * dc.ravel() / c0.ravel() ** 3, 0.0)
    d = born.born_forward(G, m, f)
    mask = geometry.receiver_mask(g)
    err = np.linalg.norm((d - dp)[mask]) / np.linalg.norm(dp[mask])
    assert err < 0.02, err

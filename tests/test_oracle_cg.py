"""Pins of the oracle's CG variant (conjugate gradients on the normal equations of the
linearised objective of Eq. 10).

* Krylov optimality (the defining property of CG, checked without its recurrences): after
  k iterations from 0, x_k minimises 1/2 x^T A x - b^T x over the Krylov space
  span{z0, (M^-1 A) z0, ..., (M^-1 A)^(k-1) z0}, z0 = M^-1 b; the minimiser is computed by
  projecting onto an orthonormal basis of that space built independently (Arnoldi).
* Finite termination: with as many iterations as unknowns (plus a few), x solves A x = b.
* The one-step update is the first preconditioned iteration: cg_update with one iteration
  and the diagonal-Hessian preconditioner gives hf_update's exact-step dc.
* Monotonicity: the linearised objective decreases with every iteration.
"""
import numpy as np
import pytest

import rbgen
from oracle import geometry as ogeom
from oracle import update as oupd


def _normal_system(n_data, n_unk, seed):
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((n_data, n_unk)) + 1j * rng.standard_normal((n_data, n_unk))
    W = (rng.uniform(size=n_data) > 0.2).astype(np.float64)
    A = np.real(B.conj().T @ (W[:, None] * B))
    b = rng.standard_normal(n_unk)
    minv = rng.uniform(0.5, 2.0, size=n_unk)
    return A, b, minv


def _krylov_min(A, b, minv, k):
    n = len(b)
    mi = minv if minv is not None else np.ones(n)
    V = np.zeros((n, k))
    v = mi * b
    for j in range(k):
        for _ in range(2):
            v = v - V[:, :j] @ (V[:, :j].T @ v)
        V[:, j] = v / np.linalg.norm(v)
        v = mi * (A @ V[:, j])
    y = np.linalg.solve(V.T @ A @ V, V.T @ b)
    return V @ y


@pytest.mark.parametrize("pre", [False, True])
def test_cg_krylov_optimality(pre):
    A, b, minv = _normal_system(48, 20, 11)
    mv = minv if pre else None
    for k in range(1, 7):
        x, hist = oupd.cg_solve(lambda p: A @ p, b, mv, k)
        xs = _krylov_min(A, b, mv, k)
        assert np.linalg.norm(x - xs) <= 1e-8 * np.linalg.norm(xs), k
        assert len(hist) == k + 1


@pytest.mark.parametrize("pre", [False, True])
def test_cg_finite_termination(pre):
    A, b, minv = _normal_system(60, 12, 12)
    x, hist = oupd.cg_solve(lambda p: A @ p, b, minv if pre else None, 16)
    xs = np.linalg.solve(A, b)
    assert np.linalg.norm(x - xs) <= 1e-8 * np.linalg.norm(xs)
    assert hist[12] <= 1e-16 * hist[0]


def _tiny_problem():
    cfg = rbgen.tiny()
    inp = rbgen.make_inputs(cfg)
    g = ogeom.from_config(cfg)
    freqs = [cfg.freqs_hz[1]]
    p_obs = oupd.synth_data(g, inp.c_init, inp.c_true, inp.alpha0, freqs, inp.noise_re, inp.noise_im)
    return g, inp, freqs, p_obs


def test_cg_first_iteration_is_the_one_step_update():
    g, inp, freqs, p_obs = _tiny_problem()
    one = oupd.hf_update(g, inp.c_init, inp.alpha0, freqs, p_obs, step="exact")
    cg = oupd.cg_update(g, inp.c_init, inp.alpha0, freqs, p_obs, 1, precond=True)
    assert np.linalg.norm(cg.dc - one.dc) <= 1e-10 * np.linalg.norm(one.dc)
    assert cg.dc_norm == pytest.approx(one.dc_norm, rel=1e-10)


def test_cg_objective_decreases():
    g, inp, freqs, p_obs = _tiny_problem()
    for pre in (True, False):
        phis = [oupd.cg_update(g, inp.c_init, inp.alpha0, freqs, p_obs, k, precond=pre).phi for k in (1, 2, 4)]
        assert phis[0] < 0.0
        assert phis[1] < phis[0] and phis[2] < phis[1], (pre, phis)


def test_scalar_preconditioner_leaves_the_iterates_unchanged():
    """Plain CG on the GPU runs with the scalar preconditioner 1/(mean H + eps) to keep A p
    inside the FP32 range; a scalar M scales r, z and p but not the iterates x_k, so it is
    plain CG.  (Checked on a well-conditioned system, where rounding stays small.)"""
    A, b, _ = _normal_system(48, 20, 13)
    for k in (1, 3, 6):
        x_plain, h_plain = oupd.cg_solve(lambda p: A @ p, b, None, k)
        x_scal, h_scal = oupd.cg_solve(lambda p: A @ p, b, np.full(len(b), 3.7e-9), k)
        assert np.allclose(x_scal, x_plain, rtol=1e-9, atol=0), k
        assert np.allclose(np.array(h_scal) / h_scal[0], np.array(h_plain) / h_plain[0], rtol=1e-9)

"""GPU-vs-oracle parity through the C-ABI (needs a CUDA GPU).

Same seeded inputs on both sides; the oracle is the FP64 CPU code in oracle/.
Tolerances (spec bounds, plus readings for the tables):
  * ray endpoints and traveltimes: 1e-6 relative for every ray that crosses
    the ring at sin(beta) >= 0.1 from tangency; grazing rays, whose crossing
    is ill-conditioned, 1e-6 / sin(beta) (at most 1e-4);
  * gridded tables: T within 1e-6 relative of the total traveltime, Q and L
    within 1e-5 of their scale, on pixels where both sides pick the same
    triangle; pixels whose first-arrival winner or coverage differs (caustic
    switches, edge pixels) must stay under 0.1 %;
  * Green's functions, ray data, Born data and gradients: 1e-4 relative L2
    (plain FP32 path);
  * the sound-speed map after a full sweep: 0.05 m/s RMS.
"""
import math

import numpy as np
import pytest

import rbgen
from oracle import born as oborn
from oracle import geometry as ogeom
from oracle import green as ogreen
from oracle import grid as ogrid
from oracle import link as olink
from oracle import rays as orays
from oracle import update as oupd
from oracle.rays import VK, VL, VQ, VT, VTH, VX, VY

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2511_16633_gb300 import rb  # noqa: E402


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rb.load()
    return torch.device("cuda:0")


def _t(a, dev, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a), device=dev).to(dtype).contiguous()


def rel_l2(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


def gpu_ends(geom, c, a0, dev, samples=False):
    ws = rb.workspace(geom, 1, rb.RB_PREC_FP32, dev)
    ends = torch.zeros((geom.n_elem, geom.n_rays, 56), dtype=torch.uint8, device=dev)
    smp = None
    if samples:
        shp = (geom.n_elem, geom.n_rays, geom.max_steps + 1)
        smp = dict(vx=torch.zeros(shp, device=dev), vy=torch.zeros(shp, device=dev),
                   vt=torch.zeros(shp, dtype=torch.float64, device=dev), vq=torch.zeros(shp, device=dev),
                   vl=torch.zeros(shp, device=dev), vkappa=torch.zeros(shp, dtype=torch.int32, device=dev))
    rb.rb_trace_rays(geom, _t(c, dev), _t(a0, dev), ends, ws, smp)
    torch.cuda.synchronize()
    out = rb.decode_ends(ends)
    if samples:
        return out, {k: v.cpu().numpy() for k, v in smp.items()}
    return out


def gpu_tables(geom, c, a0, dev, freqs=None):
    ws = rb.workspace(geom, 1, rb.RB_PREC_FP32, dev)
    npix = geom.nx * geom.ny
    tab = torch.empty((geom.n_elem, npix, 4), dtype=torch.int32, device=dev)
    g_out = None
    if freqs:
        g_out = torch.empty((len(freqs), geom.n_elem, npix), dtype=torch.complex64, device=dev)
    rb.rb_green_grid(geom, _t(c, dev), _t(a0, dev), tab, ws, freqs, g_out)
    torch.cuda.synchronize()
    return tab, (g_out.cpu().numpy() if g_out is not None else None)


CASES = {
    "tiny_init": lambda: (rbgen.tiny(), "c_init"),
    "tiny_true": lambda: (rbgen.tiny(), "c_true"),
    "tiny_ragged": lambda: (rbgen.tiny(n_rays=45, nx=70, ny=66, n_elem=40), "c_true"),
}


def _case(name):
    cfg, which = CASES[name]()
    inp = rbgen.make_inputs(rbgen.tiny(seed=cfg.seed)) if (cfg.nx, cfg.ny) == (64, 64) else None
    if inp is None:
        base = rbgen.make_inputs(rbgen.tiny(nx=cfg.nx, ny=cfg.ny, seed=cfg.seed))
        inp = base
    c = getattr(inp, which)
    return cfg, inp, c


@pytest.mark.parametrize("case", list(CASES))
def test_ray_endpoints(dev, case):
    cfg, inp, c = _case(case)
    g = ogeom.from_config(cfg)
    geom = rb.geometry_from_config(cfg)
    E, nv, lost = orays.trace_endpoints(g, c, inp.alpha0)
    G = gpu_ends(geom, c, inp.alpha0, dev)
    assert lost.sum() == 0
    ok = G["n_vert"] == nv
    assert ok.mean() >= 0.999, f"vertex counts differ on {np.sum(~ok)} rays"
    R = cfg.ring_radius
    dpos = np.hypot(G["x"] - E[..., VX], G["y"] - E[..., VY]) / R
    relT = np.abs(G["t"] - E[..., VT]) / E[..., VT]
    # The crossing of a ray with the ring is ill-conditioned when the ray meets the ring
    # almost tangentially: a position difference d moves the crossing by d / sin(beta),
    # beta the angle to the tangent.  The 1e-6 bound applies to every ray crossing at
    # sin(beta) >= 0.1 (all rays that can bracket a receiver kept by the 75 % mask);
    # grazing rays (the outermost rays of each fan) get 1e-6 / sin(beta), capped at 1e-4.
    sinb = np.abs(np.cos(E[..., VTH]) * E[..., VX] + np.sin(E[..., VTH]) * E[..., VY]) / R
    well = sinb >= 0.1
    assert well.mean() > 0.9
    assert np.max(dpos[well]) <= 1e-6, np.max(dpos[well])
    assert np.max(relT[well]) <= 1e-6, np.max(relT[well])
    bound = np.minimum(1e-6 / np.maximum(sinb, 1e-12), 1e-4)
    assert np.all(relT[~well] <= bound[~well]), np.max(relT[~well] / bound[~well])
    assert np.all(dpos[~well] <= bound[~well])
    qs = np.max(np.abs(E[..., VQ]))
    assert np.max(np.abs(G["q"] - E[..., VQ])) <= 1e-5 * qs
    ls = max(np.max(np.abs(E[..., VL])), 1e-12)
    assert np.max(np.abs(G["l"] - E[..., VL])) <= 1e-5 * ls
    assert np.mean(G["kappa"] == E[..., VK]) >= 0.999


def test_ray_samples(dev):
    cfg, inp, c = _case("tiny_true")
    g = ogeom.from_config(cfg)
    geom = rb.geometry_from_config(cfg)
    ends, S = gpu_ends(geom, c, inp.alpha0, dev, samples=True)
    worst = 0.0
    for t in (0, 7, 33):
        V, nv, _ = orays.trace_fan(g, c, inp.alpha0, t)
        for i in range(0, g.n_rays, 3):
            n = min(nv[i], ends["n_vert"][t, i])
            # interior vertices (the exit vertex is covered, with its conditioning, by the endpoint test)
            T = V[i, 1:n - 1, VT]
            worst = max(worst, float(np.max(np.abs(S["vt"][t, i, 1:n - 1] - T) / T)))
            # vertex positions are stored as float: allow their rounding (half an ulp of R)
            assert np.max(np.hypot(S["vx"][t, i, :n] - V[i, :n, VX], S["vy"][t, i, :n] - V[i, :n, VY])) <= 1e-6 * g.ring_radius
            assert np.array_equal(S["vkappa"][t, i, :n], V[i, :n, VK].astype(np.int32))
    assert worst <= 1e-6, worst


def _table_parity(cfg, inp, c, dev, tab, ot):
    g = ogeom.from_config(cfg)
    d = rb.decode_tables(tab)
    sup = ogeom.support_mask(g).ravel()
    hit_diff = d["hit"][:, sup] != ot.hit[:, sup]
    both = d["hit"] & ot.hit & sup[None, :]
    same_tri = both & (d["tri"] == ot.tri)
    frac_bad = (hit_diff.sum() + (both & ~same_tri).sum()) / (g.n_elem * sup.sum())
    Ttot = ogreen.gridded_traveltime(g, ot)
    dT = np.abs(d["t_res"] - ot.t_res)[same_tri] / Ttot[same_tri]
    qs = np.max(np.abs(ot.q))
    ls = max(np.max(np.abs(ot.l)), 1e-12)
    return dict(frac_bad=frac_bad, dT=float(np.max(dT)),
                dq=float(np.max(np.abs(d["q"] - ot.q)[same_tri]) / qs),
                dl=float(np.max(np.abs(d["l"] - ot.l)[same_tri]) / ls),
                kap=float(np.mean((d["kappa"] == ot.kappa)[same_tri])))


@pytest.mark.parametrize("case", list(CASES))
def test_tables(dev, case):
    cfg, inp, c = _case(case)
    g = ogeom.from_config(cfg)
    geom = rb.geometry_from_config(cfg)
    tab, _ = gpu_tables(geom, c, inp.alpha0, dev)
    ot = ogrid.grid(g, c, inp.alpha0)
    r = _table_parity(cfg, inp, c, dev, tab, ot)
    assert r["frac_bad"] < 1e-3, r
    assert r["dT"] <= 1e-6, r
    assert r["dq"] <= 1e-5, r
    assert r["dl"] <= 1e-5, r
    assert r["kap"] >= 0.999, r


@pytest.mark.parametrize("case", ["tiny_init", "tiny_true"])
def test_green_functions(dev, case):
    cfg, inp, c = _case(case)
    g = ogeom.from_config(cfg)
    geom = rb.geometry_from_config(cfg)
    _, Gg = gpu_tables(geom, c, inp.alpha0, dev, list(cfg.freqs_hz))
    ot = ogrid.grid(g, c, inp.alpha0)
    for j, f in enumerate(cfg.freqs_hz):
        Go = ogreen.green(g, ot, c, f)
        assert rel_l2(Gg[j], Go) <= 1e-4, (f, rel_l2(Gg[j], Go))


def test_ray_forward_data(dev):
    cfg, inp, c = _case("tiny_true")
    g = ogeom.from_config(cfg)
    geom = rb.geometry_from_config(cfg)
    E, nv, lost = orays.trace_endpoints(g, c, inp.alpha0)
    lk = olink.link(g, E, lost, c)
    ws = rb.workspace(geom, 1, rb.RB_PREC_FP32, dev)
    ends = torch.zeros((geom.n_elem, geom.n_rays, 56), dtype=torch.uint8, device=dev)
    ct = _t(c, dev)
    rb.rb_trace_rays(geom, ct, _t(inp.alpha0, dev), ends, ws)
    p = torch.empty((len(cfg.freqs_hz), g.n_elem, g.n_elem), dtype=torch.complex64, device=dev)
    linked = torch.empty((g.n_elem, g.n_elem), dtype=torch.uint8, device=dev)
    rb.rb_ray_forward(geom, ct, ends, list(cfg.freqs_hz), p, linked)
    pg = p.cpu().numpy()
    mask = ogeom.receiver_mask(g)
    assert np.mean((linked.cpu().numpy() == 1)[mask] == lk.linked[mask]) >= 0.999
    for j, f in enumerate(cfg.freqs_hz):
        po = olink.ray_data(g, lk, f)
        assert rel_l2(pg[j][mask], po[mask]) <= 1e-4, rel_l2(pg[j][mask], po[mask])


@pytest.mark.parametrize("case", ["tiny_init", "tiny_true", "tiny_ragged"])
def test_born_forward_and_adjoint(dev, case):
    cfg, inp, c = _case(case)
    g = ogeom.from_config(cfg)
    geom = rb.geometry_from_config(cfg)
    tab, _ = gpu_tables(geom, c, inp.alpha0, dev)
    ot = ogrid.grid(g, c, inp.alpha0)
    rng = np.random.default_rng(4)
    m = rng.standard_normal(g.npix).astype(np.float32) * 1e-9
    R = (rng.standard_normal((g.n_elem, g.n_elem)) + 1j * rng.standard_normal((g.n_elem, g.n_elem))).astype(np.complex64)
    W = (rng.uniform(size=(g.n_elem, g.n_elem)) > 0.2).astype(np.uint8)
    ws = rb.workspace(geom, 1, rb.RB_PREC_FP32, dev)
    ct = _t(c, dev)
    for f in (cfg.freqs_hz[0], cfg.freqs_hz[-1]):
        Go = ogreen.green(g, ot, c, f)
        d = torch.empty((g.n_elem, g.n_elem), dtype=torch.complex64, device=dev)
        rb.rb_born_forward(geom, tab, ct, f, _t(m, dev), d, ws)
        do = oborn.born_forward(Go, m.astype(np.float64), f)
        assert rel_l2(d.cpu().numpy(), do) <= 1e-4, rel_l2(d.cpu().numpy(), do)
        gg = torch.empty(g.npix, dtype=torch.complex64, device=dev)
        hh = torch.empty(g.npix, dtype=torch.float32, device=dev)
        rb.rb_born_adjoint(geom, tab, ct, f, torch.as_tensor(R, device=dev), torch.as_tensor(W, device=dev), gg, ws, hh)
        go = oborn.born_adjoint(Go, W * R.astype(np.complex128), f)
        ho = oborn.hess_diag(Go, W, f)
        assert rel_l2(gg.cpu().numpy(), go) <= 1e-4, rel_l2(gg.cpu().numpy(), go)
        assert rel_l2(hh.cpu().numpy(), ho) <= 1e-4, rel_l2(hh.cpu().numpy(), ho)


def test_adjoint_identity_on_gpu(dev):
    """<B m, S> = <m, Re B* S> with both operators on the GPU (a property at any size)."""
    cfg, inp, c = _case("tiny_true")
    geom = rb.geometry_from_config(cfg)
    tab, _ = gpu_tables(geom, c, inp.alpha0, dev)
    rng = np.random.default_rng(9)
    n, npix = cfg.n_elem, cfg.nx * cfg.ny
    m = _t(rng.standard_normal(npix) * 1e-9, dev)
    S = torch.as_tensor((rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))).astype(np.complex64), device=dev)
    W = torch.ones((n, n), dtype=torch.uint8, device=dev)
    ws = rb.workspace(geom, 1, rb.RB_PREC_FP32, dev)
    d = torch.empty((n, n), dtype=torch.complex64, device=dev)
    gg = torch.empty(npix, dtype=torch.complex64, device=dev)
    ct = _t(c, dev)
    rb.rb_born_forward(geom, tab, ct, 0.4e6, m, d, ws)
    rb.rb_born_adjoint(geom, tab, ct, 0.4e6, S, W, gg, ws)
    lhs = float(torch.sum((torch.conj(d) * S).real.double()))
    rhs = float(torch.sum(m.double() * gg.real.double()))
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


def _update_pair(cfg, inp, c0, freqs, p_obs, dev, **kw):
    g = ogeom.from_config(cfg)
    ref = oupd.hf_update(g, c0, inp.alpha0, freqs, p_obs, **kw)
    geom = rb.geometry_from_config(cfg)
    c = _t(c0, dev)
    dc = torch.empty_like(c)
    diag = torch.zeros(48, dtype=torch.uint8, device=dev)
    ws = rb.workspace(geom, len(freqs), rb.RB_PREC_FP32, dev)
    step = {"exact": rb.RB_STEP_EXACT, "diag": rb.RB_STEP_DIAG}[kw.get("step", "exact")]
    rb.rb_hf_update(geom, c, _t(inp.alpha0, dev), freqs, torch.as_tensor(p_obs.astype(np.complex64), device=dev), ws,
                    kw.get("outlier_frac", 0.01), kw.get("eps_rel", 1e-3), step, dc_out=dc, diag_out=diag)
    torch.cuda.synchronize()
    return ref, c.cpu().numpy(), dc.cpu().numpy(), rb.decode_diag(diag)


@pytest.mark.parametrize("step", ["exact", "diag"])
def test_hf_update_tiny(dev, step):
    cfg = rbgen.tiny()
    inp = rbgen.make_inputs(cfg)
    g = ogeom.from_config(cfg)
    freqs = [cfg.freqs_hz[0]]
    p_obs = oupd.synth_data(g, inp.c_init, inp.c_true, inp.alpha0, freqs, inp.noise_re, inp.noise_im)
    ref, c_new, dc, d = _update_pair(cfg, inp, inp.c_init, freqs, p_obs, dev, step=step)
    assert d["lost_rays"] == 0 and d["tc_timeouts"] == 0
    assert d["kept"] == ref.n_kept and d["zeroed"] == ref.n_zeroed
    assert d["unlinked"] == ref.n_unlinked
    assert abs(d["alpha"] - ref.alpha) <= 1e-3 * abs(ref.alpha)
    e = rel_l2(dc, ref.dc)
    print(f"tiny update step={step}: dc rel L2 {e:.3g}")
    assert e <= 1e-3, e
    assert abs(d["dc_norm"] - ref.dc_norm) <= 1e-3 * ref.dc_norm


@pytest.mark.parametrize("prec", [rb.RB_PREC_FP32, rb.RB_PREC_BF16X3], ids=["fp32", "bf16x3"])
def test_sweep_tiny_c_map(dev, prec):
    """The whole tiny sweep (3 sets) on either path against the oracle's: c within 0.05 m/s RMS."""
    cfg = rbgen.tiny()
    inp = rbgen.make_inputs(cfg)
    g = ogeom.from_config(cfg)
    p_obs = oupd.synth_data(g, inp.c_init, inp.c_true, inp.alpha0, cfg.freqs_hz, inp.noise_re, inp.noise_im)
    c_ref, norms = oupd.sweep(g, inp.c_init, inp.alpha0, cfg.freqs_hz, cfg.sets, p_obs)
    from paper_2511_16633_gb300.recon import Reconstruction
    rec = Reconstruction(cfg, inp.c_init, inp.alpha0, p_obs.astype(np.complex64), prec=prec, device=dev)
    c_gpu = rec.sweep().cpu().numpy()
    sup = ogeom.support_mask(g)
    rms = np.sqrt(np.mean((c_gpu - c_ref)[sup] ** 2))
    print(f"tiny sweep prec={prec}: c RMS difference {rms:.3g} m/s")
    assert rms <= 0.05, rms
    assert np.allclose(rec.norms, norms, rtol=5e-3)
    assert rec.diagnostics()["tc_timeouts"] == 0


def test_outlier_selection_valid(dev):
    """rb_data_weights on one set of three frequencies against the oracle's weights, entry by
    entry.  The zeroed set is unique given exact residuals: the floor(1 % kept) largest |R|
    over the set (ties by flat index).  The GPU selects on its own FP32 residuals, which match
    the oracle's to FP32 rounding, so an entry may differ only where the oracle's |R| lies
    within 1e-4 of the selection threshold; elsewhere W must be identical, and on the GPU's
    own residuals its selection must be exactly the largest ones."""
    cfg = rbgen.tiny()
    inp = rbgen.make_inputs(cfg)
    g = ogeom.from_config(cfg)
    freqs = list(cfg.freqs_hz)
    p_obs = oupd.synth_data(g, inp.c_init, inp.c_true, inp.alpha0, freqs, inp.noise_re, inp.noise_im)
    ref = oupd.hf_update(g, inp.c_init, inp.alpha0, freqs, p_obs, step="diag")
    geom = rb.geometry_from_config(cfg)
    nf, n = len(freqs), g.n_elem
    R = torch.empty((nf, n, n), dtype=torch.complex64, device=dev)
    W = torch.empty((nf, n, n), dtype=torch.uint8, device=dev)
    ws = rb.workspace(geom, nf, rb.RB_PREC_FP32, dev)
    rb.rb_data_weights(geom, _t(inp.c_init, dev), _t(inp.alpha0, dev), freqs,
                       torch.as_tensor(p_obs.astype(np.complex64), device=dev), R, W, ws, 0.01)
    torch.cuda.synchronize()
    Rg, Wg = R.cpu().numpy(), W.cpu().numpy()
    assert rel_l2(Rg, ref.R) <= 1e-4, rel_l2(Rg, ref.R)
    E, _, lost = orays.trace_endpoints(g, inp.c_init, inp.alpha0)
    lk = olink.link(g, E, lost, inp.c_init)
    kept = np.broadcast_to(ogeom.receiver_mask(g) & lk.linked, Wg.shape)
    k = math.floor(0.01 * ref.n_kept)
    assert kept.sum() == ref.n_kept and ref.n_zeroed == k
    assert not Wg[~kept].any()
    # the GPU's selection is valid on its own residuals: exactly k zeroed, all at least as large
    mg = np.abs(Rg.astype(np.complex128)) ** 2
    zg = kept & (Wg == 0)
    assert zg.sum() == k
    assert mg[zg].min() >= mg[kept & (Wg == 1)].max() * (1 - 1e-6)
    # entry by entry against the oracle's weights
    mo = np.abs(ref.R) ** 2
    t_k = mo[kept & (ref.W == 0)].min()          # the oracle's selection threshold
    diff = Wg != ref.W
    print(f"outlier selection: {int(diff.sum())} of {Wg.size} weights differ from the oracle's, k = {k}")
    assert np.all(np.abs(mo[diff] / t_k - 1.0) <= 1e-4), mo[diff] / t_k


# ---------------------------------------------------------------------------
# Mixed precision: tcgen05 BF16 x3 split products, FP32 accumulation
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("case", ["tiny_init", "tiny_true"])
def test_born_adjoint_bf16x3(dev, case):
    cfg, inp, c = _case(case)
    g = ogeom.from_config(cfg)
    geom = rb.geometry_from_config(cfg)
    tab, _ = gpu_tables(geom, c, inp.alpha0, dev)
    ot = ogrid.grid(g, c, inp.alpha0)
    rng = np.random.default_rng(4)
    R = (rng.standard_normal((g.n_elem, g.n_elem)) + 1j * rng.standard_normal((g.n_elem, g.n_elem))).astype(np.complex64)
    W = (rng.uniform(size=(g.n_elem, g.n_elem)) > 0.2).astype(np.uint8)
    ws = rb.workspace(geom, 1, rb.RB_PREC_BF16X3, dev)
    ct = _t(c, dev)
    for f in (cfg.freqs_hz[0], cfg.freqs_hz[-1]):
        Go = ogreen.green(g, ot, c, f)
        gg = torch.empty(g.npix, dtype=torch.complex64, device=dev)
        hh = torch.empty(g.npix, dtype=torch.float32, device=dev)
        rb.rb_born_adjoint(geom, tab, ct, f, torch.as_tensor(R, device=dev), torch.as_tensor(W, device=dev), gg, ws, hh,
                           prec=rb.RB_PREC_BF16X3)
        go = oborn.born_adjoint(Go, W * R.astype(np.complex128), f)
        ho = oborn.hess_diag(Go, W, f)
        eg, eh = rel_l2(gg.cpu().numpy(), go), rel_l2(hh.cpu().numpy(), ho)
        print(f"bf16x3 {case} f={f:.3g}: gradient rel L2 {eg:.3g}, Hessian diagonal rel L2 {eh:.3g}")
        assert eg <= 1e-4, eg
        assert eh <= 1e-4, eh


def test_hf_update_bf16x3_tiny(dev):
    cfg = rbgen.tiny()
    inp = rbgen.make_inputs(cfg)
    g = ogeom.from_config(cfg)
    freqs = [cfg.freqs_hz[1]]
    p_obs = oupd.synth_data(g, inp.c_init, inp.c_true, inp.alpha0, freqs, inp.noise_re, inp.noise_im)
    ref = oupd.hf_update(g, inp.c_init, inp.alpha0, freqs, p_obs)
    geom = rb.geometry_from_config(cfg)
    c = _t(inp.c_init, dev)
    dc = torch.empty_like(c)
    diag = torch.zeros(48, dtype=torch.uint8, device=dev)
    ws = rb.workspace(geom, 1, rb.RB_PREC_BF16X3, dev)
    rb.rb_hf_update(geom, c, _t(inp.alpha0, dev), freqs, torch.as_tensor(p_obs.astype(np.complex64), device=dev), ws,
                    prec=rb.RB_PREC_BF16X3, dc_out=dc, diag_out=diag)
    torch.cuda.synchronize()
    d = rb.decode_diag(diag)
    assert d["tc_timeouts"] == 0
    e = rel_l2(dc.cpu().numpy(), ref.dc)
    print(f"tiny update bf16x3: dc rel L2 {e:.3g}")
    assert e <= 1e-3, e
    assert abs(d["dc_norm"] - ref.dc_norm) <= 1e-3 * ref.dc_norm


@pytest.mark.parametrize("case", ["tiny_init", "tiny_true"])
def test_born_forward_bf16x3(dev, case):
    cfg, inp, c = _case(case)
    g = ogeom.from_config(cfg)
    geom = rb.geometry_from_config(cfg)
    tab, _ = gpu_tables(geom, c, inp.alpha0, dev)
    ot = ogrid.grid(g, c, inp.alpha0)
    rng = np.random.default_rng(5)
    m = rng.standard_normal(g.npix).astype(np.float32) * 1e-9
    ws = rb.workspace(geom, 1, rb.RB_PREC_BF16X3, dev)
    for f in (cfg.freqs_hz[0], cfg.freqs_hz[-1]):
        d = torch.empty((g.n_elem, g.n_elem), dtype=torch.complex64, device=dev)
        rb.rb_born_forward(geom, tab, _t(c, dev), f, _t(m, dev), d, ws, prec=rb.RB_PREC_BF16X3)
        do = oborn.born_forward(ogreen.green(g, ot, c, f), m.astype(np.float64), f)
        e = rel_l2(d.cpu().numpy(), do)
        print(f"bf16x3 forward {case} f={f:.3g}: rel L2 {e:.3g}")
        assert e <= 1e-4, e


# Mixed precision at the other supported ring sizes, on grids whose pixel count is not a
# multiple of the 128-pixel tile: n_elem = 128 (one N-block of U) and 192 (two N-blocks
# of 96 elements, 8-row TMA boxes in the forward).
@pytest.mark.parametrize("n_elem,nx,ny", [(128, 70, 66), (192, 66, 70)])
def test_bf16x3_ring_sizes_ragged(dev, n_elem, nx, ny):
    cfg = rbgen.tiny(n_elem=n_elem, nx=nx, ny=ny, n_rays=48)
    inp = rbgen.make_inputs(rbgen.tiny(nx=nx, ny=ny, seed=cfg.seed))
    c = inp.c_true
    g = ogeom.from_config(cfg)
    geom = rb.geometry_from_config(cfg)
    assert g.npix % 128 != 0
    tab, _ = gpu_tables(geom, c, inp.alpha0, dev)
    ot = ogrid.grid(g, c, inp.alpha0)
    rng = np.random.default_rng(7)
    R = (rng.standard_normal((g.n_elem, g.n_elem)) + 1j * rng.standard_normal((g.n_elem, g.n_elem))).astype(np.complex64)
    W = (rng.uniform(size=(g.n_elem, g.n_elem)) > 0.25).astype(np.uint8)
    m = rng.standard_normal(g.npix).astype(np.float32) * 1e-9
    ws = rb.workspace(geom, 1, rb.RB_PREC_BF16X3, dev)
    ct = _t(c, dev)
    f = cfg.freqs_hz[-1]
    Go = ogreen.green(g, ot, c, f)
    gg = torch.empty(g.npix, dtype=torch.complex64, device=dev)
    hh = torch.empty(g.npix, dtype=torch.float32, device=dev)
    rb.rb_born_adjoint(geom, tab, ct, f, torch.as_tensor(R, device=dev), torch.as_tensor(W, device=dev), gg, ws, hh,
                       prec=rb.RB_PREC_BF16X3)
    d = torch.empty((g.n_elem, g.n_elem), dtype=torch.complex64, device=dev)
    rb.rb_born_forward(geom, tab, ct, f, _t(m, dev), d, ws, prec=rb.RB_PREC_BF16X3)
    torch.cuda.synchronize()
    eg = rel_l2(gg.cpu().numpy(), oborn.born_adjoint(Go, W * R.astype(np.complex128), f))
    eh = rel_l2(hh.cpu().numpy(), oborn.hess_diag(Go, W, f))
    ed = rel_l2(d.cpu().numpy(), oborn.born_forward(Go, m.astype(np.float64), f))
    print(f"bf16x3 n={n_elem} {nx}x{ny}: gradient {eg:.3g}, Hessian diagonal {eh:.3g}, forward {ed:.3g}")
    assert eg <= 1e-4, eg
    assert eh <= 1e-4, eh
    assert ed <= 1e-4, ed


# Rings of 512 elements (the in-vivo transducer count of the paper's Sec. 4) and 1024 (the
# full array it was taken from) on the tensor cores: the adjoint in passes of 256
# elements, the forward in (row block, column group) pairs, some of which load their row
# block's own rows separately.
@pytest.mark.parametrize("n_elem", [512, 1024])
def test_bf16x3_ring_512(dev, n_elem):
    cfg = rbgen.tiny(n_elem=n_elem, n_rays=64)
    inp = rbgen.make_inputs(cfg)
    c = inp.c_true
    g = ogeom.from_config(cfg)
    geom = rb.geometry_from_config(cfg)
    tab, _ = gpu_tables(geom, c, inp.alpha0, dev)
    ot = ogrid.grid(g, c, inp.alpha0)
    rng = np.random.default_rng(9)
    R = (rng.standard_normal((g.n_elem, g.n_elem)) + 1j * rng.standard_normal((g.n_elem, g.n_elem))).astype(np.complex64)
    W = (rng.uniform(size=(g.n_elem, g.n_elem)) > 0.25).astype(np.uint8)
    m = rng.standard_normal(g.npix).astype(np.float32) * 1e-9
    ws = rb.workspace(geom, 1, rb.RB_PREC_BF16X3, dev)
    ct = _t(c, dev)
    f = cfg.freqs_hz[-1]
    Go = ogreen.green(g, ot, c, f)
    gg = torch.empty(g.npix, dtype=torch.complex64, device=dev)
    hh = torch.empty(g.npix, dtype=torch.float32, device=dev)
    rb.rb_born_adjoint(geom, tab, ct, f, torch.as_tensor(R, device=dev), torch.as_tensor(W, device=dev), gg, ws, hh,
                       prec=rb.RB_PREC_BF16X3)
    d = torch.empty((g.n_elem, g.n_elem), dtype=torch.complex64, device=dev)
    rb.rb_born_forward(geom, tab, ct, f, _t(m, dev), d, ws, prec=rb.RB_PREC_BF16X3)
    torch.cuda.synchronize()
    eg = rel_l2(gg.cpu().numpy(), oborn.born_adjoint(Go, W * R.astype(np.complex128), f))
    eh = rel_l2(hh.cpu().numpy(), oborn.hess_diag(Go, W, f))
    ef = rel_l2(d.cpu().numpy(), oborn.born_forward(Go, m.astype(np.float64), f))
    print(f"bf16x3 n={n_elem}: gradient {eg:.3g}, Hessian diagonal {eh:.3g}, forward {ef:.3g}")
    assert eg <= 1e-4 and eh <= 1e-4 and ef <= 1e-4

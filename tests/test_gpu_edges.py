"""Edge cases of the update path on the GPU: a zero residual, no outlier zeroing, the
largest ring the FP32 adjoint takes (512 elements), the largest fan the linker takes
(4096 rays), each against the oracle or the exact answer."""
import numpy as np
import pytest

import rbgen
from oracle import geometry as ogeom
from oracle import link as olink
from oracle import rays as orays
from oracle import update as oupd

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2511_16633_gb300 import rb  # noqa: E402


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rb.load()
    return torch.device("cuda:0")


def _t(a, dev):
    return torch.as_tensor(np.ascontiguousarray(a), device=dev).to(torch.float32).contiguous()


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


@pytest.mark.parametrize("prec", [rb.RB_PREC_FP32, rb.RB_PREC_BF16X3], ids=["fp32", "bf16x3"])
def test_zero_residual_gives_zero_update(dev, prec):
    """Measured data equal to the ray data of c itself: R = 0, so the gradient, the direction
    and the step are zero (the exact step's 0/0 is guarded) and c does not move."""
    cfg = rbgen.tiny()
    inp = rbgen.make_inputs(cfg)
    geom = rb.geometry_from_config(cfg)
    freqs = [cfg.freqs_hz[1]]
    ws = rb.workspace(geom, 1, prec, dev)
    c = _t(inp.c_init, dev)
    a0 = _t(inp.alpha0, dev)
    ends = torch.zeros((geom.n_elem, geom.n_rays, 56), dtype=torch.uint8, device=dev)
    rb.rb_trace_rays(geom, c, a0, ends, ws)
    p = torch.empty((1, geom.n_elem, geom.n_elem), dtype=torch.complex64, device=dev)
    rb.rb_ray_forward(geom, c, ends, freqs, p)
    for cg in (0, 3):
        c1 = c.clone()
        dc = torch.full_like(c, float("nan"))
        diag = torch.zeros(48, dtype=torch.uint8, device=dev)
        if cg:
            rb.rb_cg_update(geom, c1, a0, freqs, p, ws, cg, prec=prec, dc_out=dc, diag_out=diag)
        else:
            rb.rb_hf_update(geom, c1, a0, freqs, p, ws, prec=prec, dc_out=dc, diag_out=diag)
        torch.cuda.synchronize()
        d = rb.decode_diag(diag)
        assert torch.all(dc == 0), cg
        assert torch.equal(c1, c), cg
        assert d["dc_norm"] == 0.0 and np.isfinite(d["alpha"])


def test_no_outlier_zeroing(dev):
    cfg = rbgen.tiny()
    inp = rbgen.make_inputs(cfg)
    g = ogeom.from_config(cfg)
    freqs = list(cfg.freqs_hz[:2])
    p_obs = oupd.synth_data(g, inp.c_init, inp.c_true, inp.alpha0, freqs, inp.noise_re, inp.noise_im)
    ref = oupd.hf_update(g, inp.c_init, inp.alpha0, freqs, p_obs, outlier_frac=0.0)
    assert ref.n_zeroed == 0
    geom = rb.geometry_from_config(cfg)
    c = _t(inp.c_init, dev)
    dc = torch.empty_like(c)
    diag = torch.zeros(48, dtype=torch.uint8, device=dev)
    ws = rb.workspace(geom, 2, rb.RB_PREC_FP32, dev)
    rb.rb_hf_update(geom, c, _t(inp.alpha0, dev), freqs, torch.as_tensor(p_obs.astype(np.complex64), device=dev), ws,
                    0.0, dc_out=dc, diag_out=diag)
    torch.cuda.synchronize()
    d = rb.decode_diag(diag)
    assert d["zeroed"] == 0 and d["kept"] == ref.n_kept
    assert _rel(dc.cpu().numpy(), ref.dc) <= 1e-3


def test_ring_of_512_elements_fp32(dev):
    """The largest ring of the FP32 adjoint (each lane holds 16 elements)."""
    cfg = rbgen.tiny(n_elem=512, n_rays=64)
    inp = rbgen.make_inputs(cfg)
    g = ogeom.from_config(cfg)
    freqs = [cfg.freqs_hz[1]]
    p_obs = oupd.synth_data(g, inp.c_init, inp.c_true, inp.alpha0, freqs, inp.noise_re, inp.noise_im)
    ref = oupd.hf_update(g, inp.c_init, inp.alpha0, freqs, p_obs)
    geom = rb.geometry_from_config(cfg)
    c = _t(inp.c_init, dev)
    dc = torch.empty_like(c)
    diag = torch.zeros(48, dtype=torch.uint8, device=dev)
    ws = rb.workspace(geom, 1, rb.RB_PREC_FP32, dev)
    rb.rb_hf_update(geom, c, _t(inp.alpha0, dev), freqs, torch.as_tensor(p_obs.astype(np.complex64), device=dev), ws,
                    dc_out=dc, diag_out=diag)
    torch.cuda.synchronize()
    d = rb.decode_diag(diag)
    e = _rel(dc.cpu().numpy(), ref.dc)
    print(f"512 elements: dc rel L2 {e:.3g}, kept {d['kept']} vs {ref.n_kept}, zeroed {d['zeroed']} vs {ref.n_zeroed}")
    assert d["kept"] == ref.n_kept and d["zeroed"] == ref.n_zeroed
    assert e <= 1e-3
    assert abs(d["dc_norm"] - ref.dc_norm) <= 1e-3 * ref.dc_norm


def test_fan_of_4096_rays_linking(dev):
    """The largest fan the linker holds in shared memory: ray data at the receivers."""
    cfg = rbgen.tiny(n_rays=4096)
    inp = rbgen.make_inputs(cfg)
    c = inp.c_true
    g = ogeom.from_config(cfg)
    geom = rb.geometry_from_config(cfg)
    E, nv, lost = orays.trace_endpoints(g, c, inp.alpha0)
    lk = olink.link(g, E, lost, c)
    ws = rb.workspace(geom, 1, rb.RB_PREC_FP32, dev)
    ends = torch.zeros((geom.n_elem, geom.n_rays, 56), dtype=torch.uint8, device=dev)
    ct = _t(c, dev)
    rb.rb_trace_rays(geom, ct, _t(inp.alpha0, dev), ends, ws)
    p = torch.empty((1, g.n_elem, g.n_elem), dtype=torch.complex64, device=dev)
    linked = torch.empty((g.n_elem, g.n_elem), dtype=torch.uint8, device=dev)
    f = cfg.freqs_hz[-1]
    rb.rb_ray_forward(geom, ct, ends, [f], p, linked)
    mask = ogeom.receiver_mask(g)
    assert np.mean((linked.cpu().numpy() == 1)[mask] == lk.linked[mask]) >= 0.999
    po = olink.ray_data(g, lk, f)
    assert _rel(p.cpu().numpy()[0][mask], po[mask]) <= 1e-4


@pytest.mark.parametrize("n_elem", [512, 1024])
def test_ring_of_512_elements_bf16x3_update(dev, n_elem):
    cfg = rbgen.tiny(n_elem=n_elem, n_rays=64)
    inp = rbgen.make_inputs(cfg)
    g = ogeom.from_config(cfg)
    freqs = list(cfg.freqs_hz[1:3])
    p_obs = oupd.synth_data(g, inp.c_init, inp.c_true, inp.alpha0, freqs, inp.noise_re, inp.noise_im)
    ref = oupd.hf_update(g, inp.c_init, inp.alpha0, freqs, p_obs)
    geom = rb.geometry_from_config(cfg)
    c = _t(inp.c_init, dev)
    dc = torch.empty_like(c)
    diag = torch.zeros(48, dtype=torch.uint8, device=dev)
    ws = rb.workspace(geom, 2, rb.RB_PREC_BF16X3, dev)
    rb.rb_hf_update(geom, c, _t(inp.alpha0, dev), freqs, torch.as_tensor(p_obs.astype(np.complex64), device=dev), ws,
                    prec=rb.RB_PREC_BF16X3, dc_out=dc, diag_out=diag)
    torch.cuda.synchronize()
    d = rb.decode_diag(diag)
    e = _rel(dc.cpu().numpy(), ref.dc)
    print(f"{n_elem} elements bf16x3: dc rel L2 {e:.3g}, alpha {d['alpha']:.6g} vs {ref.alpha:.6g}")
    assert d["tc_timeouts"] == 0
    assert d["kept"] == ref.n_kept and d["zeroed"] == ref.n_zeroed
    assert e <= 1e-3


@pytest.mark.parametrize("which", ["hf", "cg"])
def test_lost_rays_reported_by_the_next_update(dev, which):
    """Rays still inside the ring after max_steps are lost: the update that lost them counts
    them (rb_diag) and sets its stream's limit word; the next update call from that stream
    returns RB_ERR_LIMIT and launches nothing (c does not move); the call after runs again,
    and a call with another workspace on that stream discards the report it left.
    Here 100 steps of 0.8 mm reach receivers up to 80 mm away but not across the 100 mm
    diameter of the ring."""
    cfg = rbgen.tiny()
    inp = rbgen.make_inputs(cfg)
    geom = rb.geometry_from_config(cfg, max_steps=100)
    stream = torch.cuda.Stream(device=dev)
    freqs = [cfg.freqs_hz[0]]
    with torch.cuda.stream(stream):
        c = _t(inp.c_init, dev)
        a0 = _t(inp.alpha0, dev)
        p = torch.zeros((1, geom.n_elem, geom.n_elem), dtype=torch.complex64, device=dev)
        ws = rb.workspace(geom, 1, rb.RB_PREC_FP32, dev)
        diag = torch.zeros(48, dtype=torch.uint8, device=dev)

        def update():
            if which == "hf":
                rb.rb_hf_update(geom, c, a0, freqs, p, ws, diag_out=diag, stream=stream)
            else:
                rb.rb_cg_update(geom, c, a0, freqs, p, ws, 2, diag_out=diag, stream=stream)

        update()
        stream.synchronize()
        d = rb.decode_diag(diag)
        assert d["lost_rays"] > 0
        c_before = c.clone()
        diag.zero_()
        with pytest.raises(rb.RbError) as ei:
            update()
        assert ei.value.code == rb.RB_ERR_LIMIT
        stream.synchronize()
        assert torch.equal(c, c_before) and not diag.any()   # nothing was launched
        update()                          # reported once: this one runs
        stream.synchronize()
        assert not torch.equal(c, c_before)
        assert rb.decode_diag(diag)["lost_rays"] > 0
        # a new problem on the same stream (another workspace) does not inherit the report
        ws_first = ws                     # kept alive, so the new workspace is another buffer
        ws = rb.workspace(geom, 1, rb.RB_PREC_FP32, dev)
        assert ws.data_ptr() != ws_first.data_ptr()
        update()
        stream.synchronize()

"""GPU parity of the time-of-flight initial guess (rb_tof_times, rb_tof_invert)
against the oracle (oracle/tof.py).

Tolerances: linked times of flight 1e-6 relative (the ray traveltime bound), the
linked masks equal on all but 0.1 % of the pairs; after three linearisations from
water the sound-speed map within 0.05 m/s RMS of the oracle's over the support and
the RMS misfit history within 1 %.  The fixed-point pixel sums make the result
bit-identical from run to run.
"""
import math

import numpy as np
import pytest

import rbgen
from oracle import geometry as ogeom
from oracle import tof as otof

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


CASES = {"tiny": lambda: rbgen.tiny(), "ragged": lambda: rbgen.tiny(n_rays=45, nx=70, ny=66, n_elem=40)}


def _gpu_times(geom, c, a0, dev):
    n = geom.n_elem
    ws = rb.workspace(geom, 1, rb.RB_PREC_FP32, dev)
    T = torch.zeros((n, n), dtype=torch.float64, device=dev)
    lk = torch.zeros((n, n), dtype=torch.uint8, device=dev)
    rb.rb_tof_times(geom, _t(c, dev), _t(a0, dev), T, ws, lk)
    torch.cuda.synchronize()
    return T, lk


@pytest.mark.parametrize("case", list(CASES))
def test_tof_times(dev, case):
    cfg = CASES[case]()
    inp = rbgen.make_inputs(cfg)
    g = ogeom.from_config(cfg)
    geom = rb.geometry_from_config(cfg)
    To, lo = otof.tof_times(g, inp.c_true, inp.alpha0)
    T, lk = _gpu_times(geom, inp.c_true, inp.alpha0, dev)
    T, lk = T.cpu().numpy(), lk.cpu().numpy().astype(bool)
    assert np.mean(lk != lo) <= 1e-3
    both = lk & lo
    assert np.max(np.abs(T[both] - To[both]) / To[both]) <= 1e-6


@pytest.mark.parametrize("case", list(CASES))
def test_tof_invert(dev, case):
    cfg = CASES[case]()
    inp = rbgen.make_inputs(cfg)
    g = ogeom.from_config(cfg)
    geom = rb.geometry_from_config(cfg)
    To, lo = otof.tof_times(g, inp.c_true, inp.alpha0)
    c0 = np.full((g.ny, g.nx), g.c_ref)
    c_ref, hist_ref = otof.tof_invert(g, c0, inp.alpha0, To, lo, 3)
    T_obs, l_obs = _gpu_times(geom, inp.c_true, inp.alpha0, dev)
    ws = rb.workspace(geom, 1, rb.RB_PREC_FP32, dev)
    outs = []
    for _ in range(2):
        c = _t(c0, dev)
        hist = torch.zeros(4, dtype=torch.float64, device=dev)
        rb.rb_tof_invert(geom, c, _t(inp.alpha0, dev), T_obs, l_obs, ws, 3, hist)
        torch.cuda.synchronize()
        outs.append((c.cpu().numpy(), hist.cpu().numpy()))
    (c1, h1), (c2, _) = outs
    assert np.array_equal(c1, c2)
    sup = ogeom.support_mask(g)
    rms = math.sqrt(float(np.mean((c1 - c_ref)[sup] ** 2)))
    e0 = math.sqrt(float(np.mean((c0 - inp.c_true)[sup] ** 2)))
    e3 = math.sqrt(float(np.mean((c1 - inp.c_true)[sup] ** 2)))
    print(f"{case}: c RMS vs oracle {rms:.3g} m/s; error vs truth {e0:.3f} -> {e3:.3f} m/s; "
          f"misfit {h1} vs {np.array(hist_ref)}")
    assert rms <= 0.05, rms
    assert np.allclose(h1, hist_ref, rtol=1e-2)
    assert e3 < e0


def test_tof_breast256_properties(dev):
    """Full size (256 elements, 256 x 256 pixels, 256 rays): three linearisations from water
    lower the ToF misfit at every step and the sound-speed error against the phantom, two
    runs agree bit for bit, and the map and misfit history match the oracle's."""
    cfg = rbgen.breast256()
    inp = rbgen.make_inputs(cfg)
    g = ogeom.from_config(cfg)
    geom = rb.geometry_from_config(cfg)
    T_obs, l_obs = _gpu_times(geom, inp.c_true, inp.alpha0, dev)
    ws = rb.workspace(geom, 1, rb.RB_PREC_FP32, dev)
    c0 = np.full((g.ny, g.nx), g.c_ref)
    outs = []
    for _ in range(2):
        c = _t(c0, dev)
        hist = torch.zeros(4, dtype=torch.float64, device=dev)
        rb.rb_tof_invert(geom, c, _t(inp.alpha0, dev), T_obs, l_obs, ws, 3, hist)
        torch.cuda.synchronize()
        outs.append((c.cpu().numpy(), hist.cpu().numpy()))
    (c1, h1), (c2, h2) = outs
    assert np.array_equal(c1, c2) and np.array_equal(h1, h2)
    assert h1[1] < h1[0] and h1[2] < h1[1] and h1[3] < h1[2], h1
    sup = ogeom.support_mask(g)
    e0 = math.sqrt(float(np.mean((c0 - inp.c_true)[sup] ** 2)))
    e3 = math.sqrt(float(np.mean((c1 - inp.c_true)[sup] ** 2)))
    print(f"breast256 ToF: misfit {h1}, c error {e0:.3f} -> {e3:.3f} m/s")
    assert e3 < 0.9 * e0
    # and against the oracle at this size (about 40 s of CPU)
    To, lo = otof.tof_times(g, inp.c_true, inp.alpha0)
    c_ref, hist_ref = otof.tof_invert(g, c0, inp.alpha0, To, lo, 3)
    rms = math.sqrt(float(np.mean((c1 - c_ref)[sup] ** 2)))
    print(f"breast256 ToF against the oracle: c RMS {rms:.3g} m/s, misfit {h1} vs {np.array(hist_ref)}")
    assert rms <= 0.05, rms
    assert np.allclose(h1, hist_ref, rtol=1e-3)


def test_pipeline_tof_then_sweep_reduces_error(dev):
    """The workflow end to end on the tiny phantom: the time-of-flight guess improves on
    water and the ray-Born sweep from it improves on the guess."""
    from paper_2511_16633_gb300.recon import pipeline
    out = pipeline(rbgen.tiny(), 3, rb.RB_PREC_BF16X3, dev)
    print(f"pipeline tiny: water {out['rms_water']:.3f}, ToF {out['rms_tof']:.3f}, sweep {out['rms_after_set']}")
    assert out["rms_tof"] < out["rms_water"]
    assert out["rms_after_set"][-1] < out["rms_tof"]

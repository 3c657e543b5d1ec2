"""An update captured into a CUDA graph and replayed gives the eager update's result bit
for bit: the library's fork onto its side stream and the join back are followed by the
capture, and nothing in a call depends on host state between launches."""
import numpy as np
import pytest

import rbgen
from oracle import geometry as ogeom
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


@pytest.mark.parametrize("prec", [rb.RB_PREC_FP32, rb.RB_PREC_BF16X3], ids=["fp32", "bf16x3"])
@pytest.mark.parametrize("cg", [0, 3], ids=["one_step", "cg3"])
def test_update_replayed_from_a_cuda_graph(dev, prec, cg):
    cfg = rbgen.tiny()
    inp = rbgen.make_inputs(cfg)
    g = ogeom.from_config(cfg)
    freqs = list(cfg.freqs_hz[:2])
    p_obs = oupd.synth_data(g, inp.c_init, inp.c_true, inp.alpha0, freqs, inp.noise_re, inp.noise_im)
    geom = rb.geometry_from_config(cfg)
    c0 = torch.as_tensor(inp.c_init, device=dev, dtype=torch.float32).contiguous()
    a0 = torch.as_tensor(inp.alpha0, device=dev, dtype=torch.float32).contiguous()
    p = torch.as_tensor(p_obs.astype(np.complex64), device=dev).contiguous()
    ws = rb.workspace(geom, len(freqs), prec, dev)

    def call(c, dc, diag):
        if cg:
            rb.rb_cg_update(geom, c, a0, freqs, p, ws, cg, prec=prec, dc_out=dc, diag_out=diag)
        else:
            rb.rb_hf_update(geom, c, a0, freqs, p, ws, prec=prec, dc_out=dc, diag_out=diag)

    c1, dc1, d1 = c0.clone(), torch.empty_like(c0), torch.zeros(48, dtype=torch.uint8, device=dev)
    call(c1, dc1, d1)
    torch.cuda.synchronize()

    c2, dc2, d2 = c0.clone(), torch.empty_like(c0), torch.zeros(48, dtype=torch.uint8, device=dev)
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        with torch.cuda.graph(graph):
            call(c2, dc2, d2)
    torch.cuda.current_stream().wait_stream(side)
    for _ in range(2):   # replays start from c0 each time
        c2.copy_(c0)
        graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(c1, c2)
    assert torch.equal(dc1, dc2)
    assert rb.decode_diag(d1) == rb.decode_diag(d2)

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


_FIRST_CALL_IN_CAPTURE = r"""
import sys
import torch
import rbgen
from paper_2511_16633_gb300 import rb, serve
from paper_2511_16633_gb300.recon import Reconstruction
dev = torch.device("cuda:0")
rb.load()
cfg = rbgen.tiny()
prob = serve.make_problem(cfg, dev)
s = torch.cuda.Stream()
with torch.cuda.stream(s):
    rec = Reconstruction(cfg, prob.c_init, prob.alpha0, prob.p_obs, prec=rb.RB_PREC_BF16X3, device=dev)
    c0 = rec.c.clone()
    g = torch.cuda.CUDAGraph()
    g.capture_begin()
    for j in range(len(cfg.sets)):
        rec.update(j, s)
    g.capture_end()
    g.replay()
s.synchronize()
c_graph = rec.c.clone()
with torch.cuda.stream(s):
    rec.c.copy_(c0)
    for j in range(len(cfg.sets)):
        rec.update(j, s)
s.synchronize()
assert torch.equal(c_graph, rec.c)
assert not torch.equal(c_graph, c0)
print("first update call inside a capture: ok")
"""


def test_first_update_call_inside_a_capture(dev):
    """A fresh process whose first update call is made inside a CUDA-graph capture (the
    library then creates its side stream during the capture): the captured sweep of all
    sets replays to the eager sweep's result."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, PYTHONPATH=root + os.pathsep + os.environ.get("PYTHONPATH", ""))
    r = subprocess.run([sys.executable, "-c", _FIRST_CALL_IN_CAPTURE], cwd=root, env=env, capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "ok" in r.stdout

"""rb_born_forward_noalloc: the Born forward for callers that cannot give the library
device scratch memory (plugins handed tensors but no allocator, real-time loops that
forbid allocation once running).  Its scratch is a fixed array inside the library.

Checked through the C-ABI against rb_born_forward (which uses a caller workspace) on
two calls in a row, within the tolerance of the other Born parity tests (1e-4
relative L2; the two differ only in the order of the split-K sums).  The file is
named to be collected last, and it passes alone in a fresh process as well as after
the other tests.
"""
import numpy as np
import pytest

import rbgen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2511_16633_gb300 import rb  # noqa: E402


def rel_l2(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


@pytest.mark.parametrize("name", ["tiny", "breast256"])
def test_noalloc_forward_matches_workspace_forward(name):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    cfg = rbgen.config_by_name(name)
    inp = rbgen.make_inputs(cfg)
    geom = rb.geometry_from_config(cfg)
    c = torch.as_tensor(inp.c_init, device=dev).contiguous()
    a0 = torch.as_tensor(inp.alpha0, device=dev).contiguous()
    ws = rb.workspace(geom, 1, rb.RB_PREC_FP32, dev)
    tab = torch.empty((geom.n_elem, geom.nx * geom.ny, 4), dtype=torch.int32, device=dev)
    rb.rb_green_grid(geom, c, a0, tab, ws)
    rng = np.random.default_rng(21)
    n = geom.n_elem
    cases = [(cfg.freqs_hz[0], rng.standard_normal(geom.nx * geom.ny) * 1e-9),
             (cfg.freqs_hz[-1], rng.standard_normal(geom.nx * geom.ny) * 1e-9)]
    refs = []
    for f, m in cases:
        d = torch.empty((n, n), dtype=torch.complex64, device=dev)
        rb.rb_born_forward(geom, tab, c, f, torch.as_tensor(m, dtype=torch.float32, device=dev), d, ws)
        refs.append(d.cpu().numpy())
    torch.cuda.synchronize()
    free_before = None
    for k, (f, m) in enumerate(cases):
        d = torch.empty((n, n), dtype=torch.complex64, device=dev)
        mt = torch.as_tensor(m, dtype=torch.float32, device=dev)
        torch.cuda.synchronize()
        if k == 1:
            free_before = torch.cuda.mem_get_info(dev)[0]
        rb.rb_born_forward_noalloc(geom, tab, c, f, mt, d)
        torch.cuda.synchronize()
        if k == 1:
            # the second call reserves nothing on the device
            assert abs(torch.cuda.mem_get_info(dev)[0] - free_before) <= 2 << 20
        assert rel_l2(d.cpu().numpy(), refs[k]) <= 1e-4, (k, rel_l2(d.cpu().numpy(), refs[k]))

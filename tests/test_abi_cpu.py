"""C-ABI checks that need no GPU: the library loads, exports every entry point
include/rb.h declares, its struct layouts match the binding, and argument
errors come back synchronously before any CUDA call."""
import ctypes
import os
import re
import subprocess

import pytest

import rbgen
from paper_2511_16633_gb300 import _build, rb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rb.h")


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return rb.load()


def _declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(rb_[a-z_]+)\s*\(", txt)))


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert set(names) == set(rb.EXPORTS)
    out = subprocess.run(["nm", "-D", "--defined-only", _build.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s(rb_\w+)", out))
    assert set(names) <= exported
    for n in names:
        assert hasattr(lib, n)


def test_struct_layouts_match_header(tmp_path):
    src = tmp_path / "lay.c"
    src.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "rb.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu\n", sizeof(rb_geometry), sizeof(rb_ray_end), sizeof(rb_cell),
         sizeof(rb_update_params), sizeof(rb_diag), sizeof(rb_rays));
  printf("%zu %zu %zu %zu\n", offsetof(rb_geometry, power_y), offsetof(rb_ray_end, kappa),
         offsetof(rb_cell, tkey), offsetof(rb_diag, kept));
  return 0; }
''')
    exe = tmp_path / "lay"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    a, b = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")[:2]
    sizes = [int(v) for v in a.split()]
    offs = [int(v) for v in b.split()]
    assert sizes == [ctypes.sizeof(rb.rb_geometry), rb.RAY_END_DTYPE.itemsize, rb.CELL_DTYPE.itemsize,
                     ctypes.sizeof(rb.rb_update_params), rb.DIAG_DTYPE.itemsize, ctypes.sizeof(rb.rb_rays)]
    assert offs == [rb.rb_geometry.power_y.offset, rb.RAY_END_DTYPE.fields["kappa"][1],
                    rb.CELL_DTYPE.fields["tkey"][1], rb.DIAG_DTYPE.fields["kept"][1]]


def test_workspace_size(lib):
    g = rb.geometry_from_config(rbgen.tiny())
    n1 = rb.rb_workspace_size(g, 1)
    n3 = rb.rb_workspace_size(g, 3)
    assert 0 < n1 < n3
    big = rb.geometry_from_config(rbgen.breast512())
    assert rb.rb_workspace_size(big, 4) > 256 * 512 * 512 * 16   # holds the tables
    assert rb.rb_workspace_size(g, 0) == 0
    assert rb.rb_workspace_size(g, rb.RB_MAX_FREQ + 1) == 0
    bad = rb.geometry_from_config(rbgen.tiny(), nx=2)
    assert rb.rb_workspace_size(bad, 1) == 0
    ring_outside = rb.geometry_from_config(rbgen.tiny(), ring_radius=0.06)
    assert rb.rb_workspace_size(ring_outside, 1) == 0


def test_argument_errors_are_synchronous(lib):
    g = rb.geometry_from_config(rbgen.tiny())
    P = ctypes.c_void_p
    fake = P(0x10000)          # never dereferenced: every call below fails validation first
    mis = P(0x10008)
    r = rb.rb_rays(None, None, None, None, None, None, None)
    assert lib.rb_trace_rays(ctypes.byref(g), None, fake, ctypes.byref(r), fake, 1 << 30, None) == rb.RB_ERR_ARG
    r.ends = 0x10000
    r.vx = 0x10000             # partial sample set
    assert lib.rb_trace_rays(ctypes.byref(g), fake, fake, ctypes.byref(r), fake, 1 << 30, None) == rb.RB_ERR_ARG
    r.vx = None
    assert lib.rb_trace_rays(ctypes.byref(g), fake, fake, ctypes.byref(r), mis, 1 << 30, None) == rb.RB_ERR_WORKSPACE
    assert lib.rb_trace_rays(ctypes.byref(g), fake, fake, ctypes.byref(r), fake, 1024, None) == rb.RB_ERR_WORKSPACE
    bad = rb.geometry_from_config(rbgen.tiny(), n_rays=1)
    assert lib.rb_trace_rays(ctypes.byref(bad), fake, fake, ctypes.byref(r), fake, 1 << 30, None) == rb.RB_ERR_SHAPE
    f17 = (ctypes.c_double * 17)(*([3e5] * 17))
    assert lib.rb_ray_forward(ctypes.byref(g), fake, fake, f17, 17, fake, None, None) == rb.RB_ERR_ARG
    fneg = (ctypes.c_double * 1)(-1.0)
    assert lib.rb_ray_forward(ctypes.byref(g), fake, fake, fneg, 1, fake, None, None) == rb.RB_ERR_ARG
    assert lib.rb_born_forward(ctypes.byref(g), fake, fake, ctypes.c_double(0.0), fake, fake, 0, fake, 1 << 30,
                               None) == rb.RB_ERR_ARG
    assert lib.rb_born_adjoint(ctypes.byref(g), fake, fake, ctypes.c_double(3e5), fake, fake, fake, None, 7, fake,
                               1 << 30, None) == rb.RB_ERR_ARG
    prm = rb.rb_update_params(1.5, 1e-3, 0)
    f1 = (ctypes.c_double * 1)(3e5)
    assert lib.rb_hf_update(ctypes.byref(g), fake, fake, f1, 1, fake, ctypes.byref(prm), 0, None, None, fake, 1 << 30,
                            None) == rb.RB_ERR_ARG
    prm = rb.rb_update_params(0.01, 1e-3, 9)
    assert lib.rb_hf_update(ctypes.byref(g), fake, fake, f1, 1, fake, ctypes.byref(prm), 0, None, None, fake, 1 << 30,
                            None) == rb.RB_ERR_ARG
    for bad_tune in (3, 12, 16, -1):
        prm = rb.rb_update_params(0.01, 1e-3, 0, bad_tune)
        assert lib.rb_hf_update(ctypes.byref(g), fake, fake, f1, 1, fake, ctypes.byref(prm), 0, None, None, fake,
                                1 << 30, None) == rb.RB_ERR_ARG
    prm = rb.rb_update_params(0.01, 1e-3, 0)
    for iters, pre in ((0, 1), (rb.RB_MAX_CG + 1, 1), (4, 2)):
        assert lib.rb_cg_update(ctypes.byref(g), fake, fake, f1, 1, fake, ctypes.byref(prm), iters, pre, 0, None, None,
                                None, fake, 1 << 30, None) == rb.RB_ERR_ARG
    assert lib.rb_cg_update(ctypes.byref(g), fake, fake, f1, 1, fake, ctypes.byref(prm), 4, 1, 0, None, None, None,
                            fake, 1024, None) == rb.RB_ERR_WORKSPACE
    for iters in (0, rb.RB_MAX_TOF_ITERS + 1):
        assert lib.rb_tof_invert(ctypes.byref(g), fake, fake, fake, fake, iters, None, fake, 1 << 30,
                                 None) == rb.RB_ERR_ARG
    assert lib.rb_tof_invert(ctypes.byref(g), fake, fake, None, fake, 3, None, fake, 1 << 30, None) == rb.RB_ERR_ARG
    assert lib.rb_tof_times(ctypes.byref(g), fake, fake, None, None, fake, 1 << 30, None) == rb.RB_ERR_ARG
    assert lib.rb_tof_times(ctypes.byref(g), fake, fake, fake, None, fake, 1024, None) == rb.RB_ERR_WORKSPACE
    f0 = (ctypes.c_double * 1)(3e5)
    assert lib.rb_hf_update(ctypes.byref(g), fake, fake, f0, 0, fake, ctypes.byref(prm), 0, None, None, fake, 1 << 30,
                            None) == rb.RB_ERR_ARG
    # the tensor-core path takes rings of 64..256 elements in multiples of 64, and 512, 768, 1024
    for n_bad in (96, 320, 640):
        gb = rb.geometry_from_config(rbgen.tiny(), n_elem=n_bad)
        assert lib.rb_hf_update(ctypes.byref(gb), fake, fake, f1, 1, fake, ctypes.byref(prm), rb.RB_PREC_BF16X3, None,
                                None, fake, 1 << 30, None) == rb.RB_ERR_UNSUPPORTED
        assert lib.rb_cg_update(ctypes.byref(gb), fake, fake, f1, 1, fake, ctypes.byref(prm), 4, 1, rb.RB_PREC_BF16X3,
                                None, None, None, fake, 1 << 30, None) == rb.RB_ERR_UNSUPPORTED
    g640 = rb.geometry_from_config(rbgen.tiny(), n_elem=640)
    assert lib.rb_hf_update(ctypes.byref(g640), fake, fake, f1, 1, fake, ctypes.byref(prm), rb.RB_PREC_FP32, None,
                            None, fake, 1 << 30, None) == rb.RB_ERR_UNSUPPORTED
    assert lib.rb_born_adjoint(ctypes.byref(g640), fake, fake, ctypes.c_double(3e5), fake, fake, fake, None,
                               rb.RB_PREC_FP32, fake, 1 << 30, None) == rb.RB_ERR_UNSUPPORTED
    # residuals and data weights of one set
    assert lib.rb_data_weights(ctypes.byref(g), fake, fake, f1, 1, fake, ctypes.c_double(0.01), None, fake, fake,
                               1 << 30, None) == rb.RB_ERR_ARG
    assert lib.rb_data_weights(ctypes.byref(g), fake, fake, f1, 1, fake, ctypes.c_double(1.0), fake, fake, fake,
                               1 << 30, None) == rb.RB_ERR_ARG
    assert lib.rb_data_weights(ctypes.byref(g), fake, fake, f17, 17, fake, ctypes.c_double(0.01), fake, fake, fake,
                               1 << 30, None) == rb.RB_ERR_ARG
    assert lib.rb_data_weights(ctypes.byref(g), fake, fake, fneg, 1, fake, ctypes.c_double(0.01), fake, fake, fake,
                               1 << 30, None) == rb.RB_ERR_ARG
    assert lib.rb_data_weights(ctypes.byref(bad), fake, fake, f1, 1, fake, ctypes.c_double(0.01), fake, fake, fake,
                               1 << 30, None) == rb.RB_ERR_SHAPE
    assert lib.rb_data_weights(ctypes.byref(g), fake, fake, f1, 1, fake, ctypes.c_double(0.01), fake, fake, fake,
                               1024, None) == rb.RB_ERR_WORKSPACE
    # the Born forward without a workspace: null pointers, bad frequency, rejected geometry,
    # all before its scratch array is looked up (no CUDA call)
    for args in ((None, fake, fake, fake), (fake, None, fake, fake), (fake, fake, None, fake), (fake, fake, fake, None)):
        tab, cc, mm, dd = args
        assert lib.rb_born_forward_noalloc(ctypes.byref(g), tab, cc, ctypes.c_double(3e5), mm, dd,
                                           None) == rb.RB_ERR_ARG
    for fbad in (0.0, -3e5, float("nan"), float("inf")):
        assert lib.rb_born_forward_noalloc(ctypes.byref(g), fake, fake, ctypes.c_double(fbad), fake, fake,
                                           None) == rb.RB_ERR_ARG
    assert lib.rb_born_forward_noalloc(None, fake, fake, ctypes.c_double(3e5), fake, fake, None) == rb.RB_ERR_ARG
    for gbad in (bad, rb.geometry_from_config(rbgen.tiny(), nx=2),
                 rb.geometry_from_config(rbgen.tiny(), ring_radius=0.06)):
        assert lib.rb_born_forward_noalloc(ctypes.byref(gbad), fake, fake, ctypes.c_double(3e5), fake, fake,
                                           None) == rb.RB_ERR_SHAPE
    misaligned_tab = P(0x10004)
    assert lib.rb_green_grid(ctypes.byref(g), fake, fake, misaligned_tab, None, 0, None, fake, 1 << 30,
                             None) == rb.RB_ERR_ARG


def test_status_strings(lib):
    for code in range(7):
        assert len(rb.status_string(code)) > 0
    assert rb.status_string(99) == "unknown status"


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """No fallback: without the compiled library the binding raises instead of computing
    anything another way."""
    from paper_2511_16633_gb300 import _build, rb
    monkeypatch.setattr(rb, "_lib", None)
    monkeypatch.setattr(_build, "LIB", str(tmp_path / "librb.so"))
    with pytest.raises(RuntimeError, match="librb.so not found"):
        rb.load(build_if_missing=False)

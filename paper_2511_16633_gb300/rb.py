"""ctypes binding of librb (include/rb.h): the same entry points, argument marshalling only.

Tensors are torch CUDA tensors; their data pointers are passed straight to the
C-ABI together with the current CUDA stream.  Every computation runs in the
library's kernels: there is no fallback, and a missing or unloadable library
raises.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

from . import _build

RB_OK, RB_ERR_ARG, RB_ERR_SHAPE, RB_ERR_WORKSPACE, RB_ERR_CUDA, RB_ERR_LIMIT, RB_ERR_UNSUPPORTED = range(7)
RB_PREC_FP32, RB_PREC_BF16X3 = 0, 1
RB_STEP_EXACT, RB_STEP_DIAG = 0, 1
RB_TUNE_RULE, RB_TUNE_RASTER_ALONG, RB_TUNE_RASTER_ACROSS = 0, 1, 2
RB_TUNE_ADJ_PAIR, RB_TUNE_ADJ_SINGLE = 1 << 2, 2 << 2
RB_MAX_FREQ = 16
RB_MAX_CG = 24
RB_MAX_TOF_ITERS = 16
RB_HOLE = 0xFFFFFFFF

EXPORTS = ("rb_workspace_size", "rb_trace_rays", "rb_green_grid", "rb_ray_forward", "rb_data_weights", "rb_born_forward",
           "rb_born_adjoint", "rb_hf_update", "rb_cg_update", "rb_tof_times", "rb_tof_invert", "rb_born_forward_noalloc",
           "rb_status_string")


class RbError(RuntimeError):
    def __init__(self, fn, code, msg):
        super().__init__(f"{fn} failed: {msg} (status {code})")
        self.code = code


class rb_geometry(ctypes.Structure):
    _fields_ = [("n_elem", ctypes.c_int32), ("ring_radius", ctypes.c_double), ("nx", ctypes.c_int32),
                ("ny", ctypes.c_int32), ("h", ctypes.c_double), ("n_rays", ctypes.c_int32),
                ("ds", ctypes.c_double), ("max_steps", ctypes.c_int32), ("support_margin", ctypes.c_double),
                ("c_ref", ctypes.c_double), ("f_ref", ctypes.c_double), ("power_y", ctypes.c_double)]


class rb_rays(ctypes.Structure):
    _fields_ = [("ends", ctypes.c_void_p), ("vx", ctypes.c_void_p), ("vy", ctypes.c_void_p), ("vt", ctypes.c_void_p),
                ("vq", ctypes.c_void_p), ("vl", ctypes.c_void_p), ("vkappa", ctypes.c_void_p)]


class rb_update_params(ctypes.Structure):
    _fields_ = [("outlier_frac", ctypes.c_double), ("eps_rel", ctypes.c_double), ("step_mode", ctypes.c_int32),
                ("tune", ctypes.c_int32), ("stage_events", ctypes.c_void_p)]


STAGES = ("fields", "trace_grid", "link", "images", "adjoint", "direction", "forward", "apply")


# numpy views of the device records
RAY_END_DTYPE = np.dtype([("t", "<f8"), ("t_res", "<f8"), ("x", "<f8"), ("y", "<f8"), ("theta", "<f4"),
                          ("q", "<f4"), ("p", "<f4"), ("l", "<f4"), ("kappa", "<i4"), ("n_vert", "<i4")])
CELL_DTYPE = np.dtype([("tag", "<u4"), ("tkey", "<u4"), ("q", "<f4"), ("l", "<f4")])
DIAG_DTYPE = np.dtype([("dc_norm", "<f8"), ("alpha", "<f8"), ("eps", "<f8"), ("lost_rays", "<u4"),
                       ("holes", "<u4"), ("unlinked", "<u4"), ("kept", "<u4"), ("zeroed", "<u4"),
                       ("tc_timeouts", "<u4")])
assert RAY_END_DTYPE.itemsize == 56 and CELL_DTYPE.itemsize == 16 and DIAG_DTYPE.itemsize == 48

_lib = None


def load(build_if_missing: bool = True):
    """Load librb.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing and _build.stale():
        _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"librb.so not found at {path}; run __graft_entry__.build()")
    L = ctypes.CDLL(path)
    P, G = ctypes.c_void_p, ctypes.POINTER(rb_geometry)
    L.rb_workspace_size.argtypes = [G, ctypes.c_int32, ctypes.c_int]
    L.rb_workspace_size.restype = ctypes.c_size_t
    L.rb_trace_rays.argtypes = [G, P, P, ctypes.POINTER(rb_rays), P, ctypes.c_size_t, P]
    L.rb_green_grid.argtypes = [G, P, P, P, P, ctypes.c_int32, P, P, ctypes.c_size_t, P]
    L.rb_ray_forward.argtypes = [G, P, P, P, ctypes.c_int32, P, P, P]
    L.rb_data_weights.argtypes = [G, P, P, P, ctypes.c_int32, P, ctypes.c_double, P, P, P, ctypes.c_size_t, P]
    L.rb_born_forward.argtypes = [G, P, P, ctypes.c_double, P, P, ctypes.c_int, P, ctypes.c_size_t, P]
    L.rb_born_adjoint.argtypes = [G, P, P, ctypes.c_double, P, P, P, P, ctypes.c_int, P, ctypes.c_size_t, P]
    L.rb_hf_update.argtypes = [G, P, P, P, ctypes.c_int32, P, ctypes.POINTER(rb_update_params), ctypes.c_int, P, P,
                               P, ctypes.c_size_t, P]
    L.rb_cg_update.argtypes = [G, P, P, P, ctypes.c_int32, P, ctypes.POINTER(rb_update_params), ctypes.c_int32,
                               ctypes.c_int32, ctypes.c_int, P, P, P, P, ctypes.c_size_t, P]
    L.rb_tof_times.argtypes = [G, P, P, P, P, P, ctypes.c_size_t, P]
    L.rb_tof_invert.argtypes = [G, P, P, P, P, ctypes.c_int32, P, P, ctypes.c_size_t, P]
    L.rb_born_forward_noalloc.argtypes = [G, P, P, ctypes.c_double, P, P, P]
    L.rb_status_string.argtypes = [ctypes.c_int]
    L.rb_status_string.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name not in ("rb_workspace_size", "rb_status_string"):
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def status_string(code: int) -> str:
    return load().rb_status_string(code).decode()


def _check(fn, code):
    if code != RB_OK:
        raise RbError(fn, code, status_string(code))


def geometry(n_elem, ring_radius, nx, ny, h, n_rays, ds=None, max_steps=None, support_margin=None, c_ref=1480.0,
             f_ref=1.0e6, power_y=1.0) -> rb_geometry:
    ds = h / 2.0 if ds is None else ds
    max_steps = int(math.ceil(4.0 * ring_radius / ds)) if max_steps is None else max_steps
    support_margin = max(2e-3, 2.0 * h) if support_margin is None else support_margin
    return rb_geometry(int(n_elem), float(ring_radius), int(nx), int(ny), float(h), int(n_rays), float(ds),
                       int(max_steps), float(support_margin), float(c_ref), float(f_ref), float(power_y))


def geometry_from_config(cfg, **over) -> rb_geometry:
    d = dict(n_elem=cfg.n_elem, ring_radius=cfg.ring_radius, nx=cfg.nx, ny=cfg.ny, h=cfg.h, n_rays=cfg.n_rays,
             ds=cfg.ds, max_steps=cfg.max_steps, support_margin=cfg.support_margin, c_ref=cfg.c_water,
             f_ref=1.0e6, power_y=cfg.power_y)
    d.update(over)
    return geometry(**d)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _freqs(freqs):
    arr = (ctypes.c_double * len(freqs))(*[float(f) for f in freqs])
    return arr, len(freqs)


def tc_supported(n_elem: int) -> bool:
    """Ring sizes the tensor-core (RB_PREC_BF16X3) contractions take."""
    return (64 <= n_elem <= 256 and n_elem % 64 == 0) or (n_elem % 256 == 0 and 512 <= n_elem <= 1024)


def rb_workspace_size(geom: rb_geometry, n_freq: int = 1, prec: int = RB_PREC_FP32) -> int:
    return int(load().rb_workspace_size(ctypes.byref(geom), int(n_freq), int(prec)))


def workspace(geom: rb_geometry, n_freq: int = 1, prec: int = RB_PREC_FP32, device="cuda"):
    """A 256-byte aligned uint8 CUDA tensor of rb_workspace_size bytes."""
    import torch
    n = rb_workspace_size(geom, n_freq, prec)
    if n == 0:
        raise RbError("rb_workspace_size", RB_ERR_SHAPE, "invalid geometry or frequency count")
    buf = torch.empty(n + 256, dtype=torch.uint8, device=device)
    off = (-buf.data_ptr()) % 256
    return buf[off:off + n]


def rb_trace_rays(geom, c, alpha0, ends, ws, samples=None, stream=None):
    """ends: uint8 tensor [n_elem, n_rays, 56]; samples: dict of vx, vy, vt, vq, vl, vkappa tensors or None."""
    r = rb_rays(ends.data_ptr(), None, None, None, None, None, None)
    if samples is not None:
        r.vx, r.vy, r.vt = samples["vx"].data_ptr(), samples["vy"].data_ptr(), samples["vt"].data_ptr()
        r.vq, r.vl, r.vkappa = samples["vq"].data_ptr(), samples["vl"].data_ptr(), samples["vkappa"].data_ptr()
    code = load().rb_trace_rays(ctypes.byref(geom), _ptr(c), _ptr(alpha0), ctypes.byref(r), _ptr(ws), ws.numel(),
                                _stream(stream))
    _check("rb_trace_rays", code)


def rb_green_grid(geom, c, alpha0, tables, ws, freqs=None, g_out=None, stream=None):
    """tables: int32 tensor [n_elem, npix, 4] (rb_cell records); g_out: complex64 [n_freq, n_elem, npix] or None."""
    fa, nf = _freqs(freqs) if freqs is not None else (None, 0)
    code = load().rb_green_grid(ctypes.byref(geom), _ptr(c), _ptr(alpha0), _ptr(tables), fa, nf, _ptr(g_out), _ptr(ws),
                                ws.numel(), _stream(stream))
    _check("rb_green_grid", code)


def rb_ray_forward(geom, c, ends, freqs, p_out, linked_out=None, stream=None):
    fa, nf = _freqs(freqs)
    code = load().rb_ray_forward(ctypes.byref(geom), _ptr(c), _ptr(ends), fa, nf, _ptr(p_out), _ptr(linked_out),
                                 _stream(stream))
    _check("rb_ray_forward", code)


def rb_data_weights(geom, c, alpha0, freqs, p_obs, resid_out, w_out, ws, outlier_frac=0.01, stream=None):
    """Residuals R = p_ray - p_obs and data weights W of one set: resid_out complex64 and w_out uint8,
    both [n_freq, n_elem, n_elem]; ws from workspace(geom, n_freq, RB_PREC_FP32)."""
    fa, nf = _freqs(freqs)
    code = load().rb_data_weights(ctypes.byref(geom), _ptr(c), _ptr(alpha0), fa, nf, _ptr(p_obs), float(outlier_frac),
                                  _ptr(resid_out), _ptr(w_out), _ptr(ws), ws.numel(), _stream(stream))
    _check("rb_data_weights", code)


def rb_born_forward(geom, tables, c, f_hz, m, d_out, ws, prec=RB_PREC_FP32, stream=None):
    code = load().rb_born_forward(ctypes.byref(geom), _ptr(tables), _ptr(c), float(f_hz), _ptr(m), _ptr(d_out),
                                  int(prec), _ptr(ws), ws.numel(), _stream(stream))
    _check("rb_born_forward", code)


def rb_born_forward_noalloc(geom, tables, c, f_hz, m, d_out, stream=None):
    """Born forward without a workspace (scratch inside the library; see include/rb.h)."""
    code = load().rb_born_forward_noalloc(ctypes.byref(geom), _ptr(tables), _ptr(c), float(f_hz), _ptr(m), _ptr(d_out),
                                          _stream(stream))
    _check("rb_born_forward_noalloc", code)


def rb_born_adjoint(geom, tables, c, f_hz, resid, w, g_out, ws, hdiag_out=None, prec=RB_PREC_FP32, stream=None):
    code = load().rb_born_adjoint(ctypes.byref(geom), _ptr(tables), _ptr(c), float(f_hz), _ptr(resid), _ptr(w),
                                  _ptr(g_out), _ptr(hdiag_out), int(prec), _ptr(ws), ws.numel(), _stream(stream))
    _check("rb_born_adjoint", code)


def stage_event_array(events):
    """A ctypes array of raw cudaEvent_t handles from 2 * len(STAGES) torch.cuda.Event objects."""
    arr = (ctypes.c_void_p * len(events))(*[ev.cuda_event for ev in events])
    return arr


def rb_hf_update(geom, c_inout, alpha0, freqs, p_obs, ws, outlier_frac=0.01, eps_rel=1e-3, step_mode=RB_STEP_EXACT,
                 prec=RB_PREC_FP32, dc_out=None, diag_out=None, stream=None, stage_events=None, tune=RB_TUNE_RULE):
    """stage_events: None or a ctypes array from stage_event_array (kept alive by the caller);
    tune: the rb_update_params.tune choice (tune.py picks it by timing)."""
    fa, nf = _freqs(freqs)
    prm = rb_update_params(float(outlier_frac), float(eps_rel), int(step_mode), int(tune),
                           ctypes.cast(stage_events, ctypes.c_void_p) if stage_events is not None else None)
    code = load().rb_hf_update(ctypes.byref(geom), _ptr(c_inout), _ptr(alpha0), fa, nf, _ptr(p_obs), ctypes.byref(prm),
                               int(prec), _ptr(dc_out), _ptr(diag_out), _ptr(ws), ws.numel(), _stream(stream))
    _check("rb_hf_update", code)


def rb_cg_update(geom, c_inout, alpha0, freqs, p_obs, ws, cg_iters, precond=True, outlier_frac=0.01, eps_rel=1e-3,
                 prec=RB_PREC_FP32, dc_out=None, hist_out=None, diag_out=None, stream=None, stage_events=None,
                 tune=RB_TUNE_RULE):
    """CG variant of the update; hist_out: None or a float64 device tensor of cg_iters + 1."""
    fa, nf = _freqs(freqs)
    prm = rb_update_params(float(outlier_frac), float(eps_rel), RB_STEP_EXACT, int(tune),
                           ctypes.cast(stage_events, ctypes.c_void_p) if stage_events is not None else None)
    code = load().rb_cg_update(ctypes.byref(geom), _ptr(c_inout), _ptr(alpha0), fa, nf, _ptr(p_obs), ctypes.byref(prm),
                               int(cg_iters), 1 if precond else 0, int(prec), _ptr(dc_out), _ptr(hist_out),
                               _ptr(diag_out), _ptr(ws), ws.numel(), _stream(stream))
    _check("rb_cg_update", code)


def rb_tof_times(geom, c, alpha0, t_out, ws, linked_out=None, stream=None):
    """Linked first-arrival times of flight: t_out [n_elem, n_elem] float64 device tensor."""
    code = load().rb_tof_times(ctypes.byref(geom), _ptr(c), _ptr(alpha0), _ptr(t_out), _ptr(linked_out), _ptr(ws),
                               ws.numel(), _stream(stream))
    _check("rb_tof_times", code)


def rb_tof_invert(geom, c_inout, alpha0, t_obs, obs_linked, ws, n_iter=3, resid_out=None, stream=None):
    """Time-of-flight initial guess: n_iter linearisations in place on c_inout."""
    code = load().rb_tof_invert(ctypes.byref(geom), _ptr(c_inout), _ptr(alpha0), _ptr(t_obs), _ptr(obs_linked),
                                int(n_iter), _ptr(resid_out), _ptr(ws), ws.numel(), _stream(stream))
    _check("rb_tof_invert", code)


# ---------------------------------------------------------------------------
# Record decoding (host side, numpy)
# ---------------------------------------------------------------------------
def decode_ends(ends_u8) -> np.ndarray:
    a = ends_u8.detach().cpu().numpy() if hasattr(ends_u8, "detach") else np.asarray(ends_u8)
    return np.ascontiguousarray(a).view(RAY_END_DTYPE).reshape(a.shape[:-1])


def decode_tables(tables_i32):
    """-> dict of numpy arrays t_res, q, l, kappa, tri, hit, each [n_elem, npix]."""
    a = tables_i32.detach().cpu().numpy() if hasattr(tables_i32, "detach") else np.asarray(tables_i32)
    rec = np.ascontiguousarray(a).view(CELL_DTYPE).reshape(a.shape[:-1])
    tkey = rec["tkey"].astype(np.uint32)
    hit = tkey != RB_HOLE
    pos = (tkey & 0x80000000) != 0
    bits = np.where(pos, tkey & 0x7FFFFFFF, ~tkey).astype(np.uint32)
    t_res = bits.view(np.float32).astype(np.float64)
    tag = rec["tag"].astype(np.int64)
    return dict(t_res=np.where(hit, t_res, 0.0), q=np.where(hit, rec["q"], 0.0), l=np.where(hit, rec["l"], 0.0),
                kappa=np.where(hit, tag & 0xFF, 0), tri=np.where(hit, tag >> 8, -1), hit=hit)


def decode_diag(diag_u8) -> dict:
    a = diag_u8.detach().cpu().numpy() if hasattr(diag_u8, "detach") else np.asarray(diag_u8)
    r = np.ascontiguousarray(a).view(DIAG_DTYPE)[0]
    return {k: r[k].item() for k in DIAG_DTYPE.names}

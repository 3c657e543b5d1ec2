"""Autotuner of the update's kernel-shape choices (``rb_update_params.tune``).

The rasteriser of the gridding has two work mappings, warps along the ray tubes or
across them, whose speed depends on how wide the tubes are against the pixels and on
how much the medium bends them; the library's rule picks by tube width alone.  The
tensor-core adjoint runs either on one CTA per pixel tile or on CTA pairs sharing each
MMA (cta_group::2), which halves the shared-memory traffic of the S operand per CTA.
The choices do not change the results, so only their time differs, and that is
measured here: for one problem, ``tune_update`` times the updates per candidate on
the caller's own data (a warm-up run, then ``reps`` timed ones, each from a scratch
copy of c, with CUDA events on a private stream; a whole sweep over the problem's
frequency sets when they are given), keeps the fastest and caches it per key (ring,
grid, pitch, fan, frequencies per set, precision) in memory and, when the environment
variable RB_TUNE_CACHE names a JSON file, in that file across processes.
"""
from __future__ import annotations

import json
import os
from typing import Dict, Optional, Tuple

from . import rb

RASTER = {rb.RB_TUNE_RASTER_ALONG: "raster along tubes", rb.RB_TUNE_RASTER_ACROSS: "raster across tubes"}
ADJOINT = {rb.RB_TUNE_ADJ_SINGLE: "adjoint one CTA per tile", rb.RB_TUNE_ADJ_PAIR: "adjoint CTA pairs"}


def candidates(prec: int):
    """The tune values tried for a precision: both raster mappings, and on the tensor-core
    path both forms of the adjoint."""
    if prec == rb.RB_PREC_BF16X3:
        return tuple(r | a for a in ADJOINT for r in RASTER)
    return tuple(RASTER)


def name(tune: int) -> str:
    parts = [RASTER.get(tune & 3, "raster by rule")]
    if tune & 12:
        parts.append(ADJOINT[tune & 12])
    return ", ".join(parts)


CANDIDATES = candidates(rb.RB_PREC_FP32)

_cache: Dict[str, dict] = {}


def key(geom, n_freq: int, prec: int) -> str:
    return (f"ne{geom.n_elem}_r{geom.ring_radius:.6g}_g{geom.nx}x{geom.ny}_h{geom.h:.6g}_rays{geom.n_rays}"
            f"_ds{geom.ds:.6g}_nf{n_freq}_p{prec}")


def _load_file() -> Dict[str, dict]:
    path = os.environ.get("RB_TUNE_CACHE")
    if not path or not os.path.exists(path):
        return {}
    try:
        with open(path) as f:
            d = json.load(f)
        return d if isinstance(d, dict) else {}
    except (OSError, ValueError):
        return {}


def _store_file(k: str, entry: dict) -> None:
    path = os.environ.get("RB_TUNE_CACHE")
    if not path:
        return
    d = _load_file()
    d[k] = entry
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def cached(geom, n_freq: int, prec: int) -> Optional[dict]:
    k = key(geom, n_freq, prec)
    if k not in _cache:
        e = _load_file().get(k)
        if e is not None:
            _cache[k] = e
    return _cache.get(k)


def tune_update(geom, c, alpha0, freqs, p_obs, prec, reps: int = 3, device=None, sets=None) -> Tuple[int, dict]:
    """The fastest ``tune`` value for this problem, and the timings (ms per candidate,
    median of ``reps``).  Without ``sets`` one rb_hf_update of the frequencies ``freqs``
    (data p_obs[len(freqs)]) is timed; with ``sets`` (index lists into ``freqs``, data
    p_obs[len(freqs)]) the whole sweep over them is, from c each time, because the
    medium the later sets see (rougher, with bent tubes) changes which choice is faster.
    c is not modified; the result is cached."""
    import torch
    nf = max(len(s) for s in sets) if sets else len(freqs)
    hit = cached(geom, nf, prec)
    if hit is not None:
        return int(hit["tune"]), hit
    dev = c.device if device is None else device
    stream = torch.cuda.Stream(device=dev)
    plan = [list(s) for s in sets] if sets else [list(range(len(freqs)))]
    times = {}
    with torch.cuda.stream(stream):
        ws = rb.workspace(geom, nf, prec, dev)
        cs = torch.empty_like(c)
        for cand in candidates(prec):
            ms = []
            for r in range(reps + 1):
                cs.copy_(c)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for s in plan:
                    rb.rb_hf_update(geom, cs, alpha0, [freqs[i] for i in s], p_obs[s[0]:s[-1] + 1], ws, prec=prec,
                                    stream=stream, tune=cand)
                e1.record(stream)
                e1.synchronize()
                if r > 0:
                    ms.append(e0.elapsed_time(e1) / len(plan))
            ms.sort()
            times[name(cand)] = ms[len(ms) // 2]
        del ws, cs
    best = min(candidates(prec), key=lambda t: times[name(t)])
    entry = {"tune": int(best), "choice": name(best), "ms_per_update": times,
             "timed": "sweep of %d sets" % len(plan) if sets else "one update"}
    k = key(geom, nf, prec)
    _cache[k] = entry
    _store_file(k, entry)
    return int(best), entry

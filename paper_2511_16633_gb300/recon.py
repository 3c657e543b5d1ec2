"""Device-resident driver for sweeps of ray-Born updates (marshalling only).

``Reconstruction`` owns the device buffers of one problem (sound speed,
absorption, measured data, workspace) and calls ``rb_hf_update`` (or, for the
CG variant, ``rb_cg_update``) once per frequency set, low to high, leaving c(x)
resident between sets.  ``compare_solvers`` (``python -m
paper_2511_16633_gb300.recon``) runs the one-step update against CG updates.  ``synth_data``
builds synthetic measurements on the device through the library's own
forward entry points (ray data plus Born-scattered data about a background
model, plus seeded noise); it is input preparation for benchmarks and demos.
"""
from __future__ import annotations

import math
from typing import List, Sequence

import numpy as np

from . import rb


def _support_mask(geom, device):
    import torch
    q = 2.0 * (geom.ring_radius - geom.support_margin) / geom.h
    r2max = math.floor(q * q)
    jx = 2 * torch.arange(geom.nx, device=device, dtype=torch.int64) - (geom.nx - 1)
    jy = 2 * torch.arange(geom.ny, device=device, dtype=torch.int64) - (geom.ny - 1)
    return (jy[:, None] ** 2 + jx[None, :] ** 2) <= r2max


def receiver_mask(n_elem: int, device):
    import torch
    e = torch.arange(n_elem, device=device)
    d = (e[:, None] - e[None, :]).abs()
    d = torch.minimum(d, n_elem - d)
    return d >= math.ceil(n_elem / 8)


def synth_data(geom, c0, c_true, alpha0, freqs: Sequence[float], noise_re=None, noise_im=None, level=0.01,
               prec=rb.RB_PREC_FP32):
    """p_obs[n_freq, n_elem, n_elem] complex64 on the device:
    p_ray(c0) + B(c0) m_true (+ level * masked-rms * (n1 + i n2)/sqrt 2), m_true = -2 h^2 (c_true - c0)/c0^3."""
    import torch
    dev = c0.device
    ne, npix = geom.n_elem, geom.nx * geom.ny
    ws = rb.workspace(geom, 1, prec, dev)
    ends = torch.empty((ne, geom.n_rays, 56), dtype=torch.uint8, device=dev)
    rb.rb_trace_rays(geom, c0, alpha0, ends, ws)
    tables = torch.empty((ne, npix, 4), dtype=torch.int32, device=dev)
    rb.rb_green_grid(geom, c0, alpha0, tables, ws)
    sup = _support_mask(geom, dev).reshape(-1)
    c0d, ctd = c0.reshape(-1).double(), c_true.reshape(-1).double()
    m = torch.where(sup, -2.0 * geom.h * geom.h * (ctd - c0d) / c0d ** 3, torch.zeros_like(c0d)).float().contiguous()
    p = torch.empty((len(freqs), ne, ne), dtype=torch.complex64, device=dev)
    for j0 in range(0, len(freqs), rb.RB_MAX_FREQ):
        j1 = min(len(freqs), j0 + rb.RB_MAX_FREQ)
        rb.rb_ray_forward(geom, c0, ends, list(freqs[j0:j1]), p[j0:j1])
    d = torch.empty((ne, ne), dtype=torch.complex64, device=dev)
    mask = receiver_mask(ne, dev)
    for j, f in enumerate(freqs):
        rb.rb_born_forward(geom, tables, c0, f, m, d, ws, prec)
        p[j] += d
        if noise_re is not None and level > 0:
            rms = torch.sqrt(torch.mean(torch.abs(p[j][mask]) ** 2))
            nz = torch.complex(torch.as_tensor(noise_re[j], device=dev, dtype=torch.float32),
                               torch.as_tensor(noise_im[j], device=dev, dtype=torch.float32))
            p[j] += (level * rms / math.sqrt(2.0)) * nz
    return p


class Reconstruction:
    """One problem resident on the device; update(j) runs frequency set j."""

    def __init__(self, cfg, c_init, alpha0, p_obs, prec=rb.RB_PREC_FP32, outlier_frac=0.01, eps_rel=1e-3,
                 step_mode=rb.RB_STEP_EXACT, device="cuda", cg_iters=0, cg_precond=True, tune=rb.RB_TUNE_RULE):
        """cg_iters > 0 solves each set's linear equation by that many CG iterations
        (rb_cg_update) instead of the one-step update.  tune: an rb_update_params.tune value,
        or "auto" to time the choices on this problem's sweep (tune.py; cached per problem
        shape)."""
        import torch
        self.cfg = cfg
        self.geom = rb.geometry_from_config(cfg)
        self.prec = prec
        self.outlier_frac, self.eps_rel, self.step_mode = outlier_frac, eps_rel, step_mode
        self.cg_iters, self.cg_precond = int(cg_iters), bool(cg_precond)
        self.device = torch.device(device)
        self.c = torch.as_tensor(np.asarray(c_init, dtype=np.float32), device=self.device).contiguous().clone()
        self.alpha0 = torch.as_tensor(np.asarray(alpha0, dtype=np.float32), device=self.device).contiguous()
        self.p_obs = torch.as_tensor(p_obs, device=self.device).to(torch.complex64).contiguous()
        self.max_set = max(len(s) for s in cfg.sets)
        self.ws = rb.workspace(self.geom, self.max_set, prec, self.device)
        self.dc = torch.empty_like(self.c)
        self.diag = torch.zeros(48, dtype=torch.uint8, device=self.device)
        self.norms: List[float] = []
        self.tune_info = None
        if tune == "auto":
            from .tune import tune_update
            tune, self.tune_info = tune_update(self.geom, self.c, self.alpha0, list(cfg.freqs_hz), self.p_obs, prec,
                                               reps=2, sets=cfg.sets)
        self.tune = int(tune)

    def update(self, j: int, stream=None):
        s = self.cfg.sets[j]
        freqs = [self.cfg.freqs_hz[i] for i in s]
        lo, hi = s[0], s[-1] + 1
        if list(s) != list(range(lo, hi)):
            raise ValueError("frequency sets must be consecutive")
        if self.cg_iters > 0:
            rb.rb_cg_update(self.geom, self.c, self.alpha0, freqs, self.p_obs[lo:hi], self.ws, self.cg_iters,
                            self.cg_precond, self.outlier_frac, self.eps_rel, self.prec, self.dc, None, self.diag,
                            stream, tune=self.tune)
        else:
            rb.rb_hf_update(self.geom, self.c, self.alpha0, freqs, self.p_obs[lo:hi], self.ws, self.outlier_frac,
                            self.eps_rel, self.step_mode, self.prec, self.dc, self.diag, stream, tune=self.tune)

    def diagnostics(self) -> dict:
        return rb.decode_diag(self.diag)

    def sweep(self):
        self.norms = []
        for j in range(len(self.cfg.sets)):
            self.update(j)
            self.norms.append(self.diagnostics()["dc_norm"])
        return self.c


def tof_guess(cfg, n_iter: int = 3, device="cuda", noise_s: float = 0.0, c_start=None):
    """The time-of-flight initial guess: times of flight through the true phantom
    (rb_tof_times; plus noise_s seconds times the seeded normal draws, as picking
    jitter), then n_iter linearisations (rb_tof_invert) from water (or c_start).
    Returns (c [device], RMS misfit history [s], device milliseconds of the inversion)."""
    import torch

    import rbgen
    dev = torch.device(device)
    inp = rbgen.make_inputs(cfg)
    geom = rb.geometry_from_config(cfg)
    n = cfg.n_elem
    ws = rb.workspace(geom, 1, rb.RB_PREC_FP32, dev)
    a0 = torch.as_tensor(inp.alpha0, device=dev, dtype=torch.float32).contiguous()
    ct = torch.as_tensor(inp.c_true, device=dev, dtype=torch.float32).contiguous()
    T = torch.zeros((n, n), dtype=torch.float64, device=dev)
    lk = torch.zeros((n, n), dtype=torch.uint8, device=dev)
    rb.rb_tof_times(geom, ct, a0, T, ws, lk)
    if noise_s > 0:
        T += noise_s * torch.as_tensor(inp.noise_re[0], device=dev, dtype=torch.float64)
    if c_start is None:
        c = torch.full((cfg.ny, cfg.nx), float(cfg.c_water), device=dev, dtype=torch.float32)
    else:
        c = torch.as_tensor(np.asarray(c_start, dtype=np.float32), device=dev).contiguous().clone()
    hist = torch.zeros(n_iter + 1, dtype=torch.float64, device=dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    e0.record()
    rb.rb_tof_invert(geom, c, a0, T, lk, ws, n_iter, hist)
    e1.record()
    e1.synchronize()
    return c, hist.cpu().numpy().tolist(), e0.elapsed_time(e1)


def compare_solvers(cfg, variants: Sequence[int], prec=rb.RB_PREC_BF16X3, device="cuda", precond=True,
                    data: str = "born") -> dict:
    """Full sweeps of one synthetic problem with the one-step update (variant 0) and with
    CG updates of k iterations (variant k): per variant the RMS error of c against the
    true phantom over the support after every set, and the device time of the sweep.
    data "born": ray data about c_init plus the Born-scattered data of the contrast (as
    ``synth_data``); "ray": the ray-model data of the true medium (no scattering term)."""
    import torch

    import rbgen
    dev = torch.device(device)
    inp = rbgen.make_inputs(cfg)
    geom = rb.geometry_from_config(cfg)
    c0 = torch.as_tensor(inp.c_init, device=dev).contiguous()
    a0 = torch.as_tensor(inp.alpha0, device=dev).contiguous()
    ct = torch.as_tensor(inp.c_true, device=dev).contiguous()
    if data == "born":
        p = synth_data(geom, c0, ct, a0, list(cfg.freqs_hz), inp.noise_re, inp.noise_im, 0.01, prec)
    elif data == "ray":
        p = synth_data(geom, ct, ct, a0, list(cfg.freqs_hz), inp.noise_re, inp.noise_im, 0.01, prec)
    else:
        raise ValueError(data)
    sup = _support_mask(geom, dev)

    def rms():
        return float(torch.sqrt(torch.mean((rec.c - ct)[sup].double() ** 2)))

    out = {"workload": cfg.name, "data": data, "precond": precond, "n_sets": len(cfg.sets), "rms_init": float(torch.sqrt(torch.mean((c0 - ct)[sup].double() ** 2))),
           "variants": []}
    for k in variants:
        rec = Reconstruction(cfg, inp.c_init, inp.alpha0, p, prec=prec, device=dev, cg_iters=k, cg_precond=precond)
        rec.update(0)   # warm-up (and first-use setup) on set 0, then the timed sweep from c_init
        rec.c.copy_(c0)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        errs = []
        ms = 0.0
        for j in range(len(cfg.sets)):
            e0.record()
            rec.update(j)
            e1.record()
            e1.synchronize()
            ms += e0.elapsed_time(e1)
            errs.append(rms())
        out["variants"].append({"solver": "one-step" if k == 0 else f"cg{k}", "sweep_ms": ms, "rms_after_set": errs})
        del rec
        torch.cuda.empty_cache()
    return out


def pipeline(cfg, tof_iters: int = 3, prec=rb.RB_PREC_BF16X3, device="cuda") -> dict:
    """The paper's workflow on one synthetic problem: the time-of-flight guess from water
    (tof_iters linearisations), then the one-step ray-Born sweep from that image over the
    frequency sets, low to high.  Data: the ray-model data of the true medium plus 1 %
    noise, and its linked times of flight.  Returns the RMS error of c against the phantom
    over the support after each stage and the device times."""
    import torch

    import rbgen
    dev = torch.device(device)
    inp = rbgen.make_inputs(cfg)
    geom = rb.geometry_from_config(cfg)
    ct = torch.as_tensor(inp.c_true, device=dev, dtype=torch.float32).contiguous()
    a0 = torch.as_tensor(inp.alpha0, device=dev, dtype=torch.float32).contiguous()
    p = synth_data(geom, ct, ct, a0, list(cfg.freqs_hz), inp.noise_re, inp.noise_im, 0.01, prec)
    sup = _support_mask(geom, dev)

    def rms(c):
        return float(torch.sqrt(torch.mean((c - ct)[sup].double() ** 2)))

    c_tof, hist, tof_ms = tof_guess(cfg, tof_iters, device)
    out = {"workload": cfg.name, "rms_water": rms(torch.full_like(ct, float(cfg.c_water))), "rms_tof": rms(c_tof),
           "tof_ms": tof_ms, "tof_misfit_s": hist}
    rec = Reconstruction(cfg, c_tof.cpu().numpy(), inp.alpha0, p, prec=prec, device=dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    errs, ms = [], 0.0
    for j in range(len(cfg.sets)):
        e0.record()
        rec.update(j)
        e1.record()
        e1.synchronize()
        ms += e0.elapsed_time(e1)
        errs.append(rms(rec.c))
    out.update(sweep_ms=ms, rms_after_set=errs)
    return out


def main():
    import argparse
    import json

    import rbgen
    ap = argparse.ArgumentParser(description="one-step update against CG updates over a full sweep")
    ap.add_argument("--workload", default="breast512", choices=sorted(rbgen.CONFIGS))
    ap.add_argument("--cg", default="0,4,12", help="comma-separated CG iteration counts (0: one-step update)")
    ap.add_argument("--prec", default="bf16x3", choices=["fp32", "bf16x3"])
    ap.add_argument("--plain-cg", action="store_true", help="CG without the diagonal preconditioner")
    ap.add_argument("--data", default="born", choices=["born", "ray"])
    ap.add_argument("--tof", type=int, default=0,
                    help="only the time-of-flight initial guess with this many linearisations (timing and error)")
    ap.add_argument("--pipeline", action="store_true",
                    help="time-of-flight guess, then the one-step sweep from it, on ray data of the true medium")
    a = ap.parse_args()
    if a.pipeline:
        prec = rb.RB_PREC_BF16X3 if a.prec == "bf16x3" else rb.RB_PREC_FP32
        print(json.dumps(pipeline(rbgen.config_by_name(a.workload), 3, prec)), flush=True)
        return
    if a.tof > 0:
        import torch
        cfg = rbgen.config_by_name(a.workload)
        inp = rbgen.make_inputs(cfg)
        tof_guess(cfg, a.tof)   # warm-up
        out = {"workload": cfg.name, "tof_iters": a.tof}
        for noise in (0.0, 20e-9):
            c, hist, ms = tof_guess(cfg, a.tof, noise_s=noise)
            sup = _support_mask(rb.geometry_from_config(cfg), c.device)
            ct = torch.as_tensor(inp.c_true, device=c.device, dtype=torch.float32)
            water = torch.full_like(ct, float(cfg.c_water))
            ci = torch.as_tensor(inp.c_init, device=c.device, dtype=torch.float32)
            rms = lambda x: float(torch.sqrt(torch.mean((x - ct)[sup].double() ** 2)))
            out[f"noise_{noise * 1e9:.0f}ns"] = {"ms": ms, "misfit_s": hist, "rms_water": rms(water),
                                                "rms_tof": rms(c), "rms_smooth_stand_in": rms(ci)}
        print(json.dumps(out), flush=True)
        return
    prec = rb.RB_PREC_BF16X3 if a.prec == "bf16x3" else rb.RB_PREC_FP32
    res = compare_solvers(rbgen.config_by_name(a.workload), [int(x) for x in a.cg.split(",")], prec,
                          precond=not a.plain_cg, data=a.data)
    print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()

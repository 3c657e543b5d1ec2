#!/usr/bin/env python3
"""Benchmark: ray-Born updates/s on the 256-element ring, 512x512 grid (breast phantom).

One step = one ``rb_hf_update`` on one frequency set of 4 frequencies: field
prep, fused ray fans + gridding, ray linking + residuals + data weights, Born
adjoint + Hessian diagonal over the set, the step's line search (Born forward
of the direction over the set) and the update of c.  Sets are taken in sweep
order, c evolving; after the last set c is restored from a device copy
(outside the timed kernels, inside the wall-clock bracket: a 1 MB copy).

Prints one JSON line (see the keys below).  ``--impl reference`` times the
FP64 CPU oracle on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import rbgen  # noqa: E402

WORKLOAD = "breast512"
METRIC = "ray-Born updates/s, 256-el ring 512² grid, mixed vs plain FP32; p50/p99 ms"


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, "fallback"


def _cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.proc = None
        self.path = os.path.join("/tmp", f"rb_clocks_{os.getpid()}.csv")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append(dict(sm=float(f[1]), smax=float(f[2]), hw=f[5], hwt=f[6], swt=f[7], pcap=f[8]))
            except ValueError:
                continue
        if not rows:
            return None
        reasons = set()
        for r in rows:
            for k, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"), ("swt", "sw_thermal_slowdown"),
                            ("pcap", "sw_power_cap")):
                if r[k].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": float(np.median([r["sm"] for r in rows])), "sm_max_mhz": rows[0]["smax"],
                "samples": len(rows), "reasons": sorted(reasons)}


def combine_ranks(ms_local, steps, world, device=None):
    """Whole-job throughput of `world` replicas: the slowest rank's time for the timed
    steps (all-reduce max; every rank gets it) and the updates of all ranks over that
    time.  Returns (ms, updates/s)."""
    ms = float(ms_local)
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, world * steps / (ms / 1e3)


def algorithmic_work(cfg, n_freq):
    """Per-update algorithmic work of the contractions (FLOP), complex products written out
    in real arithmetic: per frequency the adjoint's U = S conj(G) (8 n^2 npix), its Hessian
    contraction W |G|^2 (2 n^2 npix) and the two epilogues (10 n npix); the forward's
    G diag(m) G^T (8 n^2 npix)."""
    ne, npix = cfg.n_elem, cfg.nx * cfg.ny
    adj_flop = n_freq * (8.0 * ne * ne * npix + 2.0 * ne * ne * npix + 10.0 * ne * npix)
    fwd_flop = n_freq * 8.0 * ne * ne * npix
    table_bytes = ne * npix * 16.0
    return dict(adjoint_flop=adj_flop, forward_flop=fwd_flop, trace_grid_bytes=table_bytes)


# Tensor FLOPs the BF16 x3 path issues per algorithmic FLOP: the gradient contraction
# (8 n^2 npix per frequency) takes three bf16 products (hi.hi, hi.lo, lo.hi), the Hessian
# contraction (2 n^2 npix) two (W is exact in bf16): (3 x 8 + 2 x 2) / (8 + 2).
ADJ_ISSUE_RATIO = 2.8
# dram__bytes_read.sum + dram__bytes_write.sum of one k_adjoint_tc launch on breast512 from
# one ncu capture (--metrics, one pass) of the kernel as it stands in ADJ_TRAFFIC_SOURCE;
# set to None whenever the kernel changes until it is captured again.
ADJ_TRAFFIC_BYTES = 2157880064 + 1073678080
ADJ_TRAFFIC_SOURCE = ("ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum, one k_adjoint_tc launch on "
                      "breast512, kernel as of commit e24a358 (profiles/launches_breast512_bf16x3.md)")


def rays_grid_bytes(cfg, n_vertices):
    """Algorithmic HBM bytes of the ray and gridding stage of one update: every ray vertex
    (x, y, T, Q, L, kappa: 24 bytes) written once by the tracer and read once by the
    gridding, the per-(element, pixel) first-arrival record (16 bytes) written once, its
    64-bit first-arrival key written and read once (16 bytes), and the 7 field grids read
    once."""
    ne, npix = cfg.n_elem, cfg.nx * cfg.ny
    return 48.0 * n_vertices + 16.0 * ne * npix + 16.0 * ne * npix + 28.0 * npix


def workload_config(workload, head, world):
    """The config object of the JSON line, the same for both arms."""
    cfg = rbgen.config_by_name(workload)
    return {"workload": workload, "n_elem": cfg.n_elem, "grid": [cfg.nx, cfg.ny], "h_m": cfg.h,
            "n_rays": cfg.n_rays, "freqs_per_set": max(len(s) for s in cfg.sets), "n_sets": len(cfg.sets),
            "precision": head, "step_mode": "exact",
            "l2": "per-update working set (1.1 GB tables) larger than L2, no flush",
            "parallelism": "replicas" if world > 1 else "single"}


def run_ours(args):
    import torch
    from paper_2511_16633_gb300 import rb
    from paper_2511_16633_gb300.recon import synth_data

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    precs = {"fp32": rb.RB_PREC_FP32, "bf16x3": rb.RB_PREC_BF16X3}

    cfg = rbgen.config_by_name(args.workload)
    inp = rbgen.make_inputs(cfg)
    geom = rb.geometry_from_config(cfg)
    c0 = torch.as_tensor(inp.c_init, device=dev).contiguous()
    a0 = torch.as_tensor(inp.alpha0, device=dev).contiguous()
    ct = torch.as_tensor(inp.c_true, device=dev).contiguous()
    p_obs = synth_data(geom, c0, ct, a0, list(cfg.freqs_hz), inp.noise_re, inp.noise_im, 0.01)
    nsets = len(cfg.sets)
    nf = max(len(s) for s in cfg.sets)
    stream = torch.cuda.current_stream()
    # vertices of the rays through c_init (the algorithmic bytes of the ray and gridding stage)
    ends_u8 = torch.empty((cfg.n_elem, cfg.n_rays, 56), dtype=torch.uint8, device=dev)
    ws1 = rb.workspace(geom, 1, rb.RB_PREC_FP32, dev)
    rb.rb_trace_rays(geom, c0, a0, ends_u8, ws1)
    n_vertices = int(np.maximum(rb.decode_ends(ends_u8)["n_vert"], 0).sum())
    del ws1, ends_u8
    nst = len(rb.STAGES)

    tuned = {}

    def tune_for(prec):
        # the kernel-shape choice measured fastest on this problem (tune.py), before any timing
        if args.tune == "off":
            return rb.RB_TUNE_RULE
        if args.tune not in ("on", "off"):
            return int(args.tune)    # a fixed kernel-shape code (rb_update_params.tune)
        if prec not in tuned:
            from paper_2511_16633_gb300.tune import tune_update
            tuned[prec] = tune_update(geom, c0, a0, list(cfg.freqs_hz), p_obs, prec, reps=2, sets=cfg.sets)
            torch.cuda.empty_cache()
        return tuned[prec][0]

    def measure(prec_name, with_clocks, cg_iters=0, n_steps=None):
        prec = precs[prec_name]
        n_steps = args.steps if n_steps is None else n_steps
        tch = tune_for(prec)
        ws = rb.workspace(geom, nf, prec, dev)
        c = c0.clone()
        dc = torch.empty_like(c)
        diag = torch.zeros(48, dtype=torch.uint8, device=dev)
        def step(k, events=None):
            j = k % nsets
            # the one-step update sweeps the sets from c_init; the CG variant starts every
            # update from c_init (CG fits the Born data far more closely than the one-step
            # update and a sweep on them leaves the range where they are valid)
            if j == 0 or cg_iters:
                c.copy_(c0)
            s = cfg.sets[j]
            if cg_iters:
                rb.rb_cg_update(geom, c, a0, [cfg.freqs_hz[i] for i in s], p_obs[s[0]:s[-1] + 1], ws, cg_iters, True,
                                0.01, 1e-3, prec, dc, None, diag, stream, events, tune=tch)
                return
            rb.rb_hf_update(geom, c, a0, [cfg.freqs_hz[i] for i in s], p_obs[s[0]:s[-1] + 1], ws, 0.01, 1e-3,
                            rb.RB_STEP_EXACT, prec, dc, diag, stream, events, tune=tch)

        for k in range(args.warmup):
            step(k)
        torch.cuda.synchronize()
        stage_ms = np.zeros(nst)
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(n_steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(n_steps)]
        # stage events of their own for every timed step, so the steps are queued back to back
        # (no synchronisation between them) and the stage times are read after the last
        step_evs = [[torch.cuda.Event(enable_timing=True) for _ in range(2 * nst)] for _ in range(n_steps)]
        for es in step_evs:
            for e in es:
                e.record(stream)
        step_arrs = [rb.stage_event_array(es) for es in step_evs]
        clocks = ClockSampler(local) if with_clocks else None
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(n_steps):
            starts[k].record(stream)
            step(args.warmup + k, step_arrs[k])
            ends[k].record(stream)
        torch.cuda.synchronize()
        for k in range(n_steps):
            for s_ in range(nst):
                stage_ms[s_] += step_evs[k][2 * s_].elapsed_time(step_evs[k][2 * s_ + 1])
        if world > 1:
            torch.distributed.barrier()
        wall = time.perf_counter() - t0
        clk = clocks.stop() if clocks else None
        per_step = np.array([starts[k].elapsed_time(ends[k]) for k in range(n_steps)])
        ms, value = combine_ranks(float(np.sum(per_step)), n_steps, world, dev)
        out = {"value": value, "ms_per_step": ms / n_steps,
               "p50_ms": float(np.percentile(per_step, 50)), "p99_ms": float(np.percentile(per_step, 99)),
               "stage_ms": {name: round(stage_ms[i] / n_steps, 4) for i, name in enumerate(rb.STAGES)},
               "wall_s": wall, "clocks": clk, "diag": rb.decode_diag(diag)}

        if cg_iters:
            del ws
            torch.cuda.empty_cache()
            return out
        # end to end through the same call: pinned host data in, c and diagnostics out, every step
        host_p = torch.empty(p_obs.shape, dtype=p_obs.dtype, pin_memory=True)
        host_p.copy_(p_obs.cpu())
        host_c = torch.empty(c.shape, dtype=c.dtype, pin_memory=True)
        host_diag = torch.empty(48, dtype=torch.uint8, pin_memory=True)
        dev_p = torch.empty((nf,) + tuple(p_obs.shape[1:]), dtype=p_obs.dtype, device=dev)
        e2e_steps = max(3, min(args.steps, 10))
        torch.cuda.synchronize()
        te0 = time.perf_counter()
        for k in range(e2e_steps):
            j = k % nsets
            if j == 0:
                c.copy_(c0)
            s = cfg.sets[j]
            dev_p[:len(s)].copy_(host_p[s[0]:s[-1] + 1], non_blocking=True)
            rb.rb_hf_update(geom, c, a0, [cfg.freqs_hz[i] for i in s], dev_p[:len(s)], ws, 0.01, 1e-3,
                            rb.RB_STEP_EXACT, prec, dc, diag, stream, tune=tch)
            host_c.copy_(c, non_blocking=True)
            host_diag.copy_(diag, non_blocking=True)
            stream.synchronize()
        te = time.perf_counter() - te0
        out["e2e"] = {"value": e2e_steps / te, "unit": "updates/s",
                      "h2d_bytes_per_step": int(nf * p_obs.shape[1] * p_obs.shape[2] * 8),
                      "d2h_bytes_per_step": int(c.numel() * 4 + 48)}
        del ws
        torch.cuda.empty_cache()
        return out

    head = args.prec
    runs = {head: measure(head, True)}
    other = "fp32" if head == "bf16x3" else "bf16x3"
    if not args.no_compare:
        runs[other] = measure(other, False)
    R = runs[head]
    cg = None
    if args.cg_iters > 0:
        # the CG variant of the same update (the paper's comparison: 10-15 iterations per set)
        o = measure(head, False, cg_iters=args.cg_iters, n_steps=max(3, min(args.steps, 20)))
        cg = {"iters": args.cg_iters, "precond": "diagonal Hessian", "start": "c_init every update",
              "updates_per_s": o["value"],
              "ms_per_update": o["ms_per_step"], "stage_ms": o["stage_ms"],
              "time_vs_one_step": o["ms_per_step"] / R["ms_per_step"],
              # the gradient stages, 4 CG start kernels, per iteration a forward (+ reduce) and a
              # B-image prep (mixed path) per frequency, one partial sum, the adjoint (+ its sum over
              # the set's frequencies on the mixed path) and 3 vector kernels, then 3 apply/norm kernels
              "gpu_launches_per_update": (20 + nf + args.cg_iters * (3 * nf + 6) if head == "bf16x3"
                                          else 19 + args.cg_iters * (2 * nf + 5))}
    peaks, peak_src = _peaks()
    work = algorithmic_work(cfg, nf)
    st = R["stage_ms"]
    fp32_peak = 152 * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    bf16_burst = peaks.get("bf16_tflops", 1900.0)

    def contraction_roof(stage, flop, kern, issue_ratio):
        t = st[stage] / 1e3
        ach = flop / t / 1e12
        if head == "bf16x3":
            # algorithmic FLOP/s against the measured bf16 burst rate (a kernel of ~1 ms);
            # the 3-product split's extra tensor work is reported apart as issue utilisation
            return {"kernel": kern, "bound": "tensor", "achieved": ach, "peak": bf16_burst, "unit": "TFLOP/s",
                    "frac": ach / bf16_burst, "traffic": None,
                    "tensor_issued_tflops": ach * issue_ratio, "tensor_issue_frac": ach * issue_ratio / bf16_burst,
                    "issue_ratio": issue_ratio,
                    "peak_source": f"{peak_src} bf16 burst (MEASURED_PEAKS.json bf16_tflops, {bf16_burst} TFLOP/s); "
                                   f"algorithmic FLOP only, split-precision extras excluded"}
        return {"kernel": kern, "bound": "alu", "achieved": ach, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": ach / fp32_peak, "traffic": None,
                "peak_source": "derived: 152 SM x 128 FP32 lanes x 2 x max SM clock"}

    tc = head == "bf16x3"
    # forward: the kernels compute the column blocks on and above the block diagonal of the
    # symmetric real-form product (for 2n = 512 and 256-wide blocks: 6 of 8 block pairs)
    nbn = (2 * cfg.n_elem + 255) // 256
    nb = 2 * cfg.n_elem // nbn
    nmb = 2 * cfg.n_elem // 128
    done = sum(nbn - (128 * i) // nb for i in range(nmb))
    fwd_ratio = 3.0 * done / (nmb * nbn)
    roof_adj = contraction_roof("adjoint", work["adjoint_flop"], "k_adjoint_tc" if tc else "k_adjoint_simt",
                                ADJ_ISSUE_RATIO)
    roof_fwd = contraction_roof("forward", work["forward_flop"], "k_forward_tc" if tc else "k_forward_simt", fwd_ratio)
    # the dominant kernel: the adjoint contraction (one launch per update, alone in its stage)
    roof = dict(roof_adj)
    if tc and args.workload == WORKLOAD and ADJ_TRAFFIC_BYTES is not None:
        roof["traffic"] = ADJ_TRAFFIC_BYTES   # captured on the default workload only
        roof["traffic_source"] = ADJ_TRAFFIC_SOURCE
    hbm = peaks.get("hbm_gbs", 6800.0)
    # the ray and gridding stage against the HBM roofline (its algorithmic bytes / stage time)
    rg_bytes = rays_grid_bytes(cfg, n_vertices)
    rg_ach = rg_bytes / (st["trace_grid"] / 1e3) / 1e9
    roof_rg = {"kernels": ["k_trace", "k_raster", "k_resolve"], "bound": "hbm", "achieved": rg_ach, "peak": hbm,
               "unit": "GB/s", "frac": rg_ach / hbm, "bytes_per_update": rg_bytes, "vertices": n_vertices,
               "traffic": None,
               "peak_source": f"{peak_src} hbm_gbs (MEASURED_PEAKS.json)",
               "note": "algorithmic bytes: 24 B per ray vertex written and read, 16 B first-arrival record "
                       "written, 16 B key written and read per (element, pixel), field grids read; vertex "
                       "count of the rays through c_init"}
    # the operand-image synthesis (mixed path): HBM-bound; algorithmic bytes = the synthesis
    # records read once and the operand image (bf16 hi and lo of 2n x npix) of every
    # frequency of the set written once
    roof_img = None
    if tc and st.get("images", 0.0) > 0.05:   # a separate synthesis pass (not the fused resolve)
        npix = cfg.nx * cfg.ny
        img_bytes = cfg.n_elem * npix * 16.0 + nf * (2 * cfg.n_elem) * npix * 2 * 2.0
        ach = img_bytes / (st["images"] / 1e3) / 1e9
        roof_img = {"kernel": "k_synth_images", "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                    "frac": ach / hbm, "traffic": None, "bytes_per_launch": img_bytes,
                    "peak_source": f"{peak_src} hbm_gbs (MEASURED_PEAKS.json)" if peak_src == "measured" else "fallback"}
    line = {
        "metric": METRIC, "value": R["value"], "unit": "updates/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": R["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16x3 split products, f32 accumulate" if tc else "f32",
        "data": "synthetic (seeded breast phantom; data from the library's own ray-Born forward model + 1% noise)",
        "config": workload_config(args.workload, head, world),
        "p50_ms": R["p50_ms"], "p99_ms": R["p99_ms"], "stage_ms": st, "wall_s": R["wall_s"],
        "roofline": roof, "roofline_contractions": {"adjoint": roof_adj, "forward": roof_fwd},
        "roofline_images": roof_img, "roofline_rays_grid": roof_rg,
        "clocks": R["clocks"], "e2e": R["e2e"],
        # launches per update: positions, fields, keys reset, trace/raster/resolve (the resolve pass writes
        # the operand images on the mixed path), link, residual keys and the three selection
        # passes, adjoint (+ one B-image prep per frequency and the sum over the set's frequencies
        # on the mixed path), 4 direction kernels, forward + reduce per frequency, 4 apply/norm kernels
        "gpu_launches": (21 + 3 * nf) * args.steps if tc else (20 + 2 * nf) * args.steps,
        "diag_last": {k: R["diag"][k] for k in ("dc_norm", "alpha", "lost_rays", "holes", "kept", "zeroed")},
    }
    if tuned:
        line["tune"] = {("bf16x3" if p == rb.RB_PREC_BF16X3 else "fp32"): v[1] for p, v in tuned.items()}
    elif args.tune not in ("on", "off"):
        line["tune"] = {"fixed": int(args.tune)}
    if cg is not None:
        line["cg_variant"] = cg
    if other in runs:
        o = runs[other]
        line["compare"] = {"precision": other, "value": o["value"], "ms_per_step": o["ms_per_step"],
                           "p50_ms": o["p50_ms"], "p99_ms": o["p99_ms"], "stage_ms": o["stage_ms"],
                           "e2e": o["e2e"]["value"]}
        line["speedup_mixed_vs_plain"] = (R["value"] / o["value"]) if tc else (o["value"] / R["value"])
    if rank == 0 and not args.no_cpu_baseline and args.workload == WORKLOAD:
        line["cpu_baseline"] = cpu_baseline(sample_fans=256, sample_pix=args.cpu_pix_baseline, n_freq=4)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def cpu_baseline(sample_fans=32, sample_pix=32768, seed=0, n_freq=1, cache=None):
    """The FP64 oracle, as it stands, on a bounded sample of one breast512 update, scaled to updates/s.

    Sample: (a) rays + gridding of `sample_fans` of the 256 fans (an element subset of the same ring
    and grid, same work per fan), scaled by 256/sample_fans; (b) Green's functions, Born adjoint,
    Hessian diagonal and Born forward at `n_freq` of the set's 4 frequencies on `sample_pix` of the
    262144 pixels, scaled by the pixel and frequency ratios."""
    from oracle import born, geometry, green, grid
    cfg = rbgen.breast512()
    inp = rbgen.make_inputs(cfg)
    g = geometry.from_config(cfg)
    gs = geometry.from_config(cfg, n_elem=sample_fans)
    t0 = time.perf_counter()
    grid.grid_pixels(gs, inp.c_init, inp.alpha0, np.arange(16))
    t_rays = time.perf_counter() - t0
    rng = np.random.default_rng(seed)
    sup = np.flatnonzero(geometry.support_mask(g).ravel())
    pix = np.sort(rng.choice(sup, sample_pix, replace=False))
    # tables at the sampled pixels for all fans (not timed: it repeats the timed ray work
    # above); a caller timing several steps on the same sample passes a cache
    key = (sample_pix, seed)
    if cache is not None and key in cache:
        tabs = cache[key]
    else:
        tabs = grid.grid_pixels(g, inp.c_init, inp.alpha0, pix)
        if cache is not None:
            cache[key] = tabs
    S = rng.standard_normal((g.n_elem, g.n_elem)) + 1j * rng.standard_normal((g.n_elem, g.n_elem))
    W = (rng.uniform(size=S.shape) > 0.25).astype(np.uint8)
    nf = len(cfg.sets[0])
    n_freq = max(1, min(n_freq, nf))
    t1 = time.perf_counter()
    for f in [cfg.freqs_hz[i] for i in cfg.sets[2][:n_freq]]:
        G = green.green(g, tabs, inp.c_init, f, pix=pix)
        born.born_adjoint(G, W * S, f)
        born.hess_diag(G, W, f)
        born.born_forward(G, rng.standard_normal(pix.size), f)
    t_born = time.perf_counter() - t1
    per_update = t_rays * (cfg.n_elem / sample_fans) + t_born * (g.npix / sample_pix) * (nf / n_freq)
    return {"value": 1.0 / per_update, "unit": "updates/s", "cores": _cores(), "kind": "oracle",
            "sample": f"rays+gridding of {sample_fans}/256 fans ({t_rays:.2f} s) and G+adjoint+Hessian+forward on "
                      f"{sample_pix}/262144 pixels at {n_freq} of 4 frequencies ({t_born:.2f} s), scaled to one "
                      f"update", "seconds_per_update_est": per_update, "t_rays": t_rays, "t_born": t_born}


def run_reference(args):
    """The FP64 oracle as it stands on the host cores.  A step is a fixed eighth of one
    breast512 update: rays and gridding of 32 of the 256 fans, and the Green's functions,
    Born adjoint, Hessian diagonal and Born forward at all 4 frequencies of a set on 32768
    of the 262144 pixels.  ms_per_step is the measured time of such a step; value (updates/s)
    is the eighth of an update it did over that time."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    frac = args.cpu_fans / 256.0
    pix = int(round(262144 * frac))
    times = []
    cache = {}   # one pixel sample for every step: its tables are built once, untimed
    for k in range(args.warmup + args.steps):
        cb = cpu_baseline(sample_fans=args.cpu_fans, sample_pix=pix, seed=0, n_freq=4, cache=cache)
        if k >= args.warmup:
            times.append(cb["t_rays"] + cb["t_born"])
    t_step = float(np.mean(times))
    v = frac / t_step
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "updates/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(WORKLOAD, args.prec, 1),
            "cpu_baseline": {"value": v, "unit": "updates/s", "cores": _cores(), "kind": "oracle",
                             "sample": f"each step {frac:g} of one update: " + cb["sample"].replace(
                                 ", scaled to one update", ""),
                             "update_fraction_per_step": frac},
            "e2e": {"value": v, "unit": "updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="bf16x3", choices=["fp32", "bf16x3"],
                    help="headline precision; the other one is measured beside it unless --no-compare")
    ap.add_argument("--no-compare", action="store_true")
    ap.add_argument("--workload", default=WORKLOAD, choices=["breast512", "breast256", "invivo512", "fullring1024", "tiny"],
                    help="the timed workload is breast512; smaller ones are for profiling captures")
    ap.add_argument("--cpu-fans", type=int, default=32,
                    help="reference arm: fans per step; the step does that fraction of an update (pixels alike)")
    ap.add_argument("--cpu-pix-baseline", type=int, default=160000,
                    help="cpu_baseline of the GPU arm's line: pixels sampled (all fans, all 4 frequencies)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tune", default="on",
                    help="on: run with the kernel-shape choice the tuner measures fastest on this problem (tuned "
                         "before the warm-up); off: the library's rule; an integer: that kernel-shape code "
                         "(rb_update_params.tune: 1 raster along tubes, 2 across; + 4 adjoint CTA pairs, + 8 one CTA "
                         "per tile)")
    ap.add_argument("--cg-iters", type=int, default=12,
                    help="also time the CG variant of the update with this many iterations (0: skip)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

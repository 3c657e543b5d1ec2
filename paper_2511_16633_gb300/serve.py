"""Batched and served reconstructions: many problems resident on one GPU at once.

Each admitted request is a ``Reconstruction`` with its own workspace, sound-speed
map and data on the device, and its own CUDA stream.  The runner issues a request's
next frequency-set update (``rb_hf_update``) as soon as the previous one has
finished, so the kernels of different requests run concurrently on the device: a
latency-bound ray trace of one request shares the SMs with another request's
contractions.  State stays resident across the sets of a request; only the
per-update diagnostics are read back.

Admission (continuous batching at frequency-set granularity): requests are taken
first come, first served, as soon as they have arrived, a slot is free and the HBM
footprint of the admitted requests (library workspace plus resident buffers, known
from ``rb_workspace_size`` before anything is allocated) stays within the budget;
a request that arrives while others are running joins as soon as one of them ends.

``python -m paper_2511_16633_gb300.serve`` measures a batch of uneven
reconstructions (all arriving at once) or a Poisson request stream, mixed precision
against the plain FP32 path, and prints one JSON line.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import math
import sys
import time
from typing import Callable, Dict, List, Optional, Sequence

import numpy as np

from . import rb


def precision_for(cfg, policy: str) -> int:
    """The contraction precision of a request: the tensor-core path (BF16 x3) where the
    ring size allows it (multiples of 64 up to 256 elements, and 512), else plain FP32."""
    if policy == "plain":
        return rb.RB_PREC_FP32
    return rb.RB_PREC_BF16X3 if rb.tc_supported(cfg.n_elem) else rb.RB_PREC_FP32


def footprint_bytes(cfg, prec: int) -> int:
    """Device bytes a request holds while admitted: the library workspace for its
    largest frequency set plus c, alpha0, dc (float32 grids) and its measured data
    (complex64 [n_freq][n_elem][n_elem])."""
    geom = rb.geometry_from_config(cfg)
    nf = max(len(s) for s in cfg.sets)
    ws = rb.rb_workspace_size(geom, nf, prec)
    if ws == 0:
        raise ValueError(f"{cfg.name}: unsupported sizes")
    grids = 3 * cfg.nx * cfg.ny * 4
    data = len(cfg.freqs_hz) * cfg.n_elem * cfg.n_elem * 8
    return int(ws + grids + data + 4096)


@dataclasses.dataclass
class Job:
    """One reconstruction request: its configuration, arrival time [s from the start],
    precision and footprint; the runner fills in the rest."""
    jid: int
    cfg: object
    arrival: float
    prec: int
    footprint: int
    admitted: Optional[float] = None
    done: Optional[float] = None
    updates: int = 0


class Scheduler:
    """Admission by arrival time, free slots and HBM footprint (host logic only).

    ``admit(now)`` returns the jobs to start now, in arrival order: a job is taken
    once it has arrived, while fewer than ``max_slots`` are active and its footprint
    fits in what the active jobs leave of ``budget``.  Admission is first come, first
    served: a job that does not fit blocks the ones behind it (no overtaking), so
    large requests are not starved.  A job larger than the whole budget is rejected.
    """

    def __init__(self, jobs: Sequence[Job], budget: int, max_slots: int):
        self.waiting = sorted(jobs, key=lambda j: (j.arrival, j.jid))
        self.budget, self.max_slots = int(budget), int(max_slots)
        self.active: Dict[int, Job] = {}
        self.started: List[Job] = []   # every admitted job, in admission order
        self.rejected: List[Job] = [j for j in self.waiting if j.footprint > self.budget]
        self.waiting = [j for j in self.waiting if j.footprint <= self.budget]

    @property
    def used(self) -> int:
        return sum(j.footprint for j in self.active.values())

    def admit(self, now: float) -> List[Job]:
        out = []
        while self.waiting and self.waiting[0].arrival <= now and len(self.active) < self.max_slots:
            j = self.waiting[0]
            if self.used + j.footprint > self.budget:
                break
            self.waiting.pop(0)
            j.admitted = now
            self.active[j.jid] = j
            self.started.append(j)
            out.append(j)
        return out

    def finish(self, job: Job, now: float) -> None:
        job.done = now
        del self.active[job.jid]

    def idle(self) -> bool:
        return not self.waiting and not self.active

    def next_arrival(self) -> Optional[float]:
        return self.waiting[0].arrival if self.waiting else None


@dataclasses.dataclass
class Problem:
    """Host-side inputs of a request (c_init, alpha0) and its measured data on the device."""
    c_init: np.ndarray
    alpha0: np.ndarray
    p_obs: object


def make_problem(cfg, device, data_prec: Optional[int] = None) -> Problem:
    """Seeded phantom, initial guess and synthetic data (the library's own ray-Born
    forward model about c_init plus 1 % noise), prepared before any timing."""
    import torch

    import rbgen
    from .recon import synth_data
    inp = rbgen.make_inputs(cfg)
    geom = rb.geometry_from_config(cfg)
    c0 = torch.as_tensor(inp.c_init, device=device).contiguous()
    a0 = torch.as_tensor(inp.alpha0, device=device).contiguous()
    ct = torch.as_tensor(inp.c_true, device=device).contiguous()
    prec = precision_for(cfg, "mixed") if data_prec is None else data_prec
    p = synth_data(geom, c0, ct, a0, list(cfg.freqs_hz), inp.noise_re, inp.noise_im, 0.01, prec)
    torch.cuda.synchronize(device)
    return Problem(inp.c_init, inp.alpha0, p)


class _Running:
    """An admitted job on its stream: the resident reconstruction, the next set, and
    the event that marks the end of the work in flight.

    With ``graphs`` the job's whole sweep (every set's update, in order) is captured
    into one CUDA graph on its stream at admission and replayed once: its 20-40
    launches per set leave the host as a single graph launch, and the library's
    side-stream fork and join become edges inside the graph, so the sweeps of
    different jobs share no stream.  Without it, one set is issued at a time."""

    def __init__(self, job: Job, prob: Problem, device, graphs: bool = False, autotune: bool = False):
        import torch

        from .recon import Reconstruction
        self.job = job
        self.stream = torch.cuda.Stream(device=device)
        with torch.cuda.stream(self.stream):
            self.rec = Reconstruction(job.cfg, prob.c_init, prob.alpha0, prob.p_obs, prec=job.prec, device=device,
                                      tune="auto" if autotune else rb.RB_TUNE_RULE)
        self.next_set = 0
        self.in_flight = 0
        self.event = None
        self.graph = None
        if graphs:
            self.graph = torch.cuda.CUDAGraph()
            with torch.cuda.stream(self.stream):
                self.graph.capture_begin()
                try:
                    for j in range(len(job.cfg.sets)):
                        self.rec.update(j, self.stream)
                finally:
                    self.graph.capture_end()

    def launch(self):
        """Issue the next set (or, with a graph, the whole sweep); returns the number of
        updates issued."""
        import torch
        if self.graph is not None:
            with torch.cuda.stream(self.stream):
                self.graph.replay()
            self.in_flight = len(self.job.cfg.sets) - self.next_set
        else:
            self.rec.update(self.next_set, self.stream)
            self.in_flight = 1
        self.next_set += self.in_flight
        self.event = torch.cuda.Event()
        self.event.record(self.stream)
        return self.in_flight

    def finished_set(self) -> bool:
        return self.event is not None and self.event.query()

    def more(self) -> bool:
        return self.next_set < len(self.job.cfg.sets)


def run(jobs: Sequence[Job], problems: Dict[int, Problem], budget: int, max_slots: int, device="cuda",
        keep: Optional[Callable[[Job, object], None]] = None, realtime: bool = True, graphs: bool = False,
        autotune: bool = False) -> dict:
    """Run the jobs under the scheduler; arrival times are honoured on the host clock
    (``realtime``) or ignored (every job available at once).  ``keep(job, c)`` receives
    each finished job's sound-speed map (a device tensor) before its buffers go.
    ``graphs``: each job's sweep is captured into one CUDA graph at admission and
    replayed (the capture counts in the job's latency).  ``autotune``: each job runs with
    the kernel-shape choice tune.py measured fastest for its shape (timed at the first
    admission of a shape, then cached).  Returns per-job times and the totals."""
    import torch
    sched = Scheduler([dataclasses.replace(j, arrival=j.arrival if realtime else 0.0) for j in jobs], budget,
                      max_slots)
    running: Dict[int, _Running] = {}
    t0 = time.perf_counter()
    n_updates = 0
    peak_used = 0
    while not sched.idle():
        now = time.perf_counter() - t0
        for j in sched.admit(now):
            r = _Running(j, problems[j.jid], device, graphs, autotune)
            running[j.jid] = r
            r.launch()
        peak_used = max(peak_used, sched.used)
        progressed = False
        for jid in list(running):
            r = running[jid]
            if not r.finished_set():
                continue
            progressed = True
            r.job.updates += r.in_flight
            n_updates += r.in_flight
            if r.more():
                r.launch()
            else:
                if keep is not None:
                    keep(r.job, r.rec.c)
                sched.finish(r.job, time.perf_counter() - t0)
                del running[jid]
                del r
        if not running and not progressed:
            nxt = sched.next_arrival()
            if nxt is not None:
                time.sleep(max(0.0, nxt - (time.perf_counter() - t0)))
    torch.cuda.synchronize(device)
    span = time.perf_counter() - t0
    done = [j for j in sched.started if j.done is not None]
    lat = np.array([j.done - j.arrival for j in done]) if done else np.zeros(1)
    return {"updates": n_updates, "seconds": span, "graphs": bool(graphs), "updates_per_s": n_updates / span if span > 0 else 0.0,
            "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "rejected": [j.cfg.name for j in sched.rejected], "peak_footprint_gb": peak_used / 1e9,
            "jobs": [{"name": j.cfg.name, "prec": "bf16x3" if j.prec == rb.RB_PREC_BF16X3 else "fp32",
                      "arrival_s": j.arrival, "admitted_s": j.admitted, "done_s": j.done, "updates": j.updates}
                     for j in done]}


def main():
    import torch

    import rbgen
    ap = argparse.ArgumentParser(description="batched / served ray-Born reconstructions on one GPU")
    ap.add_argument("--mode", choices=["batch", "serve"], default="batch")
    ap.add_argument("--n", type=int, default=16, help="reconstructions (batch) or requests (serve)")
    ap.add_argument("--rate", type=float, default=4.0, help="mean arrivals per second (serve)")
    ap.add_argument("--rings", default="128,256,512")
    ap.add_argument("--grids", default="256,512,768")
    ap.add_argument("--freqs", default="8,24", help="batch: frequency-count range")
    ap.add_argument("--sets", default="3,6", help="serve: frequency-set-count range")
    ap.add_argument("--slots", type=int, default=16)
    ap.add_argument("--budget-gb", type=float, default=0.0, help="0: free device memory minus 8 GB")
    ap.add_argument("--prec", choices=["mixed", "plain", "both"], default="both")
    ap.add_argument("--seed", type=int, default=20251116 + 4)
    ap.add_argument("--graphs", choices=["off", "on", "both"], default="off",
                    help="capture each request's sweep into one CUDA graph (both: measure each way)")
    ap.add_argument("--tune", choices=["off", "on", "both"], default="off",
                    help="run each request with the kernel-shape choice measured fastest for its shape (tuned "
                         "before the timed runs; both: measure with and without)")
    args = ap.parse_args()
    dev = torch.device("cuda:0")
    rings = tuple(int(x) for x in args.rings.split(","))
    grids = tuple(int(x) for x in args.grids.split(","))
    if args.mode == "batch":
        fr = tuple(int(x) for x in args.freqs.split(","))
        items = [(0.0, c) for c in rbgen.batch_mix(args.n, rings, grids, fr, seed=args.seed)]
    else:
        st = tuple(int(x) for x in args.sets.split(","))
        items = rbgen.poisson_requests(args.rate, args.n, rings, grids, st, seed=args.seed)
    free, _ = torch.cuda.mem_get_info(dev)
    budget = int(args.budget_gb * 1e9) if args.budget_gb > 0 else int(free - 8e9)
    problems = {}
    for k, (_, cfg) in enumerate(items):
        problems[k] = make_problem(cfg, dev)
        torch.cuda.empty_cache()
    out = {"mode": args.mode, "n": args.n, "budget_gb": budget / 1e9, "slots": args.slots,
           "workload": [c.name for _, c in items]}
    pols = ["mixed", "plain"] if args.prec == "both" else [args.prec]
    tunes = [False, True] if args.tune == "both" else [args.tune == "on"]
    if True in tunes:
        # the tuner's timings, per shape, before anything is timed (cached for the runs)
        from .recon import Reconstruction
        choices = {}
        for pol in pols:
            for k, (_, cfg) in enumerate(items):
                rec = Reconstruction(cfg, problems[k].c_init, problems[k].alpha0, problems[k].p_obs,
                                     prec=precision_for(cfg, pol), device=dev, tune="auto")
                choices[f"{cfg.name}/{pol}"] = rec.tune_info
                del rec
                torch.cuda.empty_cache()
        out["tune"] = choices
    for pol in pols:
        for gr in ([False, True] if args.graphs == "both" else [args.graphs == "on"]):
            for tu in tunes:
                jobs = [Job(k, cfg, t, precision_for(cfg, pol), footprint_bytes(cfg, precision_for(cfg, pol)))
                        for k, (t, cfg) in enumerate(items)]
                res = run(jobs, problems, budget, args.slots, dev, realtime=(args.mode == "serve"), graphs=gr,
                          autotune=tu)
                name = pol + ("_graphs" if gr and args.graphs == "both" else "") + \
                    ("_tuned" if tu and args.tune == "both" else "")
                out[name] = res
                torch.cuda.empty_cache()
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    sys.exit(main())

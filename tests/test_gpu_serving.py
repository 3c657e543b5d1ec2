"""Batched and served reconstructions on one GPU: each result is the same alone and in
the mix (bit for bit: every request has its own workspace and stream, and the kernels
are deterministic), and a Poisson request stream completes under a tight budget."""
import numpy as np
import pytest

import rbgen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2511_16633_gb300 import rb, serve  # noqa: E402


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rb.load()
    return torch.device("cuda:0")


def _cfgs():
    return [rbgen.tiny(),
            rbgen.tiny(n_elem=128, nx=70, ny=66, n_rays=48, seed=20251116 + 11),
            rbgen.tiny(n_elem=40, nx=66, ny=70, n_rays=45, seed=20251116 + 12),
            rbgen.tiny(n_elem=192, nx=64, ny=64, n_rays=64, seed=20251116 + 13),
            rbgen.tiny(n_elem=512, nx=64, ny=64, n_rays=64, seed=20251116 + 14)]


def _run(cfgs, problems, dev, policy, budget, slots, arrivals=None, realtime=False, graphs=False):
    jobs = [serve.Job(k, c, 0.0 if arrivals is None else arrivals[k], serve.precision_for(c, policy),
                      serve.footprint_bytes(c, serve.precision_for(c, policy))) for k, c in enumerate(cfgs)]
    out = {}
    res = serve.run(jobs, {j.jid: problems[j.jid] for j in jobs}, budget, slots, dev,
                    keep=lambda job, c: out.__setitem__(job.jid, c.cpu().numpy().copy()), realtime=realtime,
                    graphs=graphs)
    return out, res


@pytest.mark.parametrize("policy", ["mixed", "plain"])
def test_same_result_alone_and_in_the_mix(dev, policy):
    cfgs = _cfgs()
    problems = {k: serve.make_problem(c, dev) for k, c in enumerate(cfgs)}
    alone = {}
    for k, c in enumerate(cfgs):
        o, _ = _run([c], {0: problems[k]}, dev, policy, budget=1 << 40, slots=1)
        alone[k] = o[0]
    mixed, res = _run(cfgs, problems, dev, policy, budget=1 << 40, slots=len(cfgs))
    assert res["updates"] == sum(len(c.sets) for c in cfgs)
    for k in range(len(cfgs)):
        assert np.array_equal(mixed[k], alone[k]), k
        assert np.all(np.isfinite(mixed[k]))


def test_poisson_stream_under_a_tight_budget(dev):
    cfgs = _cfgs()
    problems = {k: serve.make_problem(c, dev) for k, c in enumerate(cfgs)}
    fps = [serve.footprint_bytes(c, serve.precision_for(c, "mixed")) for c in cfgs]
    budget = max(fps) + min(fps)            # at most two of them resident at once
    arrivals = [0.01 * k for k in range(len(cfgs))]
    out, res = _run(cfgs, problems, dev, "mixed", budget, slots=4, arrivals=arrivals, realtime=True)
    assert sorted(out) == list(range(len(cfgs)))
    assert res["peak_footprint_gb"] * 1e9 <= budget
    assert res["p99_s"] >= res["p50_s"] > 0
    for j in res["jobs"]:
        assert j["admitted_s"] >= j["arrival_s"] and j["done_s"] > j["admitted_s"]


def test_graph_mode_gives_the_eager_results(dev):
    """Each job's sweep captured into one CUDA graph and replayed, all jobs at once: the
    same maps, bit for bit, as the eager runner's."""
    cfgs = _cfgs()
    problems = {k: serve.make_problem(c, dev) for k, c in enumerate(cfgs)}
    eager, _ = _run(cfgs, problems, dev, "mixed", budget=1 << 40, slots=len(cfgs))
    graphed, res = _run(cfgs, problems, dev, "mixed", budget=1 << 40, slots=len(cfgs), graphs=True)
    assert res["graphs"] and res["updates"] == sum(len(c.sets) for c in cfgs)
    assert sorted(j["updates"] for j in res["jobs"]) == sorted(len(c.sets) for c in cfgs)
    for k in range(len(cfgs)):
        assert np.array_equal(graphed[k], eager[k]), k


@pytest.mark.parametrize("policy", ["mixed", "plain"])
def test_served_results_match_the_oracle(dev, policy):
    """Four requests of different rings and grids (64, 128 on a grid with a partial pixel
    tile, 40 and 192 elements) served at once, each fed the oracle's own synthetic data:
    every final sound-speed map within 0.05 m/s RMS of the oracle's sweep on that data."""
    from oracle import geometry as ogeom
    from oracle import update as oupd
    cfgs = _cfgs()[:4]
    problems, refs = {}, {}
    for k, c in enumerate(cfgs):
        inp = rbgen.make_inputs(c)
        g = ogeom.from_config(c)
        p = oupd.synth_data(g, inp.c_init, inp.c_true, inp.alpha0, c.freqs_hz, inp.noise_re, inp.noise_im)
        refs[k], _ = oupd.sweep(g, inp.c_init, inp.alpha0, c.freqs_hz, c.sets, p)
        problems[k] = serve.Problem(inp.c_init, inp.alpha0, torch.as_tensor(p.astype(np.complex64), device=dev))
    out, res = _run(cfgs, problems, dev, policy, budget=1 << 40, slots=len(cfgs))
    assert res["updates"] == sum(len(c.sets) for c in cfgs)
    for k, c in enumerate(cfgs):
        sup = ogeom.support_mask(ogeom.from_config(c))
        rms = float(np.sqrt(np.mean((out[k] - refs[k])[sup] ** 2)))
        print(f"served {c.name} ({policy}): c RMS difference to the oracle {rms:.3g} m/s")
        assert rms <= 0.05, (k, rms)


def test_autotuned_choice_is_bit_identical_and_cached(dev, tmp_path, monkeypatch):
    """The tuner's candidates (both raster mappings, both forms of the adjoint) give the
    same map bit for bit (the choice changes only the time); it returns one of them with
    a time for each, and the second call for the same shape comes from the cache (also
    written to RB_TUNE_CACHE)."""
    from paper_2511_16633_gb300 import tune
    from paper_2511_16633_gb300.recon import Reconstruction
    monkeypatch.setenv("RB_TUNE_CACHE", str(tmp_path / "tune.json"))
    monkeypatch.setattr(tune, "_cache", {})
    cfg = _cfgs()[1]
    prob = serve.make_problem(cfg, dev)
    maps = []
    cands = tune.candidates(rb.RB_PREC_BF16X3)
    for t in cands:
        rec = Reconstruction(cfg, prob.c_init, prob.alpha0, prob.p_obs, prec=rb.RB_PREC_BF16X3, device=dev, tune=t)
        maps.append(rec.sweep().cpu().numpy())
    assert all(np.array_equal(m, maps[0]) for m in maps[1:])
    rec = Reconstruction(cfg, prob.c_init, prob.alpha0, prob.p_obs, prec=rb.RB_PREC_BF16X3, device=dev, tune="auto")
    assert rec.tune in cands and set(rec.tune_info["ms_per_update"]) == {tune.name(t) for t in cands}
    assert np.array_equal(rec.sweep().cpu().numpy(), maps[0])
    monkeypatch.setattr(tune, "_cache", {})
    again = tune.cached(rec.geom, len(cfg.sets[0]), rb.RB_PREC_BF16X3)    # from the file
    assert again is not None and again["tune"] == rec.tune

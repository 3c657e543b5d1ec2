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

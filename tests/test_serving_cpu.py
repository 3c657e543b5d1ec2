"""Admission logic of the batched / served runner (host only, no GPU)."""
import pytest

from paper_2511_16633_gb300.serve import Job, Scheduler


def _jobs(spec):
    # spec: (arrival, footprint) per job
    return [Job(k, None, a, 0, f) for k, (a, f) in enumerate(spec)]


def test_admits_in_arrival_order_within_budget_and_slots():
    s = Scheduler(_jobs([(0.0, 4), (0.0, 4), (0.0, 4), (1.0, 1)]), budget=10, max_slots=8)
    first = s.admit(0.0)
    assert [j.jid for j in first] == [0, 1]          # the third does not fit (12 > 10)
    assert s.used == 8
    assert s.admit(0.5) == []                        # nothing new fits or has arrived
    s.finish(first[0], 0.7)
    assert [j.jid for j in s.admit(0.8)] == [2]      # freed memory goes to the next in line
    assert [j.jid for j in s.admit(1.0)] == [3]      # the later arrival fits beside them
    assert s.used == 9


def test_first_come_first_served_no_overtaking():
    s = Scheduler(_jobs([(0.0, 6), (0.1, 6), (0.2, 1)]), budget=10, max_slots=8)
    assert [j.jid for j in s.admit(0.0)] == [0]
    # job 1 does not fit; job 2 would, but must wait behind job 1
    assert s.admit(0.3) == []
    s.finish(s.active[0], 0.4)
    assert [j.jid for j in s.admit(0.5)] == [1, 2]


def test_slot_limit_and_rejection_of_oversized_jobs():
    s = Scheduler(_jobs([(0.0, 1)] * 5 + [(0.0, 100)]), budget=50, max_slots=3)
    assert len(s.admit(0.0)) == 3
    assert [j.jid for j in s.rejected] == [5]
    for j in list(s.active.values()):
        s.finish(j, 1.0)
    assert len(s.admit(1.0)) == 2
    for j in list(s.active.values()):
        s.finish(j, 2.0)
    assert s.idle()
    assert [j.jid for j in s.started] == [0, 1, 2, 3, 4]
    assert all(j.done is not None for j in s.started)


def test_next_arrival_and_idle():
    s = Scheduler(_jobs([(2.5, 1), (1.5, 1)]), budget=10, max_slots=2)
    assert s.next_arrival() == pytest.approx(1.5)
    assert s.admit(1.0) == [] and not s.idle()
    assert [j.jid for j in s.admit(3.0)] == [1, 0]


def test_precision_policy_covers_the_tensor_core_ring_sizes():
    import rbgen
    from paper_2511_16633_gb300 import rb, serve
    for n, tc in ((64, True), (96, False), (192, True), (256, True), (320, False), (512, True), (768, True),
                  (1024, True)):
        cfg = rbgen.ring(n, 128, 4)
        assert rb.tc_supported(n) == tc
        assert serve.precision_for(cfg, "mixed") == (rb.RB_PREC_BF16X3 if tc else rb.RB_PREC_FP32)
        assert serve.precision_for(cfg, "plain") == rb.RB_PREC_FP32


def test_tune_cache_keys_and_file_round_trip(tmp_path, monkeypatch):
    """The tuner's cache (host logic): one key per problem shape and precision, entries kept
    in memory and, with RB_TUNE_CACHE set, in a JSON file another process reads back."""
    import rbgen
    from paper_2511_16633_gb300 import rb, tune
    monkeypatch.setenv("RB_TUNE_CACHE", str(tmp_path / "tune.json"))
    monkeypatch.setattr(tune, "_cache", {})
    g1 = rb.geometry_from_config(rbgen.tiny())
    g2 = rb.geometry_from_config(rbgen.tiny(n_rays=48))
    assert tune.key(g1, 1, rb.RB_PREC_BF16X3) != tune.key(g2, 1, rb.RB_PREC_BF16X3)
    assert tune.key(g1, 1, rb.RB_PREC_BF16X3) != tune.key(g1, 1, rb.RB_PREC_FP32)
    assert tune.cached(g1, 1, rb.RB_PREC_BF16X3) is None
    assert len(tune.candidates(rb.RB_PREC_BF16X3)) == 4 and len(tune.candidates(rb.RB_PREC_FP32)) == 2
    assert tune.name(rb.RB_TUNE_RASTER_ACROSS | rb.RB_TUNE_ADJ_PAIR) == "raster across tubes, adjoint CTA pairs"
    entry = {"tune": rb.RB_TUNE_RASTER_ACROSS, "choice": "raster across tubes", "ms_per_update": {"a": 1.0, "b": 0.9}}
    tune._store_file(tune.key(g1, 1, rb.RB_PREC_BF16X3), entry)
    assert tune.cached(g1, 1, rb.RB_PREC_BF16X3) == entry
    assert tune.cached(g2, 1, rb.RB_PREC_BF16X3) is None

"""Autotuner host logic (no GPU): candidate hints are valid, the search picks
the fastest (ties to the smaller hint), the cache round-trips and a cache hit
runs nothing."""
import json

import numpy as np
import pytest

import paper_2102_11089_gb300 as L
from paper_2102_11089_gb300 import autotune as at
from paper_2102_11089_gb300 import workloads as wl


@pytest.mark.parametrize("entry", ["decode", "queue"])
@pytest.mark.parametrize("schedule", range(6))
def test_candidates_are_valid_hints(entry, schedule):
    if entry == "queue" and schedule not in (L.LMD_CIRBP, L.ME_CIRBP, L.ME_LMD_CIRBP):
        return
    c = at.candidates(entry, schedule)
    assert c and len(set(c)) == len(c)
    for t in c:
        assert t & ~0x1FF == 0 and t & 3 != 3
        at.describe(t)
    if entry == "queue" and schedule >= L.ME_CIRBP:
        assert {t >> 4 for t in c} == {0, 1, 2, 3} and {t & 3 for t in c} == {1, 2}
    with pytest.raises(ValueError):
        at.candidates("nope", schedule)


def test_search_picks_fastest_and_breaks_ties_low():
    calls = []
    cost = {0: 5.0, 4: 3.0, 8: 3.0, 12: 9.0}

    def run(t):
        calls.append(t)

    def timer(fn):
        fn()
        return cost[calls[-1]]

    best, times = at.search(run, [12, 8, 4, 0], repeats=2, timer=timer)
    assert best == 4 and times == {12: 9.0, 8: 3.0, 4: 3.0, 0: 5.0}
    assert len(calls) == 4 * 3  # one warm-up and two timed runs per candidate
    with pytest.raises(ValueError):
        at.search(run, [], timer=timer)


def test_cache_round_trip(tmp_path):
    path = str(tmp_path / "sub" / "tune.json")
    c = at.TuneCache(path)
    assert c.get("k") is None
    c.put("k", 18, {17: 2.5, 18: 1.25})
    assert at.TuneCache(path).get("k") == 18
    data = json.load(open(path))
    assert data["k"]["ms"] == {"17": 2.5, "18": 1.25}
    open(path, "w").write("{not json")
    assert at.TuneCache(path).get("k") is None


def _codes():
    d = wl.bg2_like(3)
    return [L.Code.from_protograph(d.shifts(Z), Z, d.info_cols * Z, d.punct_cols) for Z in (16, 32)]


def test_cache_key_separates_configurations():
    codes = _codes()
    p = L.make_params("me-lmd-cirbp", n_p=32)
    k1 = at.cache_key("queue1", "GB300", codes, p)
    assert k1 == at.cache_key("queue1", "GB300", codes, L.make_params("me-lmd-cirbp", n_p=32, seed=7))
    assert k1 != at.cache_key("queue1", "GB200", codes, p)
    assert k1 != at.cache_key("queue1", "GB300", codes[:1], p)
    assert k1 != at.cache_key("queue1", "GB300", codes, L.make_params("me-lmd-cirbp", n_p=64))
    assert k1 != at.cache_key("queue0", "GB300", codes, p)


def test_tune_queue_searches_once_then_hits_cache(tmp_path, monkeypatch):
    codes = _codes()
    seen = []

    def fake_queue(codes_, items, n, llr, params, **kw):
        seen.append(params.tune)

    monkeypatch.setattr(L, "decode_queue", fake_queue)
    cost = {t: 10.0 - (t >> 4) - 0.5 * (t & 3) for t in at.candidates("queue", L.ME_LMD_CIRBP)}

    def timer(fn):
        fn()
        return cost[seen[-1]]

    cache = at.TuneCache(str(tmp_path / "t.json"))
    p = L.make_params("me-lmd-cirbp", n_p=32)
    t = at.tune_queue(codes, None, 4, None, p, cache=cache, timer=timer, device="GB300", repeats=1)
    assert t == (3 << 4) | 2 and p.tune == t
    n = len(seen)
    assert n == 2 * len(cost)
    p2 = L.make_params("me-lmd-cirbp", n_p=32)
    assert at.tune_queue(codes, None, 4, None, p2, cache=cache, timer=timer, device="GB300") == t
    assert len(seen) == n and p2.tune == t

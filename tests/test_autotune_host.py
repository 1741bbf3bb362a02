"""The autotuner's host logic (no GPU): the coordinate search, the cache
file and its keys, and the tuning knobs' validation in the binding."""
import json

import pytest

from paper_0812_4547_gb300 import _binding as B
from paper_0812_4547_gb300 import autotune as T


def test_coordinate_search_finds_the_separable_minimum():
    cands = {"a": [0, 1, 2, 3], "b": [0, 5, 10]}

    def cost(t):  # separable bowl, minimum at a = 2, b = 5
        return (t.get("a", 0) - 2) ** 2 + abs(t.get("b", 0) - 5) + 1.0

    best, t_best, t_base, trials = T.coordinate_search(cost, ["a", "b"], cands, {"a": 0, "b": 0})
    assert best == {"a": 2, "b": 5} and t_best == 1.0
    assert t_base == cost({"a": 0, "b": 0}) and trials[0] == ({"a": 0, "b": 0}, t_base)
    # every candidate of each knob was timed once (the current value is not repeated)
    assert len(trials) == 1 + 3 + 2


def test_coordinate_search_keeps_the_base_when_nothing_is_faster():
    best, t_best, t_base, _ = T.coordinate_search(lambda t: 5.0 + sum(t.values()), ["a"], {"a": [0, 1, 2]},
                                                  {"a": 0})
    assert best == {"a": 0} and t_best == t_base == 5.0


def test_coordinate_search_skips_knobs_without_candidates():
    """A caller's candidate table may cover only some of the kind's knobs:
    the others keep their base value and are not timed."""
    seen = []

    def cost(t):
        seen.append(dict(t))
        return 1.0 + t.get("a", 0)

    best, _, _, trials = T.coordinate_search(cost, ["a", "missing"], {"a": [0, 1]}, {"a": 1, "missing": 7})
    assert best == {"a": 0, "missing": 7}
    # the base, a = 0, then a = 1 again against the new best; "missing" never varies
    assert all(t["missing"] == 7 for t in seen) and len(trials) == 3


def test_cache_round_trip_and_bad_files(tmp_path):
    p = str(tmp_path / "sub" / "tuning.json")
    assert T.load_cache(p) == {"version": T.CACHE_VERSION, "entries": {}}
    c = T.load_cache(p)
    key = T.cache_key("GPU X", "single", n=1024, d=64, r=4096)
    assert key == "GPU X|single|d=64,n=1024,r=4096"
    c["entries"][key] = {"tuning": {"gram_max_splits": 16}, "ms": 1.0, "default_ms": 2.0, "trials": []}
    T.save_cache(c, p)
    assert T.load_cache(p) == c
    with open(p, "w") as f:
        f.write("{not json")
    assert T.load_cache(p)["entries"] == {}
    with open(p, "w") as f:
        json.dump({"version": 999, "entries": {"x": 1}}, f)
    assert T.load_cache(p)["entries"] == {}


def test_candidates_are_valid_tuning_values():
    assert set(T.CANDIDATES) <= set(B.TUNING_KNOBS)
    for kind, knobs in T.KNOBS_FOR.items():
        assert set(knobs) <= set(T.CANDIDATES), kind
    for k, vals in T.CANDIDATES.items():
        assert 0 in vals  # the built-in default is always a candidate


def test_binding_rejects_unknown_knobs():
    with pytest.raises(ValueError):
        B.rnnls_set_tuning(0, {"no_such_knob": 1})

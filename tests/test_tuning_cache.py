"""The tiling cache of paper_2607_24141_gb300.tuning: keys by GPU, library build and
workload shape; a stored entry is applied without timing anything."""
import json

import pytest

import paper_2607_24141_gb300 as pz
from paper_2607_24141_gb300 import inputs as I
from paper_2607_24141_gb300 import tuning


class _Synth:
    def __init__(self, prob, batched=False, n_stars=1, precision=pz.PZ_MIXED):
        self.prob, self.batched, self.n_stars, self.precision = prob, batched, n_stars, precision


def test_shape_class_separates_workloads_and_ignores_details():
    a = I.small_config1(n_lambda_span_nm=2.0, seed=1)
    b = I.small_config1(n_lambda_span_nm=2.0, seed=2)          # same shape, other numbers
    c = I.small_config1(n_lambda_span_nm=8.0, seed=1)          # 4x the grid
    ka, kb, kc = (tuning.shape_class(_Synth(p)) for p in (a, b, c))
    assert ka == kb and ka != kc
    assert tuning.shape_class(_Synth(a, precision=pz.PZ_FP64)) != ka


def test_library_hash_is_stable():
    assert tuning.library_hash() == tuning.library_hash() and len(tuning.library_hash()) == 16


def test_store_and_load_round_trip(tmp_path):
    path = str(tmp_path / "sub" / "cache.json")
    assert tuning._load(path) == {}
    tuning._store(path, {"k": {"tiling": [4, 6, 4, 32, 5]}})
    assert json.load(open(path)) == {"k": {"tiling": [4, 6, 4, 32, 5]}}
    (tmp_path / "bad.json").write_text("not json")
    assert tuning._load(str(tmp_path / "bad.json")) == {}


@pytest.mark.gpu
def test_second_call_applies_the_stored_tiling(tmp_path):
    prob = I.small_config1(n_lambda_span_nm=3.0, seed=4)
    s = pz.Synthesizer(prob)
    path = str(tmp_path / "cache.json")
    first = tuning.autotune_cached(s, path, reps=1)
    assert not first["cached"] and first["candidates"] > 0
    second = tuning.autotune_cached(s, path, reps=1)
    assert second["cached"] and second["tiling"] == first["tiling"] and second["key"] == first["key"]
    f = s.forward()                                # the applied tiling runs
    assert bool((f > 0).all())
    s.close()


def test_forward_only_entries_have_their_own_key():
    """A tiling timed on the forward alone is stored under its own key, so that a context
    that runs the backward too never picks it up; the fwd+bwd key keeps three fields."""
    both = tuning.cache_key("GPU/152sm", "0123456789abcdef", "S1-p1-nd72-nl15-W11-lpp3")
    fwd = tuning.cache_key("GPU/152sm", "0123456789abcdef", "S1-p1-nd72-nl15-W11-lpp3", with_backward=False)
    assert both == "GPU/152sm|0123456789abcdef|S1-p1-nd72-nl15-W11-lpp3"
    assert fwd == both + "|fwd" and fwd != both


def test_committed_cache_entries_are_well_formed():
    data = tuning._load(tuning.DEFAULT_CACHE)
    assert data
    for key, entry in data.items():
        parts = key.split("|")
        assert len(parts) in (3, 4) and (len(parts) == 3 or parts[3] == "fwd"), key
        assert len(entry["tiling"]) == 5 and entry["fwd_ms"] > 0
        if len(parts) == 4:
            assert not entry["bwd_ms"]          # forward-only tuning times no backward

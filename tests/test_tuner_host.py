"""Host logic of the batch autotuner: candidate shapes per problem, size classes
and the JSON cache (no GPU: problems are meta tensors, timing is not exercised)."""
import json

import torch

from paper_2211_15634_gb300 import tuner


def prob(n):
    return {"T": torch.empty((n, n, n), device="meta")}


def test_fixed_and_zmarch_candidates_pass_through():
    assert tuner.tile_for(prob(100), (32, 8, 16)) == (32, 8, 16)
    assert tuner.tile_for(prob(100), tuner.ZMARCH_DEFAULT) == tuner.ZMARCH_DEFAULT


def test_row_packed_rule_spans_whole_interior_rows():
    # n = 100: interior rows of 98 columns; 256 columns -> 3 rows
    assert tuner.tile_for(prob(100), (0, 256, 16)) == (98, 3, 16)
    # never more rows than the interior has
    assert tuner.tile_for(prob(5), (0, 512, 32)) == (3, 3, 32)
    # at most 4096 columns per item
    tx, ty, tz = tuner.tile_for({"T": torch.empty((10, 400, 3000), device="meta")}, (0, 512, 32))
    assert tx == 2998 and tx * ty <= 4096 and ty >= 1


def test_size_classes_cover_every_extent_once():
    for n in (3, 47, 48, 79, 80, 111, 112, 143, 144, 160, 5000):
        lo, hi = tuner.size_class(prob(n))
        assert lo <= n < hi
    assert tuner.size_class({"T": torch.empty((3, 200, 50), device="meta")}) == (144, 1 << 30)


def test_cache_round_trip_and_corrupt_file(tmp_path, monkeypatch):
    path = tmp_path / "sub" / "tuner.json"
    monkeypatch.setenv("PS_TUNER_CACHE", str(path))
    assert tuner._load_cache() == {}
    tuner._save_cache({"GB300|f64|zmarch|48-80": [0, 0, 64]})
    assert json.loads(path.read_text()) == {"GB300|f64|zmarch|48-80": [0, 0, 64]}
    assert tuner._load_cache() == {"GB300|f64|zmarch|48-80": [0, 0, 64]}
    path.write_text("{not json")
    assert tuner._load_cache() == {}


def test_unwritable_cache_only_costs_retuning(tmp_path, monkeypatch):
    blocker = tmp_path / "file"
    blocker.write_text("x")
    monkeypatch.setenv("PS_TUNER_CACHE", str(blocker / "tuner.json"))  # parent is a file
    tuner._save_cache({"k": [1, 2, 3]})  # no exception
    assert tuner._load_cache() == {}

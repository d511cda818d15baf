"""The autotuner's JSON cache (trk_tuning_cache_*): host-only calls of the library, no device needed."""
import json

import pytest

from paper_1711_07999_gb300 import trk


@pytest.fixture(scope="module")
def lib():
    try:
        return trk.lib()
    except Exception as e:  # no nvcc / library on this host
        pytest.skip(f"library unavailable: {e}")


def test_store_and_lookup_round_trip(lib, tmp_path):
    p = str(tmp_path / "tune.json")
    assert trk.tuning_cache_lookup(p, "n16_p0_v800000_px4900000_L55") is None  # no file yet
    trk.tuning_cache_store(p, "n16_p0_v800000_px4900000_L55", dict(groups=4, assoc_blocks=608, tail_blocks=304), 5.25)
    trk.tuning_cache_store(p, "n64_p2_v6600000_px27000000_L70", dict(groups=1, assoc_blocks=1216, tail_blocks=152), 28.5)
    cfg, ms = trk.tuning_cache_lookup(p, "n16_p0_v800000_px4900000_L55")
    assert cfg == dict(groups=4, assoc_blocks=608, tail_blocks=304) and ms == pytest.approx(5.25)
    cfg, ms = trk.tuning_cache_lookup(p, "n64_p2_v6600000_px27000000_L70")
    assert cfg == dict(groups=1, assoc_blocks=1216, tail_blocks=152) and ms == pytest.approx(28.5)
    with open(p) as f:  # a plain JSON object keyed by size class
        data = json.load(f)
    assert set(data) == {"n16_p0_v800000_px4900000_L55", "n64_p2_v6600000_px27000000_L70"}
    assert data["n16_p0_v800000_px4900000_L55"]["groups"] == 4


def test_store_replaces_an_entry_and_keeps_the_others(lib, tmp_path):
    p = str(tmp_path / "tune.json")
    trk.tuning_cache_store(p, "a", dict(groups=2, assoc_blocks=304, tail_blocks=304), 1.0)
    trk.tuning_cache_store(p, "b", dict(groups=3, assoc_blocks=304, tail_blocks=304), 2.0)
    trk.tuning_cache_store(p, "a", dict(groups=8, assoc_blocks=1216, tail_blocks=608), 0.5)
    assert trk.tuning_cache_lookup(p, "a") == (dict(groups=8, assoc_blocks=1216, tail_blocks=608), 0.5)
    assert trk.tuning_cache_lookup(p, "b")[0]["groups"] == 3
    assert trk.tuning_cache_lookup(p, "c") is None


def test_malformed_cache_and_bad_signature(lib, tmp_path):
    p = tmp_path / "tune.json"
    p.write_text("{\n  \"x\": {\"groups\": 2}\n}\n")  # no block counts
    assert trk.tuning_cache_lookup(str(p), "x") is None
    with pytest.raises(trk.TrkError):
        trk.tuning_cache_store(str(p), 'bad"name', dict(groups=1, assoc_blocks=1, tail_blocks=1), 1.0)

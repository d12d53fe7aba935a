"""Host-side autotuner cache handling (no GPU): unreadable or partial cache
files count as empty, and writes replace the file whole."""

import json

from paper_1702_08159_gb300 import tune


def test_missing_and_corrupt_cache_read_as_empty(tmp_path):
    assert tune._read_cache(str(tmp_path / "absent.json")) == {}
    bad = tmp_path / "bad.json"
    bad.write_text('{"abc": {"grain": 4, "ms": ')  # a write cut short
    assert tune._read_cache(str(bad)) == {}
    lst = tmp_path / "list.json"
    lst.write_text("[1, 2]")
    assert tune._read_cache(str(lst)) == {}


def test_cache_roundtrip(tmp_path):
    p = tmp_path / "ok.json"
    p.write_text(json.dumps({"k": {"grain": 8, "ms": {"8": 1.0}}}))
    assert tune._read_cache(str(p))["k"]["grain"] == 8


def test_feature_and_grain_entries_share_one_file(tmp_path):
    p = str(tmp_path / "c.json")
    tune._write_cache(p, "a", {"grain": 4, "ms": {"4": 1.0}})
    tune._write_cache(p, "b", {"kind": "features", "rows_per_item": 2, "staged": 1,
                               "ms": {"2,1": 0.5}})
    data = tune._read_cache(p)
    assert data["a"]["grain"] == 4 and data["b"]["rows_per_item"] == 2

"""Host logic of bench.py: the DRAM traffic of a kernel is reported only
from a capture of the same kernel source and the same options."""
import json

import bench


def _write(tmp_path, entry):
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps({"wl/k_spread": entry}))


def test_traffic_needs_same_source_and_options(tmp_path, monkeypatch):
    opts = {"weights": "segment", "brick_z": 8, "records": True}
    _write(tmp_path, {"kernel_hash": "abc", "dram_bytes_per_launch": 123, "options": opts})
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "_kernel_hash", lambda: "abc")
    assert bench._traffic("wl") == 123
    assert bench._traffic("wl", options=dict(opts, autotuned=True)) == 123
    assert bench._traffic("wl", options=dict(opts, records=False)) is None
    assert bench._traffic("wl", options=dict(opts, brick_z=16)) is None
    assert bench._traffic("wl", "k_weights", opts) is None
    monkeypatch.setattr(bench, "_kernel_hash", lambda: "other")
    assert bench._traffic("wl", options=opts) is None


def test_committed_traffic_entries_are_well_formed():
    d = json.load(open(bench.os.path.join(bench.ROOT, "profiles", "traffic.json")))
    assert d
    for key, e in d.items():
        wl, kernel = key.split("/")
        assert kernel in ("k_spread", "k_weights", "k_bweights", "k_cm_spread", "k_cm_weights")
        assert e["dram_bytes_per_launch"] > 0 and len(e["kernel_hash"]) == 16
        assert {"weights", "brick_z", "records"} <= set(e["options"]) <= {"weights", "brick_z", "records",
                                                                          "column_march"}

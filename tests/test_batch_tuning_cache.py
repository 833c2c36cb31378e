"""The JSON cache of the batched kernel's autotuner (lbm.batch_tuned_threads), on the host:
the tuner and the block-size setter are replaced by recording fakes, so no GPU is needed."""
import json

from paper_2301_12869_gb300 import lbm


def test_cache_is_written_once_and_reused(tmp_path, monkeypatch):
    calls = {"tune": 0, "set": []}

    def fake_tune(b, steps=200):
        calls["tune"] += 1
        return 512, {128: 3.0, 256: 2.5, 512: 2.0}

    monkeypatch.setattr(lbm, "lbm_batch_autotune", fake_tune)
    monkeypatch.setattr(lbm, "lbm_batch_set_threads", lambda b, t: calls["set"].append(int(t)))
    path = str(tmp_path / "tune.json")
    assert lbm.batch_tuned_threads(None, path, "GB300|fp32|4x64..128|1024") == 512
    assert calls == {"tune": 1, "set": []}  # the tuner itself keeps its choice
    with open(path) as fh:
        stored = json.load(fh)
    assert stored["GB300|fp32|4x64..128|1024"]["threads"] == 512
    assert stored["GB300|fp32|4x64..128|1024"]["us_per_step"] == {"128": 3.0, "256": 2.5, "512": 2.0}
    # second use: no timing, the stored choice is applied
    assert lbm.batch_tuned_threads(None, path, "GB300|fp32|4x64..128|1024") == 512
    assert calls == {"tune": 1, "set": [512]}
    # another key is tuned and added next to the first
    assert lbm.batch_tuned_threads(None, path, "GB300|fp64|4x64..128|1024") == 512
    assert calls["tune"] == 2
    with open(path) as fh:
        assert sorted(json.load(fh)) == ["GB300|fp32|4x64..128|1024", "GB300|fp64|4x64..128|1024"]

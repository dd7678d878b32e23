"""The JSON timing cache that lets a calibration resume (no GPU)."""
import json

import pytest

from paper_1904_09538_gb300.timings import TimingCache

GB300_A = {"uuid": "GPU-a", "name": "GB300", "sm_clocks_mhz": "2070, 2070"}
GB300_B = {"uuid": "GPU-b", "name": "GB300", "sm_clocks_mhz": "2070, 2070"}


def test_round_trip_and_keys(tmp_path):
    path = str(tmp_path / "t.json")
    c = TimingCache(path, GB300_A)
    assert c.get("stream", {"N": 1024, "L": 2}, 10, True) is None
    c.put("stream", {"N": 1024, "L": 2}, 10, True, 1.5e-5)
    c.put("stream", {"L": 2, "N": 1024}, 10, False, 1.0e-5)      # flush is part of the key
    c.put("stream", {"N": 1024, "L": 2}, 60, True, 1.4e-5)       # so is the trial count
    c.save()
    d = TimingCache(path, GB300_A)
    assert d.get("stream", {"L": 2, "N": 1024}, 10, True) == 1.5e-5   # parameter order does not matter
    assert d.get("stream", {"N": 1024, "L": 2}, 10, False) == 1.0e-5
    assert d.get("stream", {"N": 1024, "L": 2}, 60, True) == 1.4e-5
    assert d.get("stream", {"N": 2048, "L": 2}, 10, True) is None
    assert d.hits == 3 and d.stored == 0


def test_devices_and_clock_settings_are_kept_apart(tmp_path):
    path = str(tmp_path / "t.json")
    a = TimingCache(path, GB300_A)
    a.put("fma", {"F": 1024}, 10, True, 2e-4)
    a.save()
    b = TimingCache(path, GB300_B)
    assert b.get("fma", {"F": 1024}, 10, True) is None
    b.put("fma", {"F": 1024}, 10, True, 3e-4)
    b.save()
    locked = TimingCache(path, dict(GB300_A, sm_clocks_mhz="2070, 1500"))
    assert locked.get("fma", {"F": 1024}, 10, True) is None
    assert TimingCache(path, GB300_A).get("fma", {"F": 1024}, 10, True) == 2e-4
    assert TimingCache(path, GB300_B).get("fma", {"F": 1024}, 10, True) == 3e-4
    assert len(json.load(open(path))["devices"]) == 2


def test_not_a_cache_is_refused(tmp_path):
    path = tmp_path / "x.json"
    path.write_text(json.dumps({"something": 1}))
    with pytest.raises(ValueError):
        TimingCache(str(path), GB300_A)

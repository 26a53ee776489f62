"""The autotuner's cache file on the host: a JSON object with one entry per
line, read and written by the library (pma_tune_cache_lookup / _store)."""
import json

import pytest

from paper_1504_00636_gb300 import binding


def test_cache_round_trip(tmp_path):
    path = str(tmp_path / "tune.json")
    k1 = "D=4 mixed flags=0 sms=152 h=0,0,20,0,0,0"
    k2 = "D=6 fp64 flags=4 sms=152 h=15,0,0,0,5,0"
    assert binding.pma_tune_cache_lookup(path, k1) is None  # no file yet
    binding.pma_tune_cache_store(path, k1, (256, 1024, 8191, 12, 0), 0.42)
    binding.pma_tune_cache_store(path, k2, (128, 512, 2048, 24, 1), 12.5)
    assert binding.pma_tune_cache_lookup(path, k1) == (256, 1024, 8191, 12, 0)
    assert binding.pma_tune_cache_lookup(path, k2) == (128, 512, 2048, 24, 1)
    # an update replaces the entry in place
    binding.pma_tune_cache_store(path, k1, (512, 1024, 4096, 16, 1), 0.40)
    assert binding.pma_tune_cache_lookup(path, k1) == (512, 1024, 4096, 16, 1)
    assert binding.pma_tune_cache_lookup(path, "D=4 mixed flags=0 sms=1 h=") is None
    # the file is plain JSON
    d = json.load(open(path))
    assert d[k1] == [512, 1024, 4096, 16, 1, 0.4] and d[k2][:5] == [128, 512, 2048, 24, 1]
    assert len(d) == 2


def test_cache_ignores_foreign_lines_and_refuses_bad_keys(tmp_path):
    path = tmp_path / "tune.json"
    path.write_text('{\n  "a b": [1, 2, 3, 12, 0, 4.5],\n  garbage line\n  "c": [7, 8]\n'
                    '  "d": [256, 1024, 8191, 0.4],\n  "e": [256, 1024, 8191, 12, 0.4]\n}\n')
    assert binding.pma_tune_cache_lookup(str(path), "a b") == (1, 2, 3, 12, 0)
    assert binding.pma_tune_cache_lookup(str(path), "c") is None  # malformed entry
    assert binding.pma_tune_cache_lookup(str(path), "d") is None  # no class base
    assert binding.pma_tune_cache_lookup(str(path), "e") is None  # no widen entry
    with pytest.raises(binding.PmaError):
        binding.pma_tune_cache_store(str(path), 'bad"key', (1, 2, 3, 12, 0), 1.0)

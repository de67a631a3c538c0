"""Host-side logic of the batch autotuner (no GPU)."""
from paper_1905_10574_gb300 import autotune


def test_buckets_and_signature():
    assert autotune.bucket_of(16, 16) == 0
    assert autotune.bucket_of(64, 65) == 1
    assert autotune.bucket_of(300, 20) == 3
    assert autotune.bucket_of(513, 2) == 4
    assert autotune.signature([(16, 16), (300, 20), (20, 300)]) == "b1-0-0-2-0"


def test_cache_roundtrip(tmp_path, monkeypatch):
    monkeypatch.setenv("XDG_CACHE_HOME", str(tmp_path))
    autotune._save_cache({"k": {"per_bucket": [32, 32, 48, 64, 64], "ms": 1.0}})
    assert autotune._load_cache()["k"]["per_bucket"][2] == 48

"""Autotuner keys and candidate sets (host only)."""
from paper_2312_10318_gb300 import tune as T


def test_buckets_and_keys():
    assert T.bucket(1000) == 1024 and T.bucket(1500) == 2048 and T.bucket(8) == 16
    assert T.key("f32", 1024, 1000) == "f32/periodic/1024x1024"
    assert T.key("f16", 64, 64, (True, False)) == "f16/general/64x64"
    assert T.key("f64", 64, 64, (True, True), True) == "f64/general/64x64"


def test_candidates():
    t = T.Tuner(cache_path="/nonexistent/x.json", persist=False)
    c = t.candidates("f32", 1024, (True, True), False)
    assert ("vector", 0) in c and ("scalar", 256) in c
    assert ("vector", 0) not in t.candidates("f32", 1022, (True, True), False)
    assert ("vector", 0) not in t.candidates("f16", 1024, (True, False), False)
    assert [tw for v, tw in t.candidates("f64", 20, (True, True), False) if v == "scalar"] == [32]

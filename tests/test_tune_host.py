"""Autotuner keys and candidate sets (host only)."""
from paper_2312_10318_gb300 import tune as T


def test_buckets_and_keys():
    assert T.bucket(1000) == 1024 and T.bucket(1500) == 2048 and T.bucket(8) == 16
    assert T.key("f32", 1024, 1000) == "f32/periodic/1024x1024"
    assert T.key("f16", 64, 64, (True, False)) == "f16/general/64x64"
    assert T.key("f64", 64, 64, (True, True), True) == "f64/general/64x64"
    assert T.key("f32", 4096, 4096, g_mode="current") == "f32/periodic/current/4096x4096"
    assert T.key("f32", 4096, 4096, g_mode="off") == "f32/periodic/4096x4096"


def test_candidates():
    t = T.Tuner(cache_path="/nonexistent/x.json", persist=False)
    c = t.candidates("f32", 1024, (True, True), False)
    assert ("vector", 0) in c and ("scalar", 256) in c
    assert ("vector", 0) not in t.candidates("f32", 1022, (True, True), False)
    assert ("vector", 0) not in t.candidates("f16", 1024, (True, False), False)
    assert [tw for v, tw in t.candidates("f64", 20, (True, True), False) if v == "scalar"] == [32]


def test_current_phi_candidates():
    """With Phi at the current level: the plain two-buffer kernel always, the
    column kernel on periodic lattices without a mask (not for F64_DW), the
    TMA-fed one (variant 'auto') for FP32 there; one candidate needs no
    measurement."""
    t = T.Tuner(cache_path="/nonexistent/x.json", persist=False)
    per = (True, True)
    assert t.candidates("f32", 4096, per, False, "current") == [("scalar", 0), ("auto", 0), ("column", 0)]
    assert t.candidates("f16", 4096, per, False, "current") == [("scalar", 0), ("column", 0)]
    assert t.candidates("f64", 4096, per, False, "current") == [("scalar", 0), ("column", 0)]
    assert t.candidates("f64dw", 4096, per, False, "current") == [("scalar", 0)]
    assert t.candidates("f32", 4096, (True, False), False, "current") == [("scalar", 0)]
    assert t.candidates("f32", 4096, per, True, "current") == [("scalar", 0)]
    # chosen without a measurement (no GPU here): one candidate, or FP64 AA
    assert t.choose("f32", 512, 512, (True, False), False, "current") == ("scalar", 0)
    assert t.choose("f64dw", 512, 512, per, False, "current") == ("scalar", 0)
    assert t.choose("f64", 512, 512) == ("scalar", 0)
    assert not t.measured

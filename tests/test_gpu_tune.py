"""The autotuner measures, caches and applies kernel shapes; results do not
depend on the shape chosen."""
import json

import numpy as np
import pytest

from paper_2312_10318_gb300 import tune as T
from paper_2312_10318_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_tuner_measures_caches_and_applies(gpu_lib, tmp_path):
    from paper_2312_10318_gb300 import Lattice
    path = str(tmp_path / "tune.json")
    t = T.Tuner(cache_path=path, steps=32, reps=2)
    v, tw = t.choose("f32", 256, 256)
    assert v in ("scalar", "vector") and tw in (0, 32, 64, 128, 256)
    v2, _ = t.choose("f64dw", 128, 64, (True, False))
    assert v2 == "scalar"                         # walls: only scalar kernels apply
    data = json.load(open(path))
    assert set(data) == {"f32/periodic/256x256", "f64dw/general/128x64"}
    assert all(x > 0 for x in data["f32/periodic/256x256"]["candidates"].values())
    # a second tuner reuses the cache without measuring
    t2 = T.Tuner(cache_path=path)
    assert t2.choose("f32", 250, 260) == (v, tw) and not t2.measured
    # applying a shape does not change the state (FP32: bit-identical)
    pr = W.taylor_green(256, 0.04, 300.0)
    a = Lattice(256, 256, pr.tau_s, tau_s2=pr.tau_s2, storage="f32").set_kernel("scalar", 64)
    b = Lattice(256, 256, pr.tau_s, tau_s2=pr.tau_s2, storage="f32")
    t.apply(b)
    for lat in (a, b):
        lat.init(pr.ux, pr.uy, pr.rho).step(37)
    assert np.array_equal(a.get_f(), b.get_f())


def test_tuner_chooses_among_current_phi_kernels(gpu_lib, tmp_path):
    """With Phi at the current level the tuner times the plain, column and (FP32)
    TMA-fed two-buffer kernels and applies the fastest: the lattice then steps
    with that kernel, bit for bit as when it is forced."""
    from paper_2312_10318_gb300 import Lattice
    t = T.Tuner(cache_path=str(tmp_path / "tune.json"), steps=16, reps=2)
    kind = {"scalar": "ab", "auto": "ab_tma_shared", "column": "ab_column"}
    for storage in ("f32", "f16"):
        n = 512
        v, tw = t.choose(storage, n, n, g_mode="current")
        cands = t.candidates(storage, n, (True, True), False, "current")
        assert (v, tw) in cands
        assert set(t.measured[f"{storage}/periodic/current/{n}x{n}"]) == {f"{a}:{b}" for a, b in cands}
        pr = W.double_shear_layer(n, re=1e4)
        a = Lattice(n, n, pr.tau_s, storage=storage, g_mode="current", **pr.lattice_kwargs())
        t.apply(a, pr.periodic)
        assert a.step_kernel() == kind[v]
        b = Lattice(n, n, pr.tau_s, storage=storage, g_mode="current", **pr.lattice_kwargs()).set_kernel(v)
        for lat in (a, b):
            lat.init(pr.ux, pr.uy).step(5)
        assert np.array_equal(a.get_f(), b.get_f()), storage

"""Host-side serving logic (no GPU): the seeded stream, memory accounting and the
precision guard's prediction."""
import math

import numpy as np
import pytest

from paper_2312_10318_gb300 import serve as S


def test_stream_is_seeded_and_in_range():
    a = S.make_stream(200, seed=1, rate=4.0)
    b = S.make_stream(200, seed=1, rate=4.0)
    assert [(r.kind, r.n, r.steps, r.storage, r.arrival) for r in a] == \
           [(r.kind, r.n, r.steps, r.storage, r.arrival) for r in b]
    assert all(64 <= r.n <= 4096 and r.n % 8 == 0 for r in a)
    assert all(1000 <= r.steps <= 20000 for r in a)
    assert all(1.0 <= r.re <= 1e6 for r in a)
    arr = np.array([r.arrival for r in a])
    assert (np.diff(arr) >= 0).all()
    # Poisson: mean inter-arrival 1/rate
    assert abs(np.diff(arr).mean() - 0.25) < 0.05
    assert set(r.storage for r in a) == {"f64", "f32", "f16"}
    # log-uniform sides: median near sqrt(64 * 4096) = 512
    assert 300 < np.median([r.n for r in a]) < 900


def test_lattice_bytes_formula():
    # 4096^2 FP32: 9 x 4 B populations + 2 x 2 x 4 B Phi per node (pitch 4096)
    b = S.lattice_bytes(4096, 4096, "f32")
    assert b - (36 + 16) * 4096 * 4096 < 1e5
    assert S.lattice_bytes(100, 10, "f16") >= (18 + 16) * 128 * 10


def test_summary_percentiles():
    res = [S.Result(i, "ok", "f32", 10, {}, 0.0, 0.0, float(i + 1)) for i in range(100)]
    s = S.summarize(res, makespan=100.0, node_updates=1e9)
    assert s["completed"] == 100 and s["solves_per_s"] == 1.0
    assert math.isclose(s["p50_s"], 50.5) and math.isclose(s["p99_s"], 99.01)
    assert math.isclose(s["mlups"], 10.0)


def test_spec_matches_problem_parameters():
    for kind in S.KINDS:
        for n, re in ((64, 10.0), (200, 3e5)):
            req = S.Request(0, kind, n, re, 10, "f32")
            pr, sp = S.problem_of(req), S.spec_of(req)
            assert (pr.nx, pr.ny, pr.periodic) == (sp.nx, sp.ny, sp.periodic)
            assert math.isclose(pr.tau_s, sp.tau_s, rel_tol=1e-15)
            assert math.isclose(pr.tau_s2, sp.tau_s2, rel_tol=1e-15)
            assert np.allclose(pr.g, sp.g, rtol=1e-15, atol=0)
            assert pr.mask is None


def test_guard_prediction_is_the_linear_fit_of_two_probe_points():
    """The guard's end-of-run prediction: with an error that grows as e0 + r t
    it is e0 + r * steps exactly; an error that shrinks is not extrapolated
    downwards (the growth rate is clamped at zero)."""

    class Fake:
        """A lattice whose RMS velocity difference to a resting shadow is
        err(t) times the speed scale."""

        def __init__(self, err):
            self.t, self.err = 0, err

        def step(self, n):
            self.t += n

        def compare(self, other):
            return {"rms_du": abs(self.err(self.t) - other.err(other.t)) * 0.04}

    zero = Fake(lambda t: 0.0)
    g = S.PrecisionGuard()
    e_end, pred = g._predict(1000, Fake(lambda t: 1e-6 + 2e-8 * t), zero, 0.04, 16)
    assert e_end == pytest.approx(1e-6 + 16 * 2e-8, rel=1e-12)
    assert pred == pytest.approx(1e-6 + 1000 * 2e-8, rel=1e-12)
    e_end, pred = g._predict(1000, Fake(lambda t: 1e-5 / (1 + t)), Fake(lambda t: 0.0), 0.04, 16)
    assert pred == pytest.approx(e_end, rel=1e-12) and e_end == pytest.approx(1e-5 / 17, rel=1e-12)


def test_stated_bound_grows_with_the_step_count_up_to_the_cap():
    """The stated end-of-run error of a reduced format is e0 + r n, capped at
    the accuracy every served result promises; the FP64 formats state 0."""
    for st, (e0, r) in S.STATED.items():
        assert S.stated_bound(st, 0) == pytest.approx(min(e0, S.ACCURACY_CAP))
        assert S.stated_bound(st, 1000) == pytest.approx(min(e0 + 1000 * r, S.ACCURACY_CAP))
        assert S.stated_bound(st, 10 ** 9) == S.ACCURACY_CAP
    assert S.stated_bound("f32", 20000) == pytest.approx(1e-6 + 2e-3)
    assert S.stated_bound("f64", 20000) == 0.0 and S.stated_bound("f64dw", 5) == 0.0
    # wider formats never state a larger error for the same run
    for n in (10, 1000, 20000):
        assert S.stated_bound("f32", n) <= S.stated_bound("f16", n) <= S.stated_bound("bf16", n)


class _FakeLattice:
    """Stands in for a Lattice in the guard's selection: its velocity error
    against the exact solution grows with the step count by a law per format."""
    ERR = {"f16": lambda t: 5e-4 + 5e-6 * t, "bf16": lambda t: 2e-3 + 2e-5 * t,
           "f32": lambda t: 1e-7 + 1e-8 * t, "f64": lambda t: 0.0, "f64dw": lambda t: 0.0}

    def __init__(self, storage, log):
        self.storage, self.t, self.log = storage, 0, log
        log.append(("make", storage))

    def step(self, n):
        self.t += n
        return self

    def compare(self, other):
        return {"rms_du": abs(self.ERR[self.storage](self.t) - self.ERR[other.storage](other.t)) * 0.04}


def _select(guard, storage, steps, err=None):
    from paper_2312_10318_gb300 import serve as S
    log = []
    if err:
        _FakeLattice.ERR = dict(_FakeLattice.ERR, **err)
    guard.release = lambda L: log.append(("release", L.storage))
    make = lambda st: _FakeLattice(st, log)
    def init(L):
        L.t = 0
        return L
    out = guard.select(make, init, storage, steps, 0.04)
    return out, log


def test_guard_measures_16_bit_formats_against_fp32_when_the_tolerance_allows():
    """The shadow of a 16-bit format is FP32 when the tolerance is at least 10x
    FP32's own stated error for the run, else the FP64 format; a widened solve
    reuses the FP32 shadow as its lattice; every lattice not returned is
    released."""
    from paper_2312_10318_gb300 import serve as S
    saved = dict(_FakeLattice.ERR)
    try:
        g = S.PrecisionGuard(fp64="f64dw")
        out, log = _select(g, "f16", 1000)                 # default bound: FP32 shadow, kept in FP16
        assert out.storage == "f16" and ("make", "f32") in log and ("make", "f64dw") not in log
        assert log.count(("release", "f32")) == 1
        assert g.shadow_format("f16", S.stated_bound("f16", 1000), 1000) == "f32"
        assert g.shadow_format("f16", 1e-4, 1000) == "f64dw"
        assert g.shadow_format("f16", S.stated_bound("f16", 20000), 20000) == "f64dw"   # FP32's bound grows too
        assert g.shadow_format("f32", 1.0, 1000) == "f64dw"
        strict = S.PrecisionGuard(tol=1e-9, fp64="f64dw")  # too tight for FP32: FP64-level shadow, to f64dw
        out, log = _select(strict, "f16", 1000)
        assert out.storage == "f64dw" and ("make", "f32") in log
        assert [e for e in log if e[0] == "make"].count(("make", "f64dw")) == 1
        assert ("release", "f32") in log
        # FP16 misses a tolerance FP32 meets: the FP32 shadow becomes the solve
        mid = S.PrecisionGuard(tol=0.0105, fp64="f64dw")
        out, log = _select(mid, "f16", 1000, err={"f16": lambda t: 2e-2})
        assert out.storage == "f32"
        assert [e for e in log if e[0] == "make"] == [("make", "f16"), ("make", "f32"), ("make", "f64dw")]
        assert ("release", "f64dw") in log and ("release", "f32") not in log
    finally:
        _FakeLattice.ERR = saved

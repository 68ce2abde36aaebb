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
